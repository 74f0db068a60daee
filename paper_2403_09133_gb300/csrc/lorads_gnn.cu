// Learned warm start: a 3-layer message-passing network over the cost graph that proposes
// the Phase II start (U_0, y_0) of LoRADS, with its forward and backward passes and Adam,
// all in this file's kernels.  Dense layers run on the tensor cores (tcgen05, BF16 in,
// FP32 accumulate); aggregation over the normalised adjacency runs on the CUDA cores.
//
// Network (widths: hidden 64, concatenation 128, heads 32 = r_max 16 + y):
//   H_0 = features, H_l = relu([H_{l-1}, A_hat H_{l-1}] Theta_l + b_l), l = 1..3
//   Z = H_3 Theta_u,  U_0 = rows of Z[:, :r] normalised,  y_0 = H_3 theta_y + b_y
// Loss (rotation invariant): mean over edges of (U_i.U_j - Xs_ij)^2 + beta mean (y_i - ys_i)^2.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lorads.h"
#include "lorads_device.cuh"
#include "lorads_gemm_tc.cuh"

using bf16 = __nv_bfloat16;

namespace lorads {
namespace gnn {

constexpr int HID = 64;
constexpr int CATW = 128;
constexpr int RMAX = 16;
constexpr int HEADW = 32;
constexpr int NRAND = 8;
constexpr int NLAYER = 3;
constexpr float BETA = 0.1f;
constexpr int LAYER_PARAMS = CATW * HID + HID;
constexpr int OFF_THU = NLAYER * LAYER_PARAMS;
constexpr int OFF_THY = OFF_THU + HID * RMAX;
constexpr int OFF_BY = OFF_THY + HID;
constexpr int NPARAM = OFF_BY + 1;

enum Epi { EPI_LAYER = 0, EPI_HEADS = 1, EPI_F32 = 2, EPI_WGRAD = 3 };

struct GemmArgs {
  const bf16* A;
  int lda, a_trans, a_cols;  // a_cols: valid source columns (rows of A^T when a_trans)
  const bf16* B;
  int ldb, b_trans, b_rows, b_cols;
  int rows;                  // nodes
  int epi;
  float* out;                // EPI_LAYER: S (ld HID); EPI_HEADS: Z|y (ld HEADW); EPI_F32: out (ld ldo)
  int ldo;
  bf16* out_h;               // EPI_LAYER: H (BF16, ld CATW)
  const float* bias;         // EPI_LAYER: b (HID); EPI_HEADS: b_y at bias[0]
  float* partial;            // EPI_WGRAD: [tile][128][N]
  int* err;
};

template <int N, int K>
__global__ void __launch_bounds__(128) tc_gemm_kernel(GemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + 128 * K * 2;
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  const int row0 = tile * 128;
  if (warp == 0) tc::tmem_alloc(&tmem_base, N);
  if (tid == 0) tc::mbar_init(&bar, 1);
  // A tile: 128 x K, K-major
  for (int idx = tid; idx < 128 * (K / 8); idx += 128) {
    const int m = idx / (K / 8), kc = (idx % (K / 8)) * 8;
    __align__(16) bf16 v[8];
    if (!g.a_trans) {
      const int row = row0 + m;
      if (row < g.rows && kc < g.a_cols) {
        *reinterpret_cast<uint4*>(v) = *reinterpret_cast<const uint4*>(g.A + (size_t)row * g.lda + kc);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16(0.f);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int node = row0 + kc + e;
        v[e] = (node < g.rows && m < g.a_cols) ? g.A[(size_t)node * g.lda + m] : __float2bfloat16(0.f);
      }
    }
    *reinterpret_cast<uint4*>(sA + tc::sw128_offset(m, kc, 128)) = *reinterpret_cast<uint4*>(v);
  }
  // B tile: N x K, K-major
  for (int idx = tid; idx < N * (K / 8); idx += 128) {
    const int nn = idx / (K / 8), kc = (idx % (K / 8)) * 8;
    __align__(16) bf16 v[8];
    if (!g.b_trans) {
      if (nn < g.b_rows && kc < g.b_cols) {
        *reinterpret_cast<uint4*>(v) = *reinterpret_cast<const uint4*>(g.B + (size_t)nn * g.ldb + kc);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16(0.f);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int node = row0 + kc + e;
        v[e] = (node < g.rows && nn < g.b_rows) ? g.B[(size_t)node * g.ldb + nn] : __float2bfloat16(0.f);
      }
    }
    *reinterpret_cast<uint4*>(sB + tc::sw128_offset(nn, kc, N)) = *reinterpret_cast<uint4*>(v);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = tmem_base;
  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, N);
    const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
    for (int s = 0; s < K / 16; ++s) {
      const uint32_t ka = (uint32_t)(s >> 2) * (128u * 128u) + (uint32_t)(s & 3) * 32u;
      const uint32_t kb = (uint32_t)(s >> 2) * (uint32_t)(N * 128) + (uint32_t)(s & 3) * 32u;
      tc::mma_bf16(taddr, tc::sw128_desc(a0 + ka), tc::sw128_desc(b0 + kb), idesc, s > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
  }
  const bool ok = tc::mbar_wait(&bar, 0, 1LL << 24);
  if (!ok && lane == 0) atomicExch(g.err, 1);
  tc::fence_after();
  const int m = warp * 32 + lane;
  const int row = row0 + m;
#pragma unroll
  for (int c0 = 0; c0 < N; c0 += 16) {
    float acc[16];
    tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
    if (g.epi == EPI_WGRAD) {
      float* pp = g.partial + ((size_t)tile * 128 + m) * N + c0;
#pragma unroll
      for (int i = 0; i < 16; ++i) pp[i] = acc[i];
    } else if (row < g.rows) {
      if (g.epi == EPI_LAYER) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float s = acc[i] + g.bias[c0 + i];
          g.out[(size_t)row * HID + c0 + i] = s;
          g.out_h[(size_t)row * CATW + c0 + i] = __float2bfloat16(fmaxf(s, 0.f));
        }
      } else if (g.epi == EPI_HEADS) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = c0 + i;
          g.out[(size_t)row * HEADW + c] = (c == RMAX) ? acc[i] + g.bias[0] : acc[i];
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) g.out[(size_t)row * g.ldo + c0 + i] = acc[i];
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, N);
}

template <int N, int K>
static cudaError_t launch_gemm(const GemmArgs& g, int tiles, cudaStream_t s) {
  const size_t smem = (size_t)128 * K * 2 + (size_t)N * K * 2 + 1024;
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<N, K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tc_gemm_kernel<N, K><<<tiles, 128, smem, s>>>(g);
  return cudaGetLastError();
}

// ---- features: z_i (8 normals), 1, log(1+deg), d/10, s, zeros ----
__global__ void features_kernel(int n, const float* deg, const float* dsum, const float* ssum,
                                unsigned long long key, bf16* cat0) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bf16* row = cat0 + (size_t)i * CATW;
    for (int c = 0; c < NRAND; ++c)
      row[c] = __float2bfloat16((float)normal_at(key, (uint64_t)i * NRAND + c));
    row[NRAND] = __float2bfloat16(1.f);
    row[NRAND + 1] = __float2bfloat16(log1pf(deg[i]));
    row[NRAND + 2] = __float2bfloat16(dsum[i] / 10.f);
    row[NRAND + 3] = __float2bfloat16(ssum[i]);
    for (int c = NRAND + 4; c < HID; ++c) row[c] = __float2bfloat16(0.f);
  }
}

// ---- aggregation: out[:, 64:128] = A_hat H (BF16 in, FP32 accumulate), warp per row ----
__global__ void agg_bf16_kernel(int n, const int* rp, const int* col, const float* val,
                                bf16* cat) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
       i += (gridDim.x * blockDim.x) >> 5) {
    float a0 = 0.f, a1 = 0.f;
    for (int q = rp[i]; q < rp[i + 1]; ++q) {
      const __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162*>(cat + (size_t)col[q] * CATW)[lane];
      const float w = val[q];
      a0 = fmaf(w, __bfloat162float(h.x), a0);
      a1 = fmaf(w, __bfloat162float(h.y), a1);
    }
    reinterpret_cast<__nv_bfloat162*>(cat + (size_t)i * CATW + HID)[lane] = __floats2bfloat162_rn(a0, a1);
  }
}

// ---- backward of the concatenation: dH = dCAT[:, :64] + A_hat dCAT[:, 64:] (FP32) ----
__global__ void agg_back_kernel(int n, const int* rp, const int* col, const float* val,
                                const float* dcat, float* dh) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
       i += (gridDim.x * blockDim.x) >> 5) {
    float a0 = dcat[(size_t)i * CATW + 2 * lane], a1 = dcat[(size_t)i * CATW + 2 * lane + 1];
    for (int q = rp[i]; q < rp[i + 1]; ++q) {
      const float* src = dcat + (size_t)col[q] * CATW + HID;
      a0 = fmaf(val[q], src[2 * lane], a0);
      a1 = fmaf(val[q], src[2 * lane + 1], a1);
    }
    dh[(size_t)i * HID + 2 * lane] = a0;
    dh[(size_t)i * HID + 2 * lane + 1] = a1;
  }
}

// ---- heads: U = Z[:, :r] / ||Z[:, :r]||, y = Zy[:, 16] ----
__global__ void normalize_kernel(int n, int r, const float* zy, float* U, float* nz, float* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* z = zy + (size_t)i * HEADW;
    float s = 0.f;
    for (int c = 0; c < r; ++c) s = fmaf(z[c], z[c], s);
    const float nrm = sqrtf(fmaxf(s, 1e-30f));
    for (int c = 0; c < RMAX; ++c) U[(size_t)i * RMAX + c] = c < r ? z[c] / nrm : 0.f;
    nz[i] = nrm;
    y[i] = z[RMAX];
  }
}

// ---- loss and d/dZ, d/dy (one thread per node over its graph entries; no atomics) ----
__global__ void loss_grad_kernel(int n, int r, int nedges, const int* rp, const int* col,
                                 const int* eid, const float* U, const float* nz, const float* y,
                                 const float* Xs, const float* ys, bf16* dhead, double* lpart) {
  __shared__ double red[33 * MAXRED];
  double lsum = 0.0;
  const float invE = 1.f / (float)nedges, invn = 1.f / (float)n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float ui[RMAX], du[RMAX];
    for (int c = 0; c < RMAX; ++c) {
      ui[c] = U[(size_t)i * RMAX + c];
      du[c] = 0.f;
    }
    for (int q = rp[i]; q < rp[i + 1]; ++q) {
      const int j = col[q];
      float d = 0.f;
      for (int c = 0; c < r; ++c) d = fmaf(ui[c], U[(size_t)j * RMAX + c], d);
      const float g = d - Xs[eid[q]];
      if (i < j) lsum += (double)g * g * invE;
      const float co = 2.f * g * invE;
      for (int c = 0; c < r; ++c) du[c] = fmaf(co, U[(size_t)j * RMAX + c], du[c]);
    }
    const float ry = y[i] - ys[i];
    lsum += (double)BETA * ry * ry * invn;
    float ud = 0.f;
    for (int c = 0; c < r; ++c) ud = fmaf(ui[c], du[c], ud);
    bf16* dh = dhead + (size_t)i * HID;
    for (int c = 0; c < HID; ++c) {
      float v = 0.f;
      if (c < r) v = (du[c] - ui[c] * ud) / nz[i];
      else if (c == RMAX) v = 2.f * BETA * ry * invn;
      dh[c] = __float2bfloat16(v);
    }
  }
  double v[1] = {lsum};
  block_reduce(v, 1, red);
  if (threadIdx.x == 0) lpart[blockIdx.x] = v[0];
}

// ---- dS = dH * (S > 0) -> BF16 ----
__global__ void relu_back_kernel(int n, const float* dh, const float* S, bf16* ds) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * HID;
       t += (size_t)gridDim.x * blockDim.x)
    ds[t] = __float2bfloat16(S[t] > 0.f ? dh[t] : 0.f);
}

// ---- deterministic sums: weight-gradient partials over tiles, bias gradients over nodes ----
__global__ void wgrad_sum_kernel(int tiles, int N, int mrows, const float* partial, float* out,
                                 int transpose_out) {
  // out[m][c] (or out[c][m]) = sum_t partial[t][m][c], m < mrows, c < N
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < mrows * N; idx += gridDim.x * blockDim.x) {
    const int m = idx / N, c = idx % N;
    double s = 0.0;
    for (int t = 0; t < tiles; ++t) s += partial[((size_t)t * 128 + m) * N + c];
    if (transpose_out) out[(size_t)c * mrows + m] = (float)s;
    else out[(size_t)m * N + c] = (float)s;
  }
}

__global__ void colsum_bf16_kernel(int n, int cols, const bf16* x, int ldx, float* out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += (double)__bfloat162float(x[(size_t)i * ldx + c]);
    out[c] = (float)s;
  }
}

// ---- BF16 operand copies of the FP32 parameters ----
__global__ void prepare_weights_kernel(const float* P, bf16* Bf, bf16* Bd, bf16* Bh, bf16* Bhd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int l = 0; l < NLAYER; ++l) {
    const float* th = P + l * LAYER_PARAMS;      // 128 x 64, [in][out]
    for (int idx = t; idx < CATW * HID; idx += nt) {
      const int k = idx / HID, c = idx % HID;
      Bf[(size_t)l * HID * CATW + (size_t)c * CATW + k] = __float2bfloat16(th[idx]);   // 64 x 128
      Bd[(size_t)l * CATW * HID + idx] = __float2bfloat16(th[idx]);                  // 128 x 64
    }
  }
  for (int idx = t; idx < HEADW * HID; idx += nt) {
    const int c = idx / HID, k = idx % HID;       // Bh: 32 x 64, row c = output column
    float v = 0.f;
    if (c < RMAX) v = P[OFF_THU + k * RMAX + c];
    else if (c == RMAX) v = P[OFF_THY + k];
    Bh[idx] = __float2bfloat16(v);
  }
  for (int idx = t; idx < HID * HID; idx += nt) {
    const int k = idx / HID, c = idx % HID;       // Bhd: 64 x 64, row k = hidden unit
    float v = 0.f;
    if (c < RMAX) v = P[OFF_THU + k * RMAX + c];
    else if (c == RMAX) v = P[OFF_THY + k];
    Bhd[idx] = __float2bfloat16(v);
  }
}

__global__ void adam_kernel(int np, float* P, const float* G, float* M, float* V, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

}  // namespace gnn
}  // namespace lorads

using namespace lorads;
using namespace lorads::gnn;

struct lorads_gnn {
  int device = 0;
  float* P = nullptr;   // NPARAM each: params, grads, Adam moments
  float* G = nullptr;
  float* M = nullptr;
  float* V = nullptr;
  bf16* Bf = nullptr;   // 3 x 64 x 128
  bf16* Bd = nullptr;   // 3 x 128 x 64
  bf16* Bh = nullptr;   // 32 x 64
  bf16* Bhd = nullptr;  // 64 x 64
  int* err = nullptr;
  long long step = 0;
  // graph
  int n = 0, nedges = 0;
  int *rp = nullptr, *col = nullptr, *eid = nullptr;
  float *val = nullptr, *deg = nullptr, *dsum = nullptr, *ssum = nullptr;
  unsigned long long feat_key = 0;
  // activations
  bf16* cat = nullptr;   // 4 x n x 128
  float* S = nullptr;    // 3 x n x 64
  float* zy = nullptr;   // n x 32
  float* U = nullptr;    // n x 16
  float* nz = nullptr;
  float* y = nullptr;
  float* Xs = nullptr;   // nedges
  float* ys = nullptr;   // n
  bf16* dhead = nullptr; // n x 64
  float* dh = nullptr;   // n x 64
  float* dcat = nullptr; // n x 128
  bf16* ds = nullptr;    // n x 64
  float* partial = nullptr;  // tiles x 128 x 64
  double* lpart = nullptr;
  std::vector<void*> graph_allocs;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LORADS_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? LORADS_ERR_NOMEM : LORADS_ERR_CUDA;
}
#define GCU(x)                                  \
  do {                                          \
    int _s = cuda_status(x);                    \
    if (_s != LORADS_OK) return _s;             \
  } while (0)

template <typename X>
int galloc(lorads_gnn* g, X** p, size_t count) {
  void* q = nullptr;
  GCU(cudaMalloc(&q, count * sizeof(X) + 16));
  g->graph_allocs.push_back(q);
  *p = static_cast<X*>(q);
  return LORADS_OK;
}

void free_graph(lorads_gnn* g) {
  for (void* q : g->graph_allocs) cudaFree(q);
  g->graph_allocs.clear();
  g->n = g->nedges = 0;
}

// normal numbers of the SplitMix64 stream (host side, same definition as the device)
double host_normal(uint64_t key, uint64_t e) {
  const double u1 = ((double)(splitmix64_at(key, 2 * e) >> 11) + 0.5) * 0x1.0p-53;
  const double u2 = ((double)(splitmix64_at(key, 2 * e + 1) >> 11) + 0.5) * 0x1.0p-53;
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
}

int forward_impl(lorads_gnn* g, int r, cudaStream_t s) {
  const int n = g->n, tiles = (n + 127) / 128;
  const int blocks = 4 * 152;
  prepare_weights_kernel<<<64, 256, 0, s>>>(g->P, g->Bf, g->Bd, g->Bh, g->Bhd);
  features_kernel<<<blocks, 256, 0, s>>>(n, g->deg, g->dsum, g->ssum, g->feat_key, g->cat);
  for (int l = 0; l < NLAYER; ++l) {
    bf16* cin = g->cat + (size_t)l * n * CATW;
    agg_bf16_kernel<<<blocks, 256, 0, s>>>(n, g->rp, g->col, g->val, cin);
    GemmArgs a{};
    a.A = cin; a.lda = CATW; a.a_trans = 0; a.a_cols = CATW;
    a.B = g->Bf + (size_t)l * HID * CATW; a.ldb = CATW; a.b_trans = 0; a.b_rows = HID; a.b_cols = CATW;
    a.rows = n; a.epi = EPI_LAYER; a.out = g->S + (size_t)l * n * HID;
    a.out_h = g->cat + (size_t)(l + 1) * n * CATW; a.bias = g->P + l * LAYER_PARAMS + CATW * HID;
    a.err = g->err;
    GCU((launch_gemm<HID, CATW>(a, tiles, s)));
  }
  GemmArgs h{};
  h.A = g->cat + (size_t)NLAYER * n * CATW; h.lda = CATW; h.a_trans = 0; h.a_cols = HID;
  h.B = g->Bh; h.ldb = HID; h.b_trans = 0; h.b_rows = HEADW; h.b_cols = HID;
  h.rows = n; h.epi = EPI_HEADS; h.out = g->zy; h.bias = g->P + OFF_BY; h.err = g->err;
  GCU((launch_gemm<HEADW, HID>(h, tiles, s)));
  normalize_kernel<<<blocks, 256, 0, s>>>(n, r, g->zy, g->U, g->nz, g->y);
  return cuda_status(cudaGetLastError());
}

// head gradients: theta_u[k][c] = gh[k][c] (c < RMAX), theta_y[k] = gh[k][RMAX], b_y = sum dy
__global__ void scatter_head_grads_kernel(const float* gh, const float* dysum, float* G) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < HID * HEADW; idx += gridDim.x * blockDim.x) {
    const int k = idx / HEADW, c = idx % HEADW;
    if (c < RMAX) G[OFF_THU + k * RMAX + c] = gh[idx];
    else if (c == RMAX) G[OFF_THY + k] = gh[idx];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) G[OFF_BY] = dysum[0];
}

int backward_impl(lorads_gnn* g, int r, cudaStream_t s) {
  const int n = g->n, tiles = (n + 127) / 128;
  const int blocks = 4 * 152;
  loss_grad_kernel<<<152, 256, 0, s>>>(n, r, g->nedges, g->rp, g->col, g->eid, g->U, g->nz,
                                       g->y, g->Xs, g->ys, g->dhead, g->lpart);
  GCU(cudaGetLastError());
  GCU(cudaMemsetAsync(g->G, 0, sizeof(float) * NPARAM, s));
  // heads: weight gradient H_3^T dhead (64 x 32) and dH_3 = dhead Bhd^T
  {
    GemmArgs w{};
    w.A = g->cat + (size_t)NLAYER * n * CATW; w.lda = CATW; w.a_trans = 1; w.a_cols = HID;
    w.B = g->dhead; w.ldb = HID; w.b_trans = 1; w.b_rows = HEADW; w.b_cols = 0;
    w.rows = n; w.epi = EPI_WGRAD; w.partial = g->partial; w.err = g->err;
    GCU((launch_gemm<HEADW, 128>(w, tiles, s)));
    wgrad_sum_kernel<<<8, 256, 0, s>>>(tiles, HEADW, HID, g->partial, g->dcat, 0);
    colsum_bf16_kernel<<<1, 32, 0, s>>>(n, 1, g->dhead + RMAX, HID, g->dcat + HID * HEADW);
    scatter_head_grads_kernel<<<8, 256, 0, s>>>(g->dcat, g->dcat + HID * HEADW, g->G);
    GemmArgs d{};
    d.A = g->dhead; d.lda = HID; d.a_trans = 0; d.a_cols = HID;
    d.B = g->Bhd; d.ldb = HID; d.b_trans = 0; d.b_rows = HID; d.b_cols = HID;
    d.rows = n; d.epi = EPI_F32; d.out = g->dh; d.ldo = HID; d.err = g->err;
    GCU((launch_gemm<HID, HID>(d, tiles, s)));
  }
  for (int l = NLAYER - 1; l >= 0; --l) {
    relu_back_kernel<<<blocks, 256, 0, s>>>(n, g->dh, g->S + (size_t)l * n * HID, g->ds);
    GemmArgs w{};
    w.A = g->cat + (size_t)l * n * CATW; w.lda = CATW; w.a_trans = 1; w.a_cols = CATW;
    w.B = g->ds; w.ldb = HID; w.b_trans = 1; w.b_rows = HID; w.b_cols = 0;
    w.rows = n; w.epi = EPI_WGRAD; w.partial = g->partial; w.err = g->err;
    GCU((launch_gemm<HID, 128>(w, tiles, s)));
    wgrad_sum_kernel<<<32, 256, 0, s>>>(tiles, HID, CATW, g->partial, g->G + l * LAYER_PARAMS, 0);
    colsum_bf16_kernel<<<1, 64, 0, s>>>(n, HID, g->ds, HID, g->G + l * LAYER_PARAMS + CATW * HID);
    if (l > 0) {
      GemmArgs d{};
      d.A = g->ds; d.lda = HID; d.a_trans = 0; d.a_cols = HID;
      d.B = g->Bd + (size_t)l * CATW * HID; d.ldb = HID; d.b_trans = 0; d.b_rows = CATW; d.b_cols = HID;
      d.rows = n; d.epi = EPI_F32; d.out = g->dcat; d.ldo = CATW; d.err = g->err;
      GCU((launch_gemm<CATW, HID>(d, tiles, s)));
      agg_back_kernel<<<blocks, 256, 0, s>>>(n, g->rp, g->col, g->val, g->dcat, g->dh);
    }
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" {

int lorads_gnn_param_count(void) { return NPARAM; }

int lorads_gnn_create(uint64_t seed, lorads_gnn** out) {
  if (!out) return LORADS_ERR_ARG;
  *out = nullptr;
  lorads_gnn* g = new (std::nothrow) lorads_gnn();
  if (!g) return LORADS_ERR_NOMEM;
  int st = LORADS_OK;
  do {
    if ((st = cuda_status(cudaGetDevice(&g->device))) != LORADS_OK) break;
    if ((st = cuda_status(cudaMalloc(&g->P, sizeof(float) * NPARAM * 4))) != LORADS_OK) break;
    g->G = g->P + NPARAM;
    g->M = g->G + NPARAM;
    g->V = g->M + NPARAM;
    if ((st = cuda_status(cudaMalloc(&g->Bf, sizeof(bf16) * (NLAYER * HID * CATW * 2 + HEADW * HID + HID * HID)))) != LORADS_OK) break;
    g->Bd = g->Bf + NLAYER * HID * CATW;
    g->Bh = g->Bd + NLAYER * CATW * HID;
    g->Bhd = g->Bh + HEADW * HID;
    if ((st = cuda_status(cudaMalloc(&g->err, 16))) != LORADS_OK) break;
    // weights ~ N(0, 1/fan_in) from SplitMix64 streams 2000 + l, 2100, 2101; biases 0
    std::vector<float> h(NPARAM, 0.f);
    for (int l = 0; l < NLAYER; ++l) {
      const uint64_t key = stream_key(seed, 2000 + l);
      for (int i = 0; i < CATW * HID; ++i)
        h[l * LAYER_PARAMS + i] = (float)(host_normal(key, i) / std::sqrt((double)CATW));
    }
    for (int i = 0; i < HID * RMAX; ++i)
      h[OFF_THU + i] = (float)(host_normal(stream_key(seed, 2100), i) / std::sqrt((double)HID));
    for (int i = 0; i < HID; ++i)
      h[OFF_THY + i] = (float)(host_normal(stream_key(seed, 2101), i) / std::sqrt((double)HID));
    if ((st = cuda_status(cudaMemcpy(g->P, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice))) != LORADS_OK) break;
    if ((st = cuda_status(cudaMemset(g->M, 0, sizeof(float) * NPARAM * 2))) != LORADS_OK) break;
    if ((st = cuda_status(cudaMemset(g->err, 0, 16))) != LORADS_OK) break;
  } while (false);
  if (st != LORADS_OK) {
    lorads_gnn_destroy(g);
    return st;
  }
  *out = g;
  return LORADS_OK;
}

int lorads_gnn_get_params(const lorads_gnn* g, float* params) {
  if (!g || !params) return LORADS_ERR_ARG;
  return cuda_status(cudaMemcpy(params, g->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
}

int lorads_gnn_set_params(lorads_gnn* g, const float* params) {
  if (!g || !params) return LORADS_ERR_ARG;
  for (int i = 0; i < NPARAM; ++i)
    if (!std::isfinite(params[i])) return LORADS_ERR_ARG;
  GCU(cudaMemcpy(g->P, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
  GCU(cudaMemset(g->M, 0, sizeof(float) * NPARAM * 2));
  g->step = 0;
  return LORADS_OK;
}

int lorads_gnn_load_graph(lorads_gnn* g, int64_t n, int64_t nedges, const int32_t* ei,
                          const int32_t* ej, const double* w, uint64_t feature_seed) {
  if (!g || n <= 0 || nedges < 0 || n > (1 << 26) || (nedges > 0 && (!ei || !ej || !w)))
    return LORADS_ERR_ARG;
  for (int64_t e = 0; e < nedges; ++e)
    if (ei[e] < 0 || ei[e] >= n || ej[e] < 0 || ej[e] >= n || ei[e] == ej[e] || !std::isfinite(w[e]))
      return LORADS_ERR_ARG;
  free_graph(g);
  // normalised adjacency (both directions) with edge ids; node statistics
  std::vector<double> dsum(n, 1.0), wsum(n, 0.0);
  std::vector<float> deg(n, 0.f);
  std::vector<int32_t> rp(n + 1, 0);
  for (int64_t e = 0; e < nedges; ++e) {
    dsum[ei[e]] += std::fabs(w[e]);
    dsum[ej[e]] += std::fabs(w[e]);
    wsum[ei[e]] += w[e];
    wsum[ej[e]] += w[e];
    deg[ei[e]] += 1.f;
    deg[ej[e]] += 1.f;
    rp[ei[e] + 1]++;
    rp[ej[e] + 1]++;
  }
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  std::vector<int32_t> col(2 * nedges), eid(2 * nedges), fill(rp.begin(), rp.end() - 1);
  std::vector<float> val(2 * nedges);
  for (int64_t e = 0; e < nedges; ++e) {
    const float a = (float)(w[e] / std::sqrt(dsum[ei[e]] * dsum[ej[e]]));
    int32_t q = fill[ei[e]]++;
    col[q] = ej[e]; eid[q] = (int32_t)e; val[q] = a;
    q = fill[ej[e]]++;
    col[q] = ei[e]; eid[q] = (int32_t)e; val[q] = a;
  }
  std::vector<float> fd(n), fs(n);
  for (int64_t i = 0; i < n; ++i) {
    fd[i] = (float)dsum[i];
    fs[i] = (float)(wsum[i] / dsum[i]);
  }
  g->n = (int)n;
  g->nedges = (int)nedges;
  g->feat_key = stream_key(feature_seed, 1000);
  const size_t tiles = (n + 127) / 128;
  int st;
  if ((st = galloc(g, &g->rp, n + 1)) || (st = galloc(g, &g->col, 2 * nedges + 1)) ||
      (st = galloc(g, &g->eid, 2 * nedges + 1)) || (st = galloc(g, &g->val, 2 * nedges + 1)) ||
      (st = galloc(g, &g->deg, n)) || (st = galloc(g, &g->dsum, n)) || (st = galloc(g, &g->ssum, n)) ||
      (st = galloc(g, &g->cat, (size_t)(NLAYER + 1) * n * CATW)) ||
      (st = galloc(g, &g->S, (size_t)NLAYER * n * HID)) || (st = galloc(g, &g->zy, (size_t)n * HEADW)) ||
      (st = galloc(g, &g->U, (size_t)n * RMAX)) || (st = galloc(g, &g->nz, n)) ||
      (st = galloc(g, &g->y, n)) || (st = galloc(g, &g->Xs, nedges + 1)) || (st = galloc(g, &g->ys, n)) ||
      (st = galloc(g, &g->dhead, (size_t)n * HID)) || (st = galloc(g, &g->dh, (size_t)n * HID)) ||
      (st = galloc(g, &g->dcat, (size_t)n * CATW + HID * HEADW + 64)) ||
      (st = galloc(g, &g->ds, (size_t)n * HID)) || (st = galloc(g, &g->partial, tiles * 128 * CATW)) ||
      (st = galloc(g, &g->lpart, 152)))
    return st;
  GCU(cudaMemcpy(g->rp, rp.data(), 4 * (n + 1), cudaMemcpyHostToDevice));
  if (nedges > 0) {
    GCU(cudaMemcpy(g->col, col.data(), 4 * 2 * nedges, cudaMemcpyHostToDevice));
    GCU(cudaMemcpy(g->eid, eid.data(), 4 * 2 * nedges, cudaMemcpyHostToDevice));
    GCU(cudaMemcpy(g->val, val.data(), 4 * 2 * nedges, cudaMemcpyHostToDevice));
  }
  GCU(cudaMemcpy(g->deg, deg.data(), 4 * n, cudaMemcpyHostToDevice));
  GCU(cudaMemcpy(g->dsum, fd.data(), 4 * n, cudaMemcpyHostToDevice));
  GCU(cudaMemcpy(g->ssum, fs.data(), 4 * n, cudaMemcpyHostToDevice));
  return LORADS_OK;
}

int lorads_gnn_forward(lorads_gnn* g, int32_t r, double* U0, double* y0, void* stream) {
  if (!g || g->n <= 0 || r < 1 || r > RMAX) return LORADS_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  GCU(cudaMemsetAsync(g->err, 0, 16, s));
  int st = forward_impl(g, r, s);
  if (st != LORADS_OK) return st;
  const int n = g->n;
  std::vector<float> hU((size_t)n * RMAX), hy(n);
  int herr = 0;
  GCU(cudaMemcpyAsync(hU.data(), g->U, sizeof(float) * n * RMAX, cudaMemcpyDeviceToHost, s));
  GCU(cudaMemcpyAsync(hy.data(), g->y, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
  GCU(cudaMemcpyAsync(&herr, g->err, 4, cudaMemcpyDeviceToHost, s));
  GCU(cudaStreamSynchronize(s));
  if (herr) return LORADS_ERR_DEVICE;
  if (U0)
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < r; ++c) U0[(size_t)i * r + c] = hU[(size_t)i * RMAX + c];
  if (y0)
    for (int i = 0; i < n; ++i) y0[i] = hy[i];
  return LORADS_OK;
}

int lorads_gnn_train_step(lorads_gnn* g, int32_t r, const double* Xs, const double* ys, double lr,
                          double* loss, float* grads, void* stream) {
  if (!g || g->n <= 0 || r < 1 || r > RMAX || !ys || (g->nedges > 0 && !Xs) || !(lr >= 0))
    return LORADS_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = g->n;
  std::vector<float> hx(g->nedges), hy(n);
  for (int e = 0; e < g->nedges; ++e) hx[e] = (float)Xs[e];
  for (int i = 0; i < n; ++i) hy[i] = (float)ys[i];
  GCU(cudaMemcpyAsync(g->Xs, hx.data(), 4 * (size_t)g->nedges, cudaMemcpyHostToDevice, s));
  GCU(cudaMemcpyAsync(g->ys, hy.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
  GCU(cudaMemsetAsync(g->err, 0, 16, s));
  int st = forward_impl(g, r, s);
  if (st != LORADS_OK) return st;
  st = backward_impl(g, r, s);
  if (st != LORADS_OK) return st;
  if (lr > 0) {
    g->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)g->step), c2 = 1.f - std::pow(b2, (float)g->step);
    adam_kernel<<<64, 256, 0, s>>>(NPARAM, g->P, g->G, g->M, g->V, (float)lr, b1, b2, 1e-8f, c1, c2);
    GCU(cudaGetLastError());
  }
  double lp[152];
  int herr = 0;
  GCU(cudaMemcpyAsync(lp, g->lpart, sizeof(lp), cudaMemcpyDeviceToHost, s));
  GCU(cudaMemcpyAsync(&herr, g->err, 4, cudaMemcpyDeviceToHost, s));
  if (grads) GCU(cudaMemcpyAsync(grads, g->G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s));
  GCU(cudaStreamSynchronize(s));
  if (herr) return LORADS_ERR_DEVICE;
  if (loss) {
    double t = 0.0;
    for (double v : lp) t += v;
    *loss = t;
  }
  return LORADS_OK;
}

void lorads_gnn_destroy(lorads_gnn* g) {
  if (!g) return;
  free_graph(g);
  if (g->P) cudaFree(g->P);
  if (g->Bf) cudaFree(g->Bf);
  if (g->err) cudaFree(g->err);
  delete g;
}

}  // extern "C"
