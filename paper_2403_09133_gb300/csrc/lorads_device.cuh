// Device building blocks of the LoRADS solver (sm_103a).
//
// Layout
//   * Factors are row-major n x ld, ld = 4 * ceil(r / 4); padding columns are kept at 0.
//   * A row is processed by a "team" of G lanes (G a power of two <= 32, aligned inside a
//     warp).  Lane l of a team owns the 4-element chunks c = l, l + G, ... (at most KMAX),
//     loaded as 128-bit accesses (float4, or two double2 for FP64).
//   * A constraint is a list of symmetric entries a (E_rc + E_cr) or a E_rr: one entry for
//     MaxCut (A_i = e_i e_i^T, Section 5.3) and matrix completion (Section 5.4), several for
//     general constraints (tr X = 1) and for the rank-one terms of sensor-network localisation
//     (Section 2.3), which assembly expands into their entries (s a a^T has s a_k a_l at (k, l)).
//     The entries are kept twice: in constraint order (con_ptr, con_r, con_c, con_a) for the
//     products <A_i, X Y^T>, and as a symmetric CSR over rows (both triangles) that carries the
//     constraint id, for the sparse-times-dense products.  Constraints with several entries
//     are also cut into chunks of at most CON_CHUNK entries (chunk_ptr; con_chunk gives each
//     constraint's chunks) so that a long constraint is summed by many teams.
//   * Reductions are deterministic: fixed shuffle trees inside warps, warps summed in order,
//     CTAs summed in order by the last CTA to arrive at the grid barrier.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lorads {

constexpr int KMAX = 2;      // chunks per lane
constexpr int CHUNK = 4;     // elements per chunk (16 B of float, 32 B of double)
constexpr int MAXRED = 12;   // values per reduction (the last slot carries the barrier status)
constexpr int MAXMEM = 8;    // L-BFGS memory cap
constexpr int CON_CHUNK = 32;  // entries per chunk of a multi-entry constraint

// ------------------------------------------------------------------------------------
// problem view
// ------------------------------------------------------------------------------------
struct DevProblem {
  int n, m;
  // entries in constraint order: constraint i owns entries con_ptr[i] .. con_ptr[i+1]-1
  const int* con_ptr;
  const int* con_r;
  const int* con_c;
  const double* con_a;
  const double* b;
  // some constraint has several entries; then the chunks (chunk_ptr into the entries,
  // con_chunk[i] .. con_chunk[i+1]-1 the chunks of constraint i) are set
  int a_multi;
  int nchunk;
  const int* chunk_ptr;
  const int* con_chunk;
  double* op_q;   // m values of scratch for the operator entry points (multi-entry only)
  // A as symmetric CSR over rows; entry e of row j: column A_col[e], constraint A_con[e]
  const int* A_rp;
  const int* A_col;
  const int* A_con;
  const double* A_val;
  const float* A_valf;
  // C as symmetric CSR over rows
  const int* C_rp;
  const int* C_col;
  const double* C_val;
  const float* C_valf;
  // row scaling of U_0 onto diagonal constraints (NULL unless every constraint is a single
  // diagonal entry on its own row with b/a > 0): U_0 row j gets norm row_norm[j] (< 0: keep)
  const double* row_norm;
  double b_inf, C_fro, C_inf;
  double b_one, c_one;   // ||b||_1 and ||vec(C)||_1 (the normalisations of Appendix B)
  // every constraint is a diagonal entry: the Hessian of eq. linU is row-local; then
  // row_con[j] is the constraint on row j (-1: none) and row_a[j] its value (0: none)
  int a_diag_only;
  const int* row_con;
  const double* row_a;
  const float* row_af;
  // every row carries exactly one diagonal constraint with b/a > 0 (n = m, row_norm set): the
  // feasible set of the Burer-Monteiro problem is a product of spheres (Phase III applies)
  int polish_ok;
};

template <typename T> __device__ __forceinline__ const T* cval(const DevProblem& P);
template <> __device__ __forceinline__ const double* cval<double>(const DevProblem& P) { return P.C_val; }
template <> __device__ __forceinline__ const float* cval<float>(const DevProblem& P) { return P.C_valf; }
template <typename T> __device__ __forceinline__ const T* rowa(const DevProblem& P);
template <> __device__ __forceinline__ const double* rowa<double>(const DevProblem& P) { return P.row_a; }
template <> __device__ __forceinline__ const float* rowa<float>(const DevProblem& P) { return P.row_af; }
template <typename T> __device__ __forceinline__ const T* aval(const DevProblem& P);
template <> __device__ __forceinline__ const double* aval<double>(const DevProblem& P) { return P.A_val; }
template <> __device__ __forceinline__ const float* aval<float>(const DevProblem& P) { return P.A_valf; }

// ------------------------------------------------------------------------------------
// teams and fragments
// ------------------------------------------------------------------------------------
struct Team {
  int G;          // lanes per row
  int lane;       // lane inside the team
  int id;         // team index inside the scope
  int count;      // teams in the scope
  int nc;         // chunks per row (ld / 4)
  unsigned mask;  // shuffle mask of the team's lanes
};

__host__ __device__ inline int team_size_for(int ld) {
  int nc = ld / CHUNK;
  int need = (nc + KMAX - 1) / KMAX;
  int G = 1;
  while (G < need) G <<= 1;
  return G > 32 ? 32 : G;
}

__device__ inline Team make_team(int ld, int tid, int nthreads, int mult = 1) {
  Team t;
  t.G = team_size_for(ld) * (mult > 0 ? mult : 1);
  if (t.G > 32) t.G = 32;
  t.lane = tid & (t.G - 1);
  t.id = tid / t.G;
  t.count = nthreads / t.G;
  t.nc = ld / CHUNK;
  int wl = threadIdx.x & 31;
  int base = wl & ~(t.G - 1);
  t.mask = (t.G == 32) ? 0xffffffffu : (((1u << t.G) - 1u) << base);
  return t;
}

template <typename T>
struct Frag {
  T v[KMAX][CHUNK];
};

template <typename T> __device__ __forceinline__ void load4(const T* p, T* o);
template <> __device__ __forceinline__ void load4<float>(const float* p, float* o) {
  float4 x = *reinterpret_cast<const float4*>(p);
  o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
}
template <> __device__ __forceinline__ void load4<double>(const double* p, double* o) {
  double2 x = reinterpret_cast<const double2*>(p)[0];
  double2 y = reinterpret_cast<const double2*>(p)[1];
  o[0] = x.x; o[1] = x.y; o[2] = y.x; o[3] = y.y;
}
template <typename T> __device__ __forceinline__ void store4(T* p, const T* o);
template <> __device__ __forceinline__ void store4<float>(float* p, const float* o) {
  *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
template <> __device__ __forceinline__ void store4<double>(double* p, const double* o) {
  reinterpret_cast<double2*>(p)[0] = make_double2(o[0], o[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(o[2], o[3]);
}

template <typename T>
__device__ __forceinline__ void frag_zero(Frag<T>& f) {
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
#pragma unroll
    for (int e = 0; e < CHUNK; ++e) f.v[k][e] = T(0);
}

template <typename T>
__device__ __forceinline__ void frag_load(Frag<T>& f, const T* base, long long row, int ld,
                                          const Team& t) {
  const T* p = base + row * (long long)ld;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    int c = t.lane + k * t.G;
    if (c < t.nc) {
      load4<T>(p + c * CHUNK, f.v[k]);
    } else {
#pragma unroll
      for (int e = 0; e < CHUNK; ++e) f.v[k][e] = T(0);
    }
  }
}

template <typename T>
__device__ __forceinline__ void frag_store(const Frag<T>& f, T* base, long long row, int ld,
                                           const Team& t) {
  T* p = base + row * (long long)ld;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    int c = t.lane + k * t.G;
    if (c < t.nc) store4<T>(p + c * CHUNK, f.v[k]);
  }
}

// convert between element types (FP64 master <-> FP32 shadow)
template <typename D, typename S>
__device__ __forceinline__ void frag_convert(Frag<D>& d, const Frag<S>& s) {
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
#pragma unroll
    for (int e = 0; e < CHUNK; ++e) d.v[k][e] = D(s.v[k][e]);
}

// lane-local partial dot product, accumulated in T
template <typename T>
__device__ __forceinline__ T frag_dot_local(const Frag<T>& a, const Frag<T>& b) {
  T s = T(0);
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
#pragma unroll
    for (int e = 0; e < CHUNK; ++e) s = fma(a.v[k][e], b.v[k][e], s);
  return s;
}

template <typename T>
__device__ __forceinline__ T team_sum(T x, const Team& t) {
  for (int off = t.G >> 1; off > 0; off >>= 1) x += __shfl_xor_sync(t.mask, x, off);
  return x;
}

template <typename T>
__device__ __forceinline__ T frag_dot(const Frag<T>& a, const Frag<T>& b, const Team& t) {
  return team_sum(frag_dot_local(a, b), t);
}

// y += alpha x
template <typename T>
__device__ __forceinline__ void frag_axpy(Frag<T>& y, T alpha, const Frag<T>& x) {
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
#pragma unroll
    for (int e = 0; e < CHUNK; ++e) y.v[k][e] = fma(alpha, x.v[k][e], y.v[k][e]);
}

// ------------------------------------------------------------------------------------
// counter-based random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) and the
// Box-Muller transform (Box and Muller, 1958)
// ------------------------------------------------------------------------------------
__host__ __device__ inline uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// output i (0-based) of the SplitMix64 stream seeded with key
__host__ __device__ inline uint64_t splitmix64_at(uint64_t key, uint64_t i) {
  return splitmix64_mix(key + (i + 1ULL) * 0x9E3779B97F4A7C15ULL);
}
// key of sub-stream s: 0 draws U_0, g >= 1 draws the columns of the g-th rank growth
__host__ __device__ inline uint64_t stream_key(uint64_t seed, uint64_t s) {
  return splitmix64_at(seed, s);
}
__device__ inline double uniform_open01(uint64_t key, uint64_t i) {
  return ((double)(splitmix64_at(key, i) >> 11) + 0.5) * 0x1.0p-53;
}
// standard normal number e of the stream: outputs 2e and 2e+1
__device__ inline double normal_at(uint64_t key, uint64_t e) {
  double u1 = uniform_open01(key, 2 * e);
  double u2 = uniform_open01(key, 2 * e + 1);
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// ------------------------------------------------------------------------------------
// scopes: one CTA, or the whole grid of a cooperative launch
// ------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct GridCtl {
  unsigned int count;
  unsigned int gen;
  int error;
  int pad;
  double result[MAXRED];
};

// Sum over the 32 lanes of a warp of K values (K a power of two, <= 16) by recursive halving:
// each round a lane keeps half of its remaining values and adds the partner's copy of that
// half (the partner keeps the other half), so after log2 K rounds a lane holds one value
// index, completed by a butterfly over the remaining lane offsets.  K - 1 + 5 - log2 K FP64
// adds per lane instead of 5 K (FP64 issues at a small fraction of the FP32 rate here).
// The order of the additions is fixed, so the sums are deterministic; lanes holding the same
// index hold bitwise equal sums.  Returns the index held in w[0].
template <int K>
__device__ __forceinline__ int warp_sum_scatter(double* w) {
  const int lane = threadIdx.x & 31;
  int ix = 0, off = 16;
#pragma unroll
  for (int h = K / 2; h >= 1; h >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double keep = up ? w[i + h] : w[i];
      const double give = up ? w[i] : w[i + h];
      w[i] = keep + __shfl_xor_sync(0xffffffffu, give, off);
    }
    if (up) ix += h;
    off >>= 1;
  }
#pragma unroll
  for (; off > 0; off >>= 1) w[0] += __shfl_xor_sync(0xffffffffu, w[0], off);
  return ix;
}

// the lane that stores the warp sum of its value index (the first of its group)
template <int K>
__device__ __forceinline__ bool scatter_writer() {
  return ((threadIdx.x & 31) & (32 / K - 1)) == 0;
}

template <int K>
__device__ __forceinline__ void block_reduce_k(double* v, int k, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double w[K];
#pragma unroll
  for (int i = 0; i < K; ++i) w[i] = i < k ? v[i] : 0.0;
  int ix = warp_sum_scatter<K>(w);
  if (scatter_writer<K>() && ix < k) red[warp * MAXRED + ix] = w[0];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < K; ++i) w[i] = (lane < nw && i < k) ? red[lane * MAXRED + i] : 0.0;
    ix = warp_sum_scatter<K>(w);
    if (scatter_writer<K>() && ix < k) red[32 * MAXRED + ix] = w[0];
  }
  __syncthreads();
  for (int i = 0; i < k; ++i) v[i] = red[32 * MAXRED + i];
}

// deterministic CTA-wide sum of k (< MAXRED) values; every thread receives the sums in v
__device__ inline void block_reduce(double* v, int k, double* red /* smem [33*MAXRED] */) {
  if (k <= 1) block_reduce_k<1>(v, k, red);
  else if (k <= 2) block_reduce_k<2>(v, k, red);
  else if (k <= 4) block_reduce_k<4>(v, k, red);
  else if (k <= 8) block_reduce_k<8>(v, k, red);
  else block_reduce_k<16>(v, k, red);
}

// Warp 0 of a CTA: the sum over nb CTAs of the k partials each left in partials[b * MAXRED + i],
// into red[32 * MAXRED + i].  Lane l adds the CTAs l, l + 32, ...; the loads of a lane are
// issued together (32 / K CTAs per round trip), then the lanes combine by warp_sum_scatter.
template <int K>
__device__ __forceinline__ void grid_partials_k(const double* partials, int k, int nb,
                                                double* red) {
  constexpr int TC = 32 / K;
  const int lane = threadIdx.x & 31;
  double w[K];
#pragma unroll
  for (int i = 0; i < K; ++i) w[i] = 0.0;
  for (int b0 = 0; b0 < nb; b0 += 32 * TC) {
    double buf[TC][K];
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      const int b = b0 + lane + 32 * t;
#pragma unroll
      for (int i = 0; i < K; ++i)
        buf[t][i] = (b < nb && i < k) ? __ldcg(partials + b * MAXRED + i) : 0.0;
    }
#pragma unroll
    for (int t = 0; t < TC; ++t)
#pragma unroll
      for (int i = 0; i < K; ++i) w[i] += buf[t][i];
  }
  const int ix = warp_sum_scatter<K>(w);
  if (scatter_writer<K>() && ix < k) red[32 * MAXRED + ix] = w[0];
}

// Scopes: the CTA's shared array `red` holds 34 rows of MAXRED doubles: rows 0..31 the
// per-warp sums of a reduction, row 32 its results, row 33 per-CTA scalar scratch for the
// solver (no __shared__ variables are declared inside solver functions, which several kernels
// instantiate).
struct BlockScope {
  double* red;
  __device__ double* scratch() const { return red + 33 * MAXRED; }
  __device__ int tid() const { return threadIdx.x; }
  __device__ int nthreads() const { return blockDim.x; }
  __device__ bool sync() {
    __syncthreads();
    return true;
  }
  __device__ bool reduce(double* v, int k) {
    block_reduce(v, k, red);
    return true;
  }
  __device__ bool is_leader() const { return threadIdx.x == 0; }
};

struct GridScope {
  double* red;             // shared memory (34 rows of MAXRED, see BlockScope)
  GridCtl* ctl;            // zeroed before launch
  double* partials;        // 2 * gridDim.x * MAXRED (two rounds, by barrier generation)
  long long spin_limit;    // polls before a barrier gives up
  int first = 0;           // the scope spans CTAs [first, first + nb) of a cooperative launch
  int nb = 0;              // (0: the whole grid)
  unsigned gen_next = 0;   // thread 0: the generation of its next barrier (ctl->gen starts at 0)

  __device__ int count() const { return nb > 0 ? nb : (int)gridDim.x; }
  __device__ double* scratch() const { return red + 33 * MAXRED; }
  __device__ int tid() const { return ((int)blockIdx.x - first) * blockDim.x + threadIdx.x; }
  __device__ int nthreads() const { return count() * blockDim.x; }
  __device__ bool is_leader() const { return (int)blockIdx.x == first && threadIdx.x == 0; }

  // Bounded barrier over the scope's CTAs.  With k > 0 it also sums, over CTAs in CTA order, the
  // CTA sums left in red[32*MAXRED + i] by block_reduce.  Arrival is an acq_rel increment of
  // ctl->count; the last CTA resets the count and releases the generation; the others poll
  // the generation with acquire loads (bounded).  Every CTA then loads all partials -- the
  // loads of one lane are issued together, eight CTAs at a time, so their L2 round trips
  // overlap -- and adds them in the same fixed order.
  // The partials of consecutive barriers go to two buffers chosen by the parity of the
  // barrier's generation: a CTA released early may reach the next reduction and store its
  // next partial while a later CTA still loads this round's, so one buffer would let the later
  // CTA add a value of the wrong round.  Two rounds suffice, since no CTA passes the next
  // barrier before every CTA has arrived there, that is, has finished reading this round.
  // Thread 0 knows the generation in advance (the one it saw released, plus one), so nothing
  // is loaded before the arrival: on the critical path are the arrival's atomic, the release's
  // visibility to the waiters and the load of the partials.  (Loading the generation first, as
  // a check, cost one more L2 round trip per barrier.  Per-CTA release flags that every CTA
  // polls, with no atomic, were slower: 152 CTAs polling 152 lines.)
  __device__ bool barrier(int k) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int ok = 1;
      unsigned parity = 0;
      if (lane == 0) {
        parity = gen_next & 1u;
        double* mine = partials + (size_t)parity * gridDim.x * MAXRED;
        for (int i = 0; i < k; ++i) mine[blockIdx.x * MAXRED + i] = red[32 * MAXRED + i];
        const unsigned my_gen = gen_next;
        gen_next = my_gen + 1u;
        const unsigned arrived = atom_add_acq_rel_u32(&ctl->count, 1u);
        if (arrived == (unsigned)count() - 1) {
          ctl->count = 0;
          red_add_release_u32(&ctl->gen, 1u);
        } else {
          long long it = 0;
          while (ld_acquire_u32(&ctl->gen) == my_gen) {
            if ((++it & 63) == 0 && ld_acquire_s32(&ctl->error)) {
              ok = 0;
              break;
            }
            if (it > spin_limit) {
              atomicExch(&ctl->error, 1);
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
        }
        red[32 * MAXRED + MAXRED - 1] = ok ? 0.0 : 1.0;
      }
      // lane 0's acquire orders the other lanes' loads through __syncwarp
      __syncwarp();
      parity = __shfl_sync(0xffffffffu, parity, 0);
      if (k > 0) {
        const int c = count();
        const double* pp = partials + ((size_t)parity * gridDim.x + first) * MAXRED;
        if (k <= 1) grid_partials_k<1>(pp, k, c, red);
        else if (k <= 2) grid_partials_k<2>(pp, k, c, red);
        else if (k <= 4) grid_partials_k<4>(pp, k, c, red);
        else if (k <= 8) grid_partials_k<8>(pp, k, c, red);
        else grid_partials_k<16>(pp, k, c, red);
      }
    }
    __syncthreads();
    return red[32 * MAXRED + MAXRED - 1] == 0.0;
  }

  __device__ bool sync() {
    __syncthreads();
    return barrier(0);
  }
  __device__ bool reduce(double* v, int k) {
    block_reduce(v, k, red);   // leaves CTA sums in red[32*MAXRED + i]
    bool ok = barrier(k);
    for (int i = 0; i < k; ++i) v[i] = red[32 * MAXRED + i];
    return ok;
  }
};

// The scope of a CTA group inside a batch launch: the grid scope's code, as a type of its own
// so that each kernel instantiates its own solver (no solver instantiation is reached from
// two kernels).
struct GroupScope : GridScope {};

// ------------------------------------------------------------------------------------
// per-row operators (shared by the solver and the operator entry points)
// ------------------------------------------------------------------------------------

// Hessian of eq. linU on row j with fixed factor W:
//   (H P)_j = rho * sum_{entries (j,k) of A_i} a q_i W_k + gamma P_j,
//   q_i = <A_i, P W^T> = a (P_j . W_k + P_k . W_j)   (off-diagonal)   or   a P_j . W_j.
// Returns the row in out; Pj is loaded by the caller (it is also needed for p.Hp).
template <typename T>
__device__ __forceinline__ void hessian_row(const DevProblem& P, const T* Wm, const T* Pm,
                                            int ld, int j, const Frag<T>& Pj, T rho, T gamma,
                                            const Team& t, Frag<T>& out) {
  Frag<T> Wj, acc;
  frag_load(Wj, Wm, j, ld, t);
  frag_zero(acc);
  const T* av = aval<T>(P);
  const int e0 = P.A_rp[j], e1 = P.A_rp[j + 1];
  for (int e = e0; e < e1; ++e) {
    const int k = P.A_col[e];
    const T a = av[e];
    if (k == j) {
      T q = a * frag_dot(Pj, Wj, t);
      frag_axpy(acc, a * q, Wj);
    } else {
      Frag<T> Wk, Pk;
      frag_load(Wk, Wm, k, ld, t);
      frag_load(Pk, Pm, k, ld, t);
      T q = a * team_sum(frag_dot_local(Pj, Wk) + frag_dot_local(Pk, Wj), t);
      frag_axpy(acc, a * q, Wk);
    }
  }
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk)
#pragma unroll
    for (int ee = 0; ee < CHUNK; ++ee) out.v[kk][ee] = fma(rho, acc.v[kk][ee], gamma * Pj.v[kk][ee]);
}

// (A^T(w) - C) W on row j, w_i = wb * b_i + wl * lambda_i + we * e_i (e may be NULL),
// plus gamma W_j.  All in T.
template <typename T>
__device__ __forceinline__ void spmm_row(const DevProblem& P, const T* Wm, int ld, int j,
                                         const double* lam, const double* e, double wb, double wl,
                                         double we, T gamma, const Team& t, Frag<T>& out) {
  Frag<T> acc;
  frag_zero(acc);
  const T* cv = cval<T>(P);
  {
    // four rows in flight: the column indices, then the rows, then the sums
    int q = P.C_rp[j];
    const int qe = P.C_rp[j + 1];
    for (; q + 4 <= qe; q += 4) {
      const int k0 = P.C_col[q], k1 = P.C_col[q + 1], k2 = P.C_col[q + 2], k3 = P.C_col[q + 3];
      const T c0 = cv[q], c1 = cv[q + 1], c2 = cv[q + 2], c3 = cv[q + 3];
      Frag<T> W0, W1, W2, W3;
      frag_load(W0, Wm, k0, ld, t);
      frag_load(W1, Wm, k1, ld, t);
      frag_load(W2, Wm, k2, ld, t);
      frag_load(W3, Wm, k3, ld, t);
      frag_axpy(acc, -c0, W0);
      frag_axpy(acc, -c1, W1);
      frag_axpy(acc, -c2, W2);
      frag_axpy(acc, -c3, W3);
    }
    for (; q < qe; ++q) {
      Frag<T> Wk;
      frag_load(Wk, Wm, P.C_col[q], ld, t);
      frag_axpy(acc, -cv[q], Wk);
    }
  }
  const T* av = aval<T>(P);
  const bool a_part = (wb != 0.0) || (lam != nullptr) || (e != nullptr);
  for (int q = a_part ? P.A_rp[j] : 0; q < (a_part ? P.A_rp[j + 1] : 0); ++q) {
    const int i = P.A_con[q];
    double w = wb * P.b[i];
    if (lam) w += wl * lam[i];
    if (e) w += we * e[i];
    Frag<T> Wk;
    frag_load(Wk, Wm, P.A_col[q], ld, t);
    frag_axpy(acc, (T)(w * (double)av[q]), Wk);
  }
  if (gamma != T(0)) {
    Frag<T> Wj;
    frag_load(Wj, Wm, j, ld, t);
    frag_axpy(acc, gamma, Wj);
  }
  out = acc;
}

// <a (E_rc + E_cr), U V^T> = a (U_r . V_c + U_c . V_r), or a U_r . V_r when r = c
// (team-cooperative; the value in every lane)
template <typename T>
__device__ __forceinline__ double sddmm_entry(const T* Um, const T* Vm, int ld, int r, int c,
                                              double a, const Team& t) {
  Frag<T> Ur, Vc;
  frag_load(Ur, Um, r, ld, t);
  frag_load(Vc, Vm, c, ld, t);
  T loc = frag_dot_local(Ur, Vc);
  if (r != c) {
    Frag<T> Uc, Vr;
    frag_load(Uc, Um, c, ld, t);
    frag_load(Vr, Vm, r, ld, t);
    loc += frag_dot_local(Uc, Vr);
  }
  return a * (double)team_sum(loc, t);
}

// <A_i, U V^T>: the sum over constraint i's entries (team-cooperative)
template <typename T>
__device__ __forceinline__ double sddmm_con(const DevProblem& P, const T* Um, const T* Vm, int ld,
                                            int i, const Team& t) {
  double s = 0.0;
  for (int e = P.con_ptr[i]; e < P.con_ptr[i + 1]; ++e)
    s += sddmm_entry<T>(Um, Vm, ld, P.con_r[e], P.con_c[e], P.con_a[e], t);
  return s;
}

// Hessian row of eq. linU for multi-entry constraints, from q_i = <A_i, P W^T> computed
// beforehand: (H P)_j = rho sum_{entries (j,k) of A_i} a q_i W_k + gamma P_j (one team)
template <typename T>
__device__ __forceinline__ void hessian_row_q(const DevProblem& P, const T* Wm, int ld, int j,
                                              const Frag<T>& Pj, const double* q, T rho, T gamma,
                                              const Team& t, Frag<T>& out) {
  Frag<T> acc;
  frag_zero(acc);
  const T* av = aval<T>(P);
  for (int e = P.A_rp[j]; e < P.A_rp[j + 1]; ++e) {
    Frag<T> Wk;
    frag_load(Wk, Wm, P.A_col[e], ld, t);
    frag_axpy(acc, av[e] * (T)q[P.A_con[e]], Wk);
  }
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk)
#pragma unroll
    for (int ee = 0; ee < CHUNK; ++ee) out.v[kk][ee] = fma(rho, acc.v[kk][ee], gamma * Pj.v[kk][ee]);
}

// ------------------------------------------------------------------------------------
// warp-split rows: one warp per row, S = 32/G sub-teams of G lanes; sub-team s takes the
// row's entries s, s+S, s+2S, ... two at a time (four rows in flight per sub-team), and the
// partial sums are combined over sub-teams with shuffles.  Used where rows carry many
// entries (matrix completion: ~785 per row at n = 40,000), which a single team would walk
// as a chain of dependent loads.
// ------------------------------------------------------------------------------------
struct WarpRow {
  Team st;     // the lane's sub-team
  int sub;     // sub-team index inside the warp
  int S;       // sub-teams per warp
  int warp;    // warp index inside the scope
  int nwarps;  // warps in the scope
};

__device__ inline WarpRow make_warp_row(int ld, int tid, int nthreads, int mult = 1) {
  WarpRow w;
  w.st = make_team(ld, threadIdx.x & 31, 32, mult);   // team ids 0..S-1 inside the warp
  w.sub = w.st.id;
  w.S = 32 / w.st.G;
  w.warp = tid >> 5;
  w.nwarps = nthreads >> 5;
  return w;
}

template <typename T>
__device__ __forceinline__ void frag_warp_combine(Frag<T>& f, int G) {
  __syncwarp();
#pragma unroll
  for (int k = 0; k < KMAX; ++k)
#pragma unroll
    for (int e = 0; e < CHUNK; ++e) {
      T x = f.v[k][e];
      for (int off = G; off < 32; off <<= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      f.v[k][e] = x;
    }
}

// contribution of one A entry (j,k,a) to (H P)_j: a q W_k, q = a (P_j.W_k + P_k.W_j)
template <typename T>
__device__ __forceinline__ void hess_entry(const T* Wm, const T* Pm, int ld, int j, int k, T a,
                                           const Frag<T>& Pj, const Frag<T>& Wj, const Team& t,
                                           Frag<T>& acc) {
  if (k == j) {
    const T q = a * frag_dot(Pj, Wj, t);
    frag_axpy(acc, a * q, Wj);
  } else {
    Frag<T> Wk, Pk;
    frag_load(Wk, Wm, k, ld, t);
    frag_load(Pk, Pm, k, ld, t);
    const T q = a * team_sum(frag_dot_local(Pj, Wk) + frag_dot_local(Pk, Wj), t);
    frag_axpy(acc, a * q, Wk);
  }
}

// (H P)_j = rho sum a q W_k + gamma P_j with the whole warp; out valid in every lane
template <typename T>
__device__ void hessian_row_warp(const DevProblem& P, const T* Wm, const T* Pm, int ld, int j,
                                 const Frag<T>& Pj, T rho, T gamma, const WarpRow& w,
                                 Frag<T>& out) {
  const Team& t = w.st;
  Frag<T> Wj, acc;
  frag_load(Wj, Wm, j, ld, t);
  frag_zero(acc);
  const T* av = aval<T>(P);
  const int e0 = P.A_rp[j], e1 = P.A_rp[j + 1];
  int e = e0 + w.sub;
  for (; e + w.S < e1; e += 2 * w.S) {
    const int k0 = P.A_col[e], k1 = P.A_col[e + w.S];
    const T a0 = av[e], a1 = av[e + w.S];
    if (k0 != j && k1 != j) {
      Frag<T> W0, P0, W1, P1;
      frag_load(W0, Wm, k0, ld, t);
      frag_load(P0, Pm, k0, ld, t);
      frag_load(W1, Wm, k1, ld, t);
      frag_load(P1, Pm, k1, ld, t);
      const T q0 = a0 * team_sum(frag_dot_local(Pj, W0) + frag_dot_local(P0, Wj), t);
      const T q1 = a1 * team_sum(frag_dot_local(Pj, W1) + frag_dot_local(P1, Wj), t);
      frag_axpy(acc, a0 * q0, W0);
      frag_axpy(acc, a1 * q1, W1);
    } else {
      hess_entry(Wm, Pm, ld, j, k0, a0, Pj, Wj, t, acc);
      hess_entry(Wm, Pm, ld, j, k1, a1, Pj, Wj, t, acc);
    }
  }
  if (e < e1) hess_entry(Wm, Pm, ld, j, P.A_col[e], av[e], Pj, Wj, t, acc);
  frag_warp_combine(acc, t.G);
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk)
#pragma unroll
    for (int ee = 0; ee < CHUNK; ++ee) out.v[kk][ee] = fma(rho, acc.v[kk][ee], gamma * Pj.v[kk][ee]);
}

// (A^T(w) - C) W on row j with the whole warp (same weights as spmm_row); out in every lane
template <typename T>
__device__ void spmm_row_warp(const DevProblem& P, const T* Wm, int ld, int j, const double* lam,
                              const double* e, double wb, double wl, double we, T gamma,
                              const WarpRow& w, Frag<T>& out) {
  const Team& t = w.st;
  Frag<T> acc;
  frag_zero(acc);
  const T* cv = cval<T>(P);
  for (int q = P.C_rp[j] + w.sub; q < P.C_rp[j + 1]; q += w.S) {
    Frag<T> Wk;
    frag_load(Wk, Wm, P.C_col[q], ld, t);
    frag_axpy(acc, -cv[q], Wk);
  }
  const T* av = aval<T>(P);
  const bool a_part = (wb != 0.0) || (lam != nullptr) || (e != nullptr);
  if (a_part) {
    const int q1 = P.A_rp[j + 1];
    int q = P.A_rp[j] + w.sub;
    for (; q + w.S < q1; q += 2 * w.S) {
      const int i0 = P.A_con[q], i1 = P.A_con[q + w.S];
      const int k0 = P.A_col[q], k1 = P.A_col[q + w.S];
      double c0 = wb * P.b[i0], c1 = wb * P.b[i1];
      if (lam) { c0 += wl * lam[i0]; c1 += wl * lam[i1]; }
      if (e) { c0 += we * e[i0]; c1 += we * e[i1]; }
      Frag<T> W0, W1;
      frag_load(W0, Wm, k0, ld, t);
      frag_load(W1, Wm, k1, ld, t);
      frag_axpy(acc, (T)(c0 * (double)av[q]), W0);
      frag_axpy(acc, (T)(c1 * (double)av[q + w.S]), W1);
    }
    if (q < q1) {
      const int i = P.A_con[q];
      double c = wb * P.b[i];
      if (lam) c += wl * lam[i];
      if (e) c += we * e[i];
      Frag<T> Wk;
      frag_load(Wk, Wm, P.A_col[q], ld, t);
      frag_axpy(acc, (T)(c * (double)av[q]), Wk);
    }
  }
  frag_warp_combine(acc, t.G);
  if (gamma != T(0)) {
    Frag<T> Wj;
    frag_load(Wj, Wm, j, ld, t);
    frag_axpy(acc, gamma, Wj);
  }
  out = acc;
}

// hessian_row_q with the whole warp (entries split across sub-teams); out in every lane
template <typename T>
__device__ void hessian_row_q_warp(const DevProblem& P, const T* Wm, int ld, int j,
                                   const Frag<T>& Pj, const double* q, T rho, T gamma,
                                   const WarpRow& w, Frag<T>& out) {
  const Team& t = w.st;
  Frag<T> acc;
  frag_zero(acc);
  const T* av = aval<T>(P);
  for (int e = P.A_rp[j] + w.sub; e < P.A_rp[j + 1]; e += w.S) {
    Frag<T> Wk;
    frag_load(Wk, Wm, P.A_col[e], ld, t);
    frag_axpy(acc, av[e] * (T)q[P.A_con[e]], Wk);
  }
  frag_warp_combine(acc, t.G);
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk)
#pragma unroll
    for (int ee = 0; ee < CHUNK; ++ee) out.v[kk][ee] = fma(rho, acc.v[kk][ee], gamma * Pj.v[kk][ee]);
}

}  // namespace lorads
