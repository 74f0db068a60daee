// Host runtime of the C ABI declared in include/lorads.h.
//
// lorads_problem keeps the caller's triplets on the host until the first solve or operator
// call, then assembles the device form once (see lorads_device.cuh: constraints in
// constraint order plus a symmetric CSR of A and of C), resolves the parameters and
// launches the persistent solver.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/lorads.h"
#include "lorads_kernels.cuh"

using namespace lorads;

namespace {

struct Rank1Term {
  int32_t con;
  std::vector<int32_t> idx;
  std::vector<double> a;
  double scale;
};

// where device memory comes from: the caller's allocator (lorads_params dev_alloc/dev_free)
// or cudaMalloc / cudaFree
struct DevAlloc {
  lorads_alloc_fn alloc = nullptr;
  lorads_free_fn free = nullptr;
  void* ctx = nullptr;
  void* stream = nullptr;
  static DevAlloc from(const lorads_params* prm, void* stream) {
    DevAlloc a;
    if (prm) {
      a.alloc = prm->dev_alloc;
      a.free = prm->dev_free;
      a.ctx = prm->alloc_ctx;
    }
    a.stream = stream;
    return a;
  }
  bool valid() const { return (alloc == nullptr) == (free == nullptr); }
  // nullptr when the memory cannot be had or is not 256-byte aligned
  void* get(size_t bytes) const {
    if (!alloc) {
      void* p = nullptr;
      if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      return p;
    }
    void* p = alloc(bytes, stream, ctx);
    if (p && (reinterpret_cast<uintptr_t>(p) & 255) != 0) {
      free(p, bytes, stream, ctx);
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t bytes) const {
    if (!p) return;
    if (free) free(p, bytes, stream, ctx);
    else cudaFree(p);
  }
};

// one device allocation carved into 256-byte aligned pieces; it remembers the allocator
// that made it and returns the block there
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  DevAlloc owner;
  void release() {
    if (base) owner.put(base, cap);
    base = nullptr;
    cap = used = 0;
  }
  int reserve(size_t bytes, const DevAlloc& al) {
    if (bytes <= cap) {
      used = 0;
      return LORADS_OK;
    }
    release();
    base = static_cast<char*>(al.get(bytes));
    if (!base) return LORADS_ERR_NOMEM;
    owner = al;
    cap = bytes;
    used = 0;
    return LORADS_OK;
  }
  template <typename X>
  X* take(size_t count) {
    size_t bytes = ((count * sizeof(X) + 255) / 256) * 256;
    X* p = reinterpret_cast<X*>(base + used);
    used += bytes;
    return p;
  }
  static size_t need(size_t count, size_t elem) { return ((count * elem + 255) / 256) * 256; }
};

}  // namespace

struct lorads_problem {
  int64_t n = 0, m = 0;
  int device = 0;
  // host triplets
  std::vector<int32_t> C_row, C_col;
  std::vector<double> C_val;
  std::vector<int32_t> A_con, A_row, A_col;
  std::vector<double> A_val;
  std::vector<Rank1Term> rank1;
  std::vector<double> b;
  bool has_b = false;
  // Phase II start (phase1 == 0): lorads_set_start (V = U) or lorads_set_state (a resume)
  int32_t start_r = 0;
  int32_t start_nz = 0;   // columns start_nz .. start_r-1 of the start are zero
  std::vector<double> start_U, start_V, start_lam;
  double start_rho = 0.0;
  bool has_start = false;
  bool start_resume = false;
  lorads_state start_state{};
  // device problem
  bool assembled = false;
  int assemble_status = LORADS_OK;
  Arena prob_mem;
  DevProblem dp{};
  bool diag_separable = false;
  double C_fro = 0, C_inf = 0, b_inf = 0, b_one = 0, c_one = 0;
  // solver state
  Arena state_mem;
  double* dU = nullptr;
  double* dV = nullptr;
  double* dUh = nullptr;
  double* dlam = nullptr;
  void* dargs = nullptr;  // SolverArgs<T> on the device
  SolveOut* dout = nullptr;
  GridCtl* dctl = nullptr;
  double* dpartials = nullptr;
  int* dqueue = nullptr;
  int sol_r = 0, sol_ld = 0;
  bool has_solution = false;
  lorads_result last{};
  SolveOut last_out{};
};

// ---------------------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------------------
// polls a grid or group barrier makes before it gives up and fails the solve
// (LORADS_ERR_DEVICE): the caller's limit, else about a few seconds of polling
static long long barrier_polls(const lorads_params* prm) {
  return prm->barrier_polls > 0 ? (long long)prm->barrier_polls : 50LL * 1000 * 1000;
}

static bool is_finite_value(double x) { return std::isfinite(x); }

static int check_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LORADS_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? LORADS_ERR_NOMEM : LORADS_ERR_CUDA;
}

#define CU(x)                                   \
  do {                                          \
    int _s = check_cuda(x);                     \
    if (_s != LORADS_OK) return _s;             \
  } while (0)

// 1 + the last column of the n x r row-major factors (V may be NULL) with a non-zero entry
static int32_t trailing_zero_from(const double* U, const double* V, int64_t n, int32_t r) {
  int32_t last = -1;
  for (int64_t j = 0; j < n; ++j)
    for (int32_t c = r - 1; c > last; --c)
      if (U[j * r + c] != 0.0 || (V != nullptr && V[j * r + c] != 0.0)) {
        last = c;
        break;
      }
  return last + 1;
}

static void invalidate(lorads_problem* p) {
  p->assembled = false;
  p->has_solution = false;
}

// Symmetric CSR (both triangles) from upper triplets; entry payload carried along.
struct SymEntry {
  int32_t row, col, con;
  double val;
};

static void build_sym_csr(int64_t n, std::vector<SymEntry>& ent, std::vector<int32_t>& rp,
                          std::vector<int32_t>& col, std::vector<int32_t>& con,
                          std::vector<double>& val) {
  std::sort(ent.begin(), ent.end(), [](const SymEntry& a, const SymEntry& b) {
    return a.row != b.row ? a.row < b.row : (a.col != b.col ? a.col < b.col : a.con < b.con);
  });
  rp.assign(n + 1, 0);
  for (const auto& e : ent) rp[e.row + 1]++;
  for (int64_t j = 0; j < n; ++j) rp[j + 1] += rp[j];
  col.resize(ent.size());
  con.resize(ent.size());
  val.resize(ent.size());
  for (size_t k = 0; k < ent.size(); ++k) {
    col[k] = ent[k].col;
    con[k] = ent[k].con;
    val[k] = ent[k].val;
  }
}

static void static_path_setup(int device);

// assemble the device form of (C, A, b)
static int assemble(lorads_problem* p, const DevAlloc& al) {
  if (p->assembled) return p->assemble_status;
  if (!p->has_b) return LORADS_ERR_STATE;
  if (cudaSetDevice(p->device) != cudaSuccess) return check_cuda(cudaGetLastError());
  const int64_t n = p->n, m = p->m;
  // Constraint entries in constraint order.  A sparse triplet (r, c, a) with r != c is the
  // symmetric entry a (E_rc + E_cr), so (r, c) and (c, r) are the same entry; a rank-one term
  // s a a^T expands into s a_k a_l at (k, l), k <= l (a's repeated indices summed first).
  struct ConEntry {
    int32_t con, r, c;
    double a;
  };
  std::vector<ConEntry> ce;
  ce.reserve(p->A_con.size());
  for (size_t t = 0; t < p->A_con.size(); ++t)
    ce.push_back({p->A_con[t], std::min(p->A_row[t], p->A_col[t]),
                  std::max(p->A_row[t], p->A_col[t]), p->A_val[t]});
  const size_t kMaxEntries = (size_t)1 << 29;   // the symmetric CSR indexes 2x with int32
  for (const auto& term : p->rank1) {
    std::vector<std::pair<int32_t, double>> av;
    for (size_t k = 0; k < term.idx.size(); ++k) av.push_back({term.idx[k], term.a[k]});
    std::sort(av.begin(), av.end());
    std::vector<std::pair<int32_t, double>> merged;
    for (const auto& x : av) {
      if (!merged.empty() && merged.back().first == x.first)
        merged.back().second += x.second;
      else
        merged.push_back(x);
    }
    const size_t sz = merged.size();
    if (ce.size() + sz * (sz + 1) / 2 > kMaxEntries) return LORADS_ERR_UNSUPPORTED;
    for (size_t k = 0; k < sz; ++k)
      for (size_t l = k; l < sz; ++l)
        ce.push_back({term.con, merged[k].first, merged[l].first,
                      term.scale * merged[k].second * merged[l].second});
  }
  if (ce.size() > kMaxEntries) return LORADS_ERR_UNSUPPORTED;
  std::sort(ce.begin(), ce.end(), [](const ConEntry& x, const ConEntry& y) {
    if (x.con != y.con) return x.con < y.con;
    return x.r != y.r ? x.r < y.r : x.c < y.c;
  });
  std::vector<int32_t> con_ptr(m + 1, 0), con_r, con_c;
  std::vector<double> con_a;
  for (size_t k = 0; k < ce.size();) {
    size_t l = k;
    double v = 0.0;
    for (; l < ce.size() && ce[l].con == ce[k].con && ce[l].r == ce[k].r && ce[l].c == ce[k].c; ++l)
      v += ce[l].a;
    if (v != 0.0) {
      con_r.push_back(ce[k].r);
      con_c.push_back(ce[k].c);
      con_a.push_back(v);
      con_ptr[ce[k].con + 1]++;
    }
    k = l;
  }
  bool multi = false;
  for (int64_t i = 0; i < m; ++i) {
    if (con_ptr[i + 1] == 0) return LORADS_ERR_ARG;   // A_i = 0
    multi = multi || con_ptr[i + 1] > 1;
    con_ptr[i + 1] += con_ptr[i];
  }
  const size_t nent = con_a.size();
  // chunks of at most CON_CHUNK entries per constraint (multi-entry problems)
  std::vector<int32_t> chunk_ptr(1, 0), con_chunk(m + 1, 0);
  if (multi) {
    for (int64_t i = 0; i < m; ++i) {
      for (int32_t e = con_ptr[i]; e < con_ptr[i + 1]; e += CON_CHUNK)
        chunk_ptr.push_back(std::min(e + CON_CHUNK, con_ptr[i + 1]));
      con_chunk[i + 1] = (int32_t)chunk_ptr.size() - 1;
    }
  }
  const int64_t nchunk = (int64_t)chunk_ptr.size() - 1;
  // A as symmetric CSR
  std::vector<SymEntry> ent;
  ent.reserve(2 * nent);
  for (int64_t i = 0; i < m; ++i)
    for (int32_t e = con_ptr[i]; e < con_ptr[i + 1]; ++e) {
      ent.push_back({con_r[e], con_c[e], (int32_t)i, con_a[e]});
      if (con_r[e] != con_c[e]) ent.push_back({con_c[e], con_r[e], (int32_t)i, con_a[e]});
    }
  std::vector<int32_t> A_rp, A_col, A_con;
  std::vector<double> A_val;
  build_sym_csr(n, ent, A_rp, A_col, A_con, A_val);
  // C: merge duplicates, both triangles
  std::vector<SymEntry> cent;
  {
    std::vector<int64_t> co(p->C_row.size());
    std::iota(co.begin(), co.end(), 0);
    std::sort(co.begin(), co.end(), [&](int64_t a, int64_t b) {
      return p->C_row[a] != p->C_row[b] ? p->C_row[a] < p->C_row[b] : p->C_col[a] < p->C_col[b];
    });
    std::vector<SymEntry> merged;
    for (int64_t t : co) {
      if (!merged.empty() && merged.back().row == p->C_row[t] && merged.back().col == p->C_col[t])
        merged.back().val += p->C_val[t];
      else
        merged.push_back({p->C_row[t], p->C_col[t], 0, p->C_val[t]});
    }
    for (const auto& e : merged) {
      if (e.val == 0.0) continue;
      cent.push_back(e);
      if (e.row != e.col) cent.push_back({e.col, e.row, 0, e.val});
    }
  }
  std::vector<int32_t> C_rp, C_col, C_dummy;
  std::vector<double> C_val;
  build_sym_csr(n, cent, C_rp, C_col, C_dummy, C_val);
  // norms of the data
  double cf = 0.0, cinf = 0.0, cone = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double rs = 0.0;
    for (int32_t q = C_rp[j]; q < C_rp[j + 1]; ++q) {
      cf += C_val[q] * C_val[q];
      rs += std::fabs(C_val[q]);
    }
    cinf = std::max(cinf, rs);
    cone += rs;
  }
  double binf = 0.0, bone = 0.0;
  for (double x : p->b) {
    binf = std::max(binf, std::fabs(x));
    bone += std::fabs(x);
  }
  p->C_fro = std::sqrt(cf);
  p->C_inf = cinf;
  p->b_inf = binf;
  p->c_one = cone;
  p->b_one = bone;
  // diagonal-separable constraints: U_0 rows can be scaled onto the constraints
  std::vector<double> row_norm(n, -1.0);
  bool dsep = true;
  for (int64_t i = 0; i < m && dsep; ++i) {
    const int32_t e = con_ptr[i];
    const double ratio = p->b[i] / con_a[e];
    if (multi || con_r[e] != con_c[e] || row_norm[con_r[e]] >= 0.0 || !(ratio > 0.0))
      dsep = false;
    else
      row_norm[con_r[e]] = std::sqrt(ratio);
  }
  p->diag_separable = dsep;
  // upload
  std::vector<float> A_valf(A_val.begin(), A_val.end()), C_valf(C_val.begin(), C_val.end());
  size_t bytes = Arena::need(nent, 4) * 2 + Arena::need(nent, 8) + Arena::need(m + 1, 4) * 2 +
                 Arena::need(nchunk + 1, 4) + Arena::need(m, 8) * 2 + Arena::need(n + 1, 4) * 2 +
                 Arena::need(A_col.size(), 4) * 2 + Arena::need(A_val.size(), 8) +
                 Arena::need(A_val.size(), 4) + Arena::need(C_col.size(), 4) +
                 Arena::need(C_val.size(), 8) + Arena::need(C_val.size(), 4) +
                 Arena::need(n, 8) + Arena::need(n, 4) * 2 + Arena::need(n, 8) + 4096;
  int st = p->prob_mem.reserve(bytes, al);
  if (st != LORADS_OK) return st;
  Arena& a = p->prob_mem;
  auto up = [](void* d, const void* h, size_t b) {
    return b ? cudaMemcpy(d, h, b, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  DevProblem dp{};
  dp.n = (int)n;
  dp.m = (int)m;
  int* d_con_ptr = a.take<int>(m + 1);
  int* d_con_r = a.take<int>(nent);
  int* d_con_c = a.take<int>(nent);
  double* d_con_a = a.take<double>(nent);
  int* d_chunk_ptr = a.take<int>(nchunk + 1);
  int* d_con_chunk = a.take<int>(m + 1);
  double* d_op_q = a.take<double>(m);
  double* d_b = a.take<double>(m);
  int* d_A_rp = a.take<int>(n + 1);
  int* d_A_col = a.take<int>(A_col.size());
  int* d_A_con = a.take<int>(A_con.size());
  double* d_A_val = a.take<double>(A_val.size());
  float* d_A_valf = a.take<float>(A_val.size());
  int* d_C_rp = a.take<int>(n + 1);
  int* d_C_col = a.take<int>(C_col.size());
  double* d_C_val = a.take<double>(C_val.size());
  float* d_C_valf = a.take<float>(C_val.size());
  double* d_row_norm = a.take<double>(n);
  CU(up(d_con_ptr, con_ptr.data(), (m + 1) * 4));
  CU(up(d_con_r, con_r.data(), nent * 4));
  CU(up(d_con_c, con_c.data(), nent * 4));
  CU(up(d_con_a, con_a.data(), nent * 8));
  CU(up(d_chunk_ptr, chunk_ptr.data(), (nchunk + 1) * 4));
  CU(up(d_con_chunk, con_chunk.data(), (m + 1) * 4));
  CU(up(d_b, p->b.data(), m * 8));
  CU(up(d_A_rp, A_rp.data(), (n + 1) * 4));
  CU(up(d_A_col, A_col.data(), A_col.size() * 4));
  CU(up(d_A_con, A_con.data(), A_con.size() * 4));
  CU(up(d_A_val, A_val.data(), A_val.size() * 8));
  CU(up(d_A_valf, A_valf.data(), A_valf.size() * 4));
  CU(up(d_C_rp, C_rp.data(), (n + 1) * 4));
  CU(up(d_C_col, C_col.data(), C_col.size() * 4));
  CU(up(d_C_val, C_val.data(), C_val.size() * 8));
  CU(up(d_C_valf, C_valf.data(), C_valf.size() * 4));
  CU(up(d_row_norm, row_norm.data(), n * 8));
  dp.con_ptr = d_con_ptr;
  dp.con_r = d_con_r;
  dp.con_c = d_con_c;
  dp.con_a = d_con_a;
  dp.a_multi = multi ? 1 : 0;
  dp.nchunk = (int)nchunk;
  dp.chunk_ptr = d_chunk_ptr;
  dp.con_chunk = d_con_chunk;
  dp.op_q = d_op_q;
  dp.b = d_b;
  dp.A_rp = d_A_rp;
  dp.A_col = d_A_col;
  dp.A_con = d_A_con;
  dp.A_val = d_A_val;
  dp.A_valf = d_A_valf;
  dp.C_rp = d_C_rp;
  dp.C_col = d_C_col;
  dp.C_val = d_C_val;
  dp.C_valf = d_C_valf;
  dp.row_norm = dsep ? d_row_norm : nullptr;
  dp.b_inf = binf;
  dp.C_fro = p->C_fro;
  dp.C_inf = cinf;
  dp.b_one = bone;
  dp.c_one = cone;
  // row-local form: every constraint one diagonal entry, at most one constraint per row
  bool diag_only = !multi;
  for (int64_t i = 0; i < m && diag_only; ++i) diag_only = con_r[i] == con_c[i];
  std::vector<int32_t> row_con(n, -1);
  std::vector<double> row_a(n, 0.0);
  for (int64_t i = 0; i < m && diag_only; ++i) {
    if (row_con[con_r[i]] >= 0) diag_only = false;
    row_con[con_r[i]] = (int32_t)i;
    row_a[con_r[i]] = con_a[i];
  }
  dp.a_diag_only = diag_only ? 1 : 0;
  dp.polish_ok = (diag_only && dsep && n == m) ? 1 : 0;
  if (diag_only) {
    std::vector<float> row_af(row_a.begin(), row_a.end());
    int* d_row_con = a.take<int>(n);
    double* d_row_a = a.take<double>(n);
    float* d_row_af = a.take<float>(n);
    CU(up(d_row_con, row_con.data(), n * 4));
    CU(up(d_row_a, row_a.data(), n * 8));
    CU(up(d_row_af, row_af.data(), n * 4));
    dp.row_con = d_row_con;
    dp.row_a = d_row_a;
    dp.row_af = d_row_af;
  }
  p->dp = dp;
  p->assembled = true;
  p->assemble_status = LORADS_OK;
  static_path_setup(p->device);
  return LORADS_OK;
}

static int resolve_rank_cap(const lorads_problem* p, const lorads_params* prm) {
  if (prm->rank_max > 0) return (int)std::min<int64_t>(prm->rank_max, p->n);
  int64_t c = (int64_t)std::floor(std::sqrt(2.0 * (double)p->m));
  c = std::min<int64_t>(std::min<int64_t>(c, p->n), 256);
  return (int)std::max<int64_t>(c, 1);
}

static int resolve_r0(const lorads_problem* p, const lorads_params* prm, int cap) {
  int64_t r = prm->r0 > 0 ? prm->r0
                          : (int64_t)std::ceil(std::log2((double)std::max<int64_t>(p->m, 2)));
  r = std::min<int64_t>(std::min<int64_t>(r, p->n), cap);
  return (int)std::max<int64_t>(r, 1);
}

// resolves the caller's parameters for problem p (auto values, gamma, ranks, limits)
static int fill_params(const lorads_problem* p, const lorads_params* prm, DevParams& dv) {
  dv = DevParams{};
  const int cap = resolve_rank_cap(p, prm);
  dv.rank_cap = cap;
  dv.r0 = resolve_r0(p, prm, cap);
  dv.rank_factor = prm->rank_factor;
  dv.tol = prm->tol;
  dv.switch_tol = prm->switch_tol >= 0 ? prm->switch_tol : (p->diag_separable ? 1e-2 : 1e-3);
  dv.h = prm->h >= 0 ? prm->h : (p->diag_separable ? 10.0 : 1.0);
  dv.rho_max = prm->rho_max;
  dv.rho_growth = prm->rho_growth;
  dv.rho_every = std::max(1, prm->rho_every);
  const double gscale = prm->gamma_scale >= 0 ? prm->gamma_scale : (p->diag_separable ? 1.0 : 2.0);
  dv.gamma = prm->gamma_fixed > 0 ? prm->gamma_fixed : gscale * (p->C_inf > 0 ? p->C_inf : 1.0);
  dv.max_admm_iter = prm->max_admm_iter;
  dv.cg_max_iter = prm->cg_max_iter;
  dv.cg_rel_tol = prm->cg_rel_tol;
  dv.cg_abs_floor = prm->cg_abs_floor;
  dv.lbfgs_mem = std::min(std::max(prm->lbfgs_mem, 1), MAXMEM);
  dv.inner_max_iter = prm->inner_max_iter;
  dv.inner_tol_factor = prm->inner_tol_factor;
  dv.inner_tol_max = prm->inner_tol_max;
  dv.max_outer = prm->max_outer;
  dv.sigma_factor = prm->sigma_factor;
  dv.sigma_decrease = prm->sigma_decrease;
  dv.sigma_max = prm->sigma_max;
  if (prm->lanczos_store_mb < 0) return LORADS_ERR_ARG;
  if (prm->iter_log_cap < 0 || (prm->iter_log_cap > 0 && prm->iter_log == nullptr))
    return LORADS_ERR_ARG;
  dv.iter_log = prm->iter_log_cap > 0 ? prm->iter_log : nullptr;
  dv.iter_log_cap = prm->iter_log_cap;
  dv.new_col_std = prm->new_col_std;
  dv.seed = prm->seed;
  dv.phase1 = prm->phase1 ? 1 : 0;
  dv.r_start = p->start_r;
  dv.nz0 = p->start_nz;
  dv.rho0 = p->start_rho > 0 ? p->start_rho : 100.0;
  dv.prev_dinf0 = std::numeric_limits<double>::quiet_NaN();
  if (!dv.phase1 && p->has_start && p->start_resume) {
    // continuation of a checkpointed Phase II: its gamma, counters and final-test schedule
    const lorads_state& q = p->start_state;
    dv.resume = 1;
    dv.gamma = q.gamma;
    dv.k0 = q.admm_iters;
    dv.next_test0 = q.next_dual_test;
    dv.cg0 = q.cg_iters;
    dv.hess0 = q.hessian_applies;
    dv.outer0 = q.alm_outer;
    dv.lbfgs0 = q.lbfgs_iters;
    dv.growths0 = q.rank_growths;
    dv.prev_dinf0 = q.prev_d_infeas;
    dv.sigma0 = q.sigma;
  }
  dv.time_limit_ns = (long long)(prm->time_limit_s * 1e9);
  dv.team_mult = prm->team_mult > 0 ? prm->team_mult : 1;
  if (dv.team_mult != 1 && dv.team_mult != 2 && dv.team_mult != 4 && dv.team_mult != 8)
    return LORADS_ERR_ARG;
  dv.kkt_dinf = prm->kkt_dinf ? 1 : 0;
  dv.lanczos_steps = prm->lanczos_steps;
  dv.dinf_every = std::max(1, prm->dinf_every);
  dv.escape_scale = prm->escape_scale;
  if (!(prm->escape_scale >= 0.0)) return LORADS_ERR_ARG;
  dv.subsolver = prm->subsolver;
  if (prm->polish != 0 && prm->polish != 1) return LORADS_ERR_ARG;
  if (prm->newton_max < 0 || prm->newton_cg_max < 1) return LORADS_ERR_ARG;
  dv.polish = prm->polish;
  dv.newton_max = prm->newton_max;
  dv.newton_cg_max = prm->newton_cg_max;
  if (prm->subsolver != 0 && prm->subsolver != 1) return LORADS_ERR_ARG;
  if (prm->subsolver == 1 && !p->dp.a_diag_only) return LORADS_ERR_UNSUPPORTED;
  if (prm->lanczos_steps < 0 || prm->lanczos_steps > LANCZOS_MAX) return LORADS_ERR_ARG;
  if (dv.kkt_dinf && prm->lanczos_steps == 0) return LORADS_ERR_ARG;
  if (!dv.phase1) {
    if (!p->has_start) return LORADS_ERR_STATE;
    if (p->start_r > 256) return LORADS_ERR_ARG;
  }
  return LORADS_OK;
}

// uploads the Phase II start in the solver's layout (n x round4(r) row-major, zero padding):
// U, V for a resume (else the kernel sets V = U), lambda (zero when not given)
static int upload_start(const lorads_problem* p, double* dU, double* dV, double* dlam,
                        cudaStream_t s) {
  const int64_t n = p->n, m = p->m;
  const int r = p->start_r, ld = round4(r);
  CU(cudaMemsetAsync(dU, 0, (size_t)n * ld * 8, s));
  CU(cudaMemcpy2DAsync(dU, (size_t)ld * 8, p->start_U.data(), (size_t)r * 8, (size_t)r * 8,
                       (size_t)n, cudaMemcpyHostToDevice, s));
  if (p->start_resume) {
    CU(cudaMemsetAsync(dV, 0, (size_t)n * ld * 8, s));
    CU(cudaMemcpy2DAsync(dV, (size_t)ld * 8, p->start_V.data(), (size_t)r * 8, (size_t)r * 8,
                         (size_t)n, cudaMemcpyHostToDevice, s));
  }
  if (!p->start_lam.empty())
    CU(cudaMemcpyAsync(dlam, p->start_lam.data(), m * 8, cudaMemcpyHostToDevice, s));
  else
    CU(cudaMemsetAsync(dlam, 0, m * 8, s));
  return LORADS_OK;
}

// allocates (or reuses) p's state arena, lays out the solver arrays, uploads the Phase II
// start if any and the argument block, and clears what must start at zero
template <typename T>
static int prepare_state(lorads_problem* p, const DevParams& dv, cudaStream_t s,
                         const DevAlloc& al, SolverArgs<T>& h, SolverArgs<T>** dargs_out,
                         size_t store_cap_bytes = 0) {
  const int64_t n = p->n, m = p->m;
  const int rmax = std::max(dv.rank_cap, dv.phase1 ? 0 : p->start_r);
  const long long ld_cap = round4(rmax);
  const size_t NS = (size_t)n * ld_cap;
  const int ring = dv.lbfgs_mem + 1;
  const bool mixed = sizeof(T) == 4;
  int dev_sms = 0;
  CU(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, p->device));
  size_t bytes = Arena::need(NS, 8) * 8 + Arena::need(NS, sizeof(T)) * (mixed ? 7 : 5) +
                 Arena::need(m, 8) * 2 + Arena::need(3 * (size_t)p->dp.nchunk + m, 8) +
                 Arena::need(NS * ring, 8) * 2 +
                 Arena::need(1, sizeof(SolverArgs<T>)) + Arena::need(1, sizeof(SolveOut)) +
                 Arena::need(1, sizeof(GridCtl)) +
                 Arena::need((size_t)dev_sms * 8 * MAXRED * 3, 8) + Arena::need(4, 4) + 4096;
  // the Lanczos vectors of a dual test: slots 0..Kmax of n x 4 doubles, when they fit the cap
  const int kmax = std::min(std::min(dv.lanczos_steps, LANCZOS_MAX), (int)std::min<int64_t>(n, INT32_MAX));
  const size_t store_count = dv.kkt_dinf && kmax > 0 ? (size_t)(kmax + 1) * (size_t)n * 4 : 0;
  const bool store = store_count > 0 && store_count * 8 <= store_cap_bytes;
  if (store) bytes += Arena::need(store_count, 8);
  int st = p->state_mem.reserve(bytes, al);
  if (st != LORADS_OK) return st;
  Arena& a = p->state_mem;
  h = SolverArgs<T>{};
  h.P = p->dp;
  h.prm = dv;
  h.U = a.take<double>(NS);
  h.V = a.take<double>(NS);
  if (mixed) {
    h.Ut = a.take<T>(NS);
    h.Vt = a.take<T>(NS);
  } else {
    h.Ut = reinterpret_cast<T*>(h.U);
    h.Vt = reinterpret_cast<T*>(h.V);
  }
  h.Dl = a.take<T>(NS);
  h.R = a.take<T>(NS);
  h.Pd = a.take<T>(NS);
  h.HP = a.take<T>(NS);
  h.Sv = a.take<T>(NS);
  h.lam = a.take<double>(m);
  h.e = a.take<double>(m);
  h.cq = a.take<double>(3 * (size_t)p->dp.nchunk + m);
  h.grad = a.take<double>(NS);
  h.grad_old = a.take<double>(NS);
  h.dir = a.take<double>(NS);
  h.tmp = a.take<double>(NS);
  h.CWn = a.take<double>(NS);
  h.S = a.take<double>(NS * ring);
  h.Y = a.take<double>(NS * ring);
  h.lz_store = store ? a.take<double>(store_count) : nullptr;
  h.ld_cap = ld_cap;
  SolverArgs<T>* dargs = a.take<SolverArgs<T>>(1);
  p->dout = a.take<SolveOut>(1);
  h.out = p->dout;
  p->dctl = a.take<GridCtl>(1);
  p->dpartials = a.take<double>((size_t)dev_sms * 8 * MAXRED * 3);
  p->dqueue = a.take<int>(4);
  p->dU = h.U;
  p->dV = h.V;
  p->dUh = h.tmp;
  p->dlam = h.lam;
  p->has_solution = false;
  // Phase II start supplied by the caller
  if (!dv.phase1) {
    st = upload_start(p, h.U, h.V, h.lam, s);
    if (st != LORADS_OK) return st;
  }
  CU(cudaMemcpyAsync(dargs, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  // the report starts as a device error: a solve that never runs (a launch that failed, a
  // batch group that stopped at a failed barrier) cannot read as a success
  SolveOut unreached{};
  unreached.status = ST_DEVICE;
  CU(cudaMemcpyAsync(p->dout, &unreached, sizeof(SolveOut), cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(p->dctl, 0, sizeof(GridCtl), s));
  CU(cudaMemsetAsync(p->dpartials, 0xFF, sizeof(double) * (size_t)dev_sms * 8 * MAXRED * 3, s));
  CU(cudaMemsetAsync(p->dqueue, 0, 16, s));
  *dargs_out = dargs;
  return LORADS_OK;
}

static void to_result(const SolveOut& out, lorads_result& r) {
  r = lorads_result{};
  r.status = out.status;
  r.rank = out.rank;
  r.objective = out.objective;
  r.dual_objective = out.dual_objective;
  r.r_P = out.r_P;
  r.r_P_split = out.r_P_split;
  r.r_stop = out.r_stop;
  r.r_D = out.r_D;
  r.gap = out.gap;
  r.rho = out.rho;
  r.gamma = out.gamma;
  r.sigma = out.sigma;
  r.admm_iters = out.admm_iters;
  r.cg_iters = out.cg_iters;
  r.hessian_applies = out.hess_applies;
  r.alm_outer = out.alm_outer;
  r.lbfgs_iters = out.lbfgs_iters;
  r.rank_growths = out.growths;
  r.time_phase1_s = out.t_phase1_ns * 1e-9;
  r.time_phase2_s = out.t_phase2_ns * 1e-9;
  r.p_infeas = out.p_infeas;
  r.d_infeas = out.d_infeas;
  r.lambda_min = out.lambda_min;
  r.dual_psd = out.dual_psd;
  r.time_phase3_s = out.t_phase3_ns * 1e-9;
  r.polished = out.polished;
  r.newton_steps = out.newton_steps;
  r.newton_cg_iters = out.newton_cg;
  r.refine_outer = out.refine_outer;
  r.refine_lbfgs_iters = out.refine_lbfgs;
  r.lanczos_steps = out.lanczos_steps;
  r.time_lanczos_s = out.t_lanczos_ns * 1e-9;
}

static void record_solution(lorads_problem* p, const SolveOut& out, const lorads_result& r) {
  p->last = r;
  p->last_out = out;
  p->sol_r = out.rank;
  p->sol_ld = out.ld;
  p->has_solution = out.ld > 0;
}

// Launch geometry of a single-problem solve: one CTA for small problems (n < 512), the whole
// GPU from a few hundred rows up.  One-CTA solves take prm->threads (default SOLVER_THREADS);
// whole-GPU solves take prm->threads or, by default, enough teams for one row each at the
// initial rank, within [128, 320] threads, and at most as many CTAs as are co-resident.
// lorads_solve and lorads_solve_static both launch with it, so that the same parameters
// give the same reduction order and iterates on either path.
template <typename T>
static int solve_geometry(const lorads_problem* p, const lorads_params* prm,
                          const DevParams& dv, int dev_sms, bool* whole_gpu, int* grid_out,
                          int* threads_out) {
  int grid = prm->grid;
  if (grid <= 0) grid = (p->n < 512) ? 1 : dev_sms;
  *whole_gpu = grid != 1;
  if (grid == 1) {
    const int threads = prm->threads > 0 ? prm->threads : SOLVER_THREADS;
    if (threads % 32 != 0 || threads < SOLVER_THREADS_MIN || threads > BLOCK_THREADS_MAX)
      return LORADS_ERR_ARG;
    *grid_out = 1;
    *threads_out = threads;
    return LORADS_OK;
  }
  int gthreads = prm->threads > 0 ? prm->threads : 0;
  if (gthreads == 0) {
    const int G = team_size_for(round4(dv.phase1 ? dv.r0 : p->start_r)) * dv.team_mult;
    const long long lanes = (long long)p->n * std::min(G, 32);
    const int per = (int)((lanes + grid - 1) / grid);
    gthreads = std::min(GRID_THREADS_MAX, std::max(128, ((per + 31) / 32) * 32));
  }
  if (gthreads % 32 != 0 || gthreads < SOLVER_THREADS_MIN || gthreads > GRID_THREADS_MAX)
    return LORADS_ERR_ARG;
  int per_sm = 0;
  CU(Launch<T>::grid_capacity(dv.subsolver, gthreads, &per_sm));
  const int maxg = std::max(1, per_sm) * dev_sms;
  *grid_out = std::min(std::min(grid, maxg), dev_sms * 8);
  *threads_out = gthreads;
  return LORADS_OK;
}

template <typename T>
static int run_solve(lorads_problem* p, const lorads_params* prm, cudaStream_t s,
                     lorads_result* res) {
  DevParams dv;
  int st = fill_params(p, prm, dv);
  if (st != LORADS_OK) return st;
  int dev_sms = 0;
  CU(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, p->device));
  bool whole = false;
  int grid = 1, threads = SOLVER_THREADS;
  st = solve_geometry<T>(p, prm, dv, dev_sms, &whole, &grid, &threads);
  if (st != LORADS_OK) return st;
  SolverArgs<T> h;
  SolverArgs<T>* dargs = nullptr;
  st = prepare_state<T>(p, dv, s, DevAlloc::from(prm, s), h, &dargs,
                        (size_t)prm->lanczos_store_mb << 20);
  if (st != LORADS_OK) return st;
  cudaError_t le;
  if (!whole) {
    le = Launch<T>::solve_block(dv.subsolver, dargs, 1, p->dqueue, 1, threads, s);
  } else {
    le = Launch<T>::solve_grid(dv.subsolver, dargs, p->dctl, p->dpartials, barrier_polls(prm),
                               grid, threads, s);
  }
  CU(le);
  SolveOut out{};
  CU(cudaMemcpyAsync(&out, p->dout, sizeof(out), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  lorads_result r;
  to_result(out, r);
  record_solution(p, out, r);
  if (res) *res = r;
  return r.status;
}

// ---------------------------------------------------------------------------------------
// batches: one CTA per problem, CTAs take problems from a device queue, largest first
// ---------------------------------------------------------------------------------------
template <typename T>
static int run_batch_once(lorads_problem* const* ps, int count, const lorads_params* prm,
                          cudaStream_t s, int threads, int team_mult, int group,
                          lorads_result* res, double* seconds) {
  const int device = ps[0]->device;
  std::vector<SolverArgs<T>> hs(count);
  std::vector<std::pair<double, int>> order(count);
  lorads_params q = *prm;
  q.team_mult = team_mult;
  q.iter_log = nullptr;      // problems of a batch would share one log
  q.iter_log_cap = 0;
  const int sub = prm->subsolver;
  const DevAlloc al = DevAlloc::from(prm, s);
  for (int i = 0; i < count; ++i) {
    lorads_problem* p = ps[i];
    if (p->device != device) return LORADS_ERR_ARG;
    int st = assemble(p, al);
    if (st != LORADS_OK) return st;
    DevParams dv;
    st = fill_params(p, &q, dv);
    if (st != LORADS_OK) return st;
    SolverArgs<T>* unused = nullptr;
    st = prepare_state<T>(p, dv, s, al, hs[i], &unused);
    if (st != LORADS_OK) return st;
    // work estimate: rows times (A + C entries per row), for largest-first scheduling
    order[i] = {-(double)p->n * (double)(p->C_row.size() + p->A_con.size() + p->n) / p->n, i};
  }
  std::stable_sort(order.begin(), order.end());
  std::vector<SolverArgs<T>> sorted(count);
  for (int k = 0; k < count; ++k) sorted[k] = hs[order[k].second];
  int dev_sms = 0, per_sm = 0;
  CU(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, device));
  if (group > 1) CU(Launch<T>::group_capacity(sub, threads, &per_sm));
  else CU(Launch<T>::block_capacity(sub, threads, &per_sm));
  // one CTA per problem, or groups of `group` CTAs per problem (never more than resident)
  int grid = std::max(1, std::min(count, std::max(1, per_sm) * dev_sms));
  int groups = 0;
  if (group > 1) {
    groups = std::min(count, std::max(1, per_sm) * dev_sms / group);
    if (groups < 1) return LORADS_ERR_ARG;
    grid = groups * group;
  }
  // argument block, queue, and for groups their barriers, problem slots and partial sums
  const size_t a_bytes = (sizeof(SolverArgs<T>) * count + 255) / 256 * 256;
  const size_t c_bytes = (sizeof(GridCtl) * groups + 255) / 256 * 256;
  const size_t s_bytes = (sizeof(int) * groups + 255) / 256 * 256;
  const size_t p_bytes = sizeof(double) * (size_t)grid * MAXRED * (group > 1 ? 2 : 0);
  const size_t base_bytes = a_bytes + 256 + c_bytes + s_bytes + p_bytes;
  char* base = static_cast<char*>(al.get(base_bytes));
  if (!base) return LORADS_ERR_NOMEM;
  SolverArgs<T>* dargs = reinterpret_cast<SolverArgs<T>*>(base);
  int* dqueue = reinterpret_cast<int*>(base + a_bytes);
  GridCtl* dctls = reinterpret_cast<GridCtl*>(base + a_bytes + 256);
  int* dslots = reinterpret_cast<int*>(base + a_bytes + 256 + c_bytes);
  double* dparts = reinterpret_cast<double*>(base + a_bytes + 256 + c_bytes + s_bytes);
  int st = LORADS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  do {
    if ((st = check_cuda(cudaMemcpyAsync(dargs, sorted.data(), sizeof(SolverArgs<T>) * count,
                                         cudaMemcpyHostToDevice, s))) != LORADS_OK) break;
    // the device work (queue and barrier resets + the persistent kernel) as one CUDA graph:
    // captured on a private stream (the legacy default stream cannot be captured), launched
    // on the caller's
    if ((st = check_cuda(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) != LORADS_OK)
      break;
    if ((st = check_cuda(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) !=
        LORADS_OK) break;
    cudaError_t c1 = cudaMemsetAsync(dqueue, 0, 16, cap);
    if (c1 == cudaSuccess && group > 1) c1 = cudaMemsetAsync(dctls, 0, c_bytes, cap);
    const cudaError_t c2 =
        group > 1 ? Launch<T>::solve_group(sub, dargs, count, dqueue, dctls, dparts, dslots, group,
                                           barrier_polls(prm), grid, threads, cap)
                  : Launch<T>::solve_block(sub, dargs, count, dqueue, grid, threads, cap);
    const cudaError_t c3 = cudaStreamEndCapture(cap, &graph);
    if ((st = check_cuda(c1 != cudaSuccess ? c1 : (c2 != cudaSuccess ? c2 : c3))) != LORADS_OK)
      break;
    if ((st = check_cuda(cudaGraphInstantiate(&gexec, graph, 0))) != LORADS_OK) break;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    if ((st = check_cuda(cudaGraphLaunch(gexec, s))) != LORADS_OK) break;
    cudaEventRecord(e1, s);
    if ((st = check_cuda(cudaStreamSynchronize(s))) != LORADS_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (seconds) *seconds = ms * 1e-3;
    for (int i = 0; i < count; ++i) {
      SolveOut out{};
      if ((st = check_cuda(cudaMemcpy(&out, ps[i]->dout, sizeof(out), cudaMemcpyDeviceToHost))) !=
          LORADS_OK) break;
      lorads_result r;
      to_result(out, r);
      record_solution(ps[i], out, r);
      if (res) res[i] = r;
    }
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  // every use of base has finished (the stream was synchronized, or nothing ran)
  cudaStreamSynchronize(s);
  al.put(base, base_bytes);
  return st;
}

// Autotuner: times a sample of the batch (every k-th problem, largest included) under each
// (CTA size, lanes-per-row multiplier) candidate and returns the fastest.
template <typename T>
static int autotune_batch(lorads_problem* const* ps, int count, const lorads_params* prm,
                          cudaStream_t s, int group, int* threads_out, int* mult_out) {
  const int cand_threads[] = {128, 256, 384};
  const int cand_mult[] = {1, 2, 4};
  std::vector<lorads_problem*> sample;
  const int want = std::min(count, 24);
  for (int k = 0; k < want; ++k) sample.push_back(ps[(int64_t)k * count / want]);
  lorads_params q = *prm;
  q.max_admm_iter = std::min(prm->max_admm_iter, 200);
  q.iter_log = nullptr;
  q.iter_log_cap = 0;
  double best = 1e300;
  *threads_out = SOLVER_THREADS;
  *mult_out = 1;
  for (int th : cand_threads)
    for (int mu : cand_mult) {
      double sec = 0.0;
      int st = run_batch_once<T>(sample.data(), (int)sample.size(), &q, s, th, mu, group,
                                 nullptr, &sec);
      if (st != LORADS_OK) return st;
      if (sec < best) {
        best = sec;
        *threads_out = th;
        *mult_out = mu;
      }
    }
  return LORADS_OK;
}

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
extern "C" {

int lorads_create(int64_t n, int64_t m, lorads_problem** out) {
  if (!out) return LORADS_ERR_ARG;
  *out = nullptr;
  if (n <= 0 || m <= 0 || n > INT32_MAX / 2 || m > INT32_MAX / 2) return LORADS_ERR_ARG;
  lorads_problem* p = new (std::nothrow) lorads_problem();
  if (!p) return LORADS_ERR_NOMEM;
  p->n = n;
  p->m = m;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return LORADS_ERR_CUDA;
  }
  *out = p;
  return LORADS_OK;
}

int lorads_set_C(lorads_problem* p, int64_t nnz, const int32_t* row, const int32_t* col,
                 const double* val) {
  if (!p || nnz < 0 || (nnz > 0 && (!row || !col || !val))) return LORADS_ERR_ARG;
  for (int64_t t = 0; t < nnz; ++t)
    if (row[t] < 0 || col[t] < row[t] || col[t] >= p->n || !is_finite_value(val[t])) return LORADS_ERR_ARG;
  p->C_row.assign(row, row + nnz);
  p->C_col.assign(col, col + nnz);
  p->C_val.assign(val, val + nnz);
  invalidate(p);
  return LORADS_OK;
}

int lorads_add_A_sparse(lorads_problem* p, int64_t nnz, const int32_t* con, const int32_t* row,
                        const int32_t* col, const double* val) {
  if (!p || nnz < 0 || (nnz > 0 && (!con || !row || !col || !val))) return LORADS_ERR_ARG;
  for (int64_t t = 0; t < nnz; ++t)
    if (con[t] < 0 || con[t] >= p->m || row[t] < 0 || col[t] < row[t] || col[t] >= p->n ||
        !is_finite_value(val[t]))
      return LORADS_ERR_ARG;
  p->A_con.insert(p->A_con.end(), con, con + nnz);
  p->A_row.insert(p->A_row.end(), row, row + nnz);
  p->A_col.insert(p->A_col.end(), col, col + nnz);
  p->A_val.insert(p->A_val.end(), val, val + nnz);
  invalidate(p);
  return LORADS_OK;
}

int lorads_add_A_rank1(lorads_problem* p, int32_t con, int64_t nnz, const int32_t* idx,
                       const double* a, double scale) {
  if (!p || con < 0 || con >= p->m || nnz <= 0 || !idx || !a || !is_finite_value(scale))
    return LORADS_ERR_ARG;
  for (int64_t t = 0; t < nnz; ++t)
    if (idx[t] < 0 || idx[t] >= p->n || !is_finite_value(a[t])) return LORADS_ERR_ARG;
  p->rank1.push_back({con, std::vector<int32_t>(idx, idx + nnz), std::vector<double>(a, a + nnz),
                      scale});
  invalidate(p);
  return LORADS_OK;
}

int lorads_set_b(lorads_problem* p, const double* b) {
  if (!p || !b) return LORADS_ERR_ARG;
  for (int64_t i = 0; i < p->m; ++i)
    if (!is_finite_value(b[i])) return LORADS_ERR_ARG;
  p->b.assign(b, b + p->m);
  p->has_b = true;
  invalidate(p);
  return LORADS_OK;
}

void lorads_default_params(lorads_params* prm) {
  if (!prm) return;
  std::memset(prm, 0, sizeof(*prm));
  prm->r0 = 0;
  prm->rank_max = 0;
  prm->rank_factor = 1.5;
  prm->tol = 1e-6;
  prm->switch_tol = -1.0;
  prm->h = -1.0;
  prm->rho_max = 5000.0;
  prm->rho_growth = 1.2;
  prm->rho_every = 5;
  prm->gamma_scale = -1.0;
  prm->gamma_fixed = 0.0;
  prm->max_admm_iter = 5000;
  prm->cg_max_iter = 1000;
  prm->cg_rel_tol = 1e-3;
  prm->cg_abs_floor = 1e-13;
  prm->lbfgs_mem = 4;
  prm->inner_max_iter = 300;
  prm->inner_tol_factor = 10.0;
  prm->inner_tol_max = 0.1;
  prm->max_outer = 500;
  prm->sigma_factor = 2.0;
  prm->sigma_decrease = 0.25;
  prm->sigma_max = 1e4;
  prm->new_col_std = 1e-2;
  prm->seed = 1;
  prm->precision = LORADS_PREC_FP64;
  prm->phase1 = 1;
  prm->time_limit_s = 60.0;
  prm->threads = 0;
  prm->grid = 0;
  prm->team_mult = 0;
  prm->kkt_dinf = 1;
  prm->lanczos_steps = 2048;
  prm->lanczos_store_mb = 2048;
  prm->dinf_every = 10;
  prm->escape_scale = 0.3;
  prm->group = 0;
  prm->polish = 1;
  prm->newton_max = 200;
  prm->newton_cg_max = 1000;
}

int lorads_set_start(lorads_problem* p, int32_t r, const double* U0, const double* lambda0,
                     double rho0) {
  if (!p || r <= 0 || r > p->n || !U0) return LORADS_ERR_ARG;
  for (int64_t t = 0; t < p->n * r; ++t)
    if (!is_finite_value(U0[t])) return LORADS_ERR_ARG;
  p->start_r = r;
  p->start_nz = trailing_zero_from(U0, nullptr, p->n, r);
  p->start_U.assign(U0, U0 + p->n * r);
  if (lambda0)
    p->start_lam.assign(lambda0, lambda0 + p->m);
  else
    p->start_lam.clear();
  p->start_rho = rho0;
  p->start_V.clear();
  p->start_resume = false;
  p->has_start = true;
  return LORADS_OK;
}

static int solve_impl(lorads_problem* p, const lorads_params* prm, void* stream,
                      lorads_result* res) {
  if (!p) return LORADS_ERR_ARG;
  lorads_params defaults;
  if (!prm) {
    lorads_default_params(&defaults);
    prm = &defaults;
  }
  if (prm->precision != LORADS_PREC_FP64 && prm->precision != LORADS_PREC_MIXED)
    return LORADS_ERR_ARG;
  if (!(prm->tol > 0) || prm->max_admm_iter < 1 || prm->cg_max_iter < 1) return LORADS_ERR_ARG;
  const DevAlloc al = DevAlloc::from(prm, stream);
  if (!al.valid()) return LORADS_ERR_ARG;
  int st = assemble(p, al);
  if (st != LORADS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (prm->precision == LORADS_PREC_MIXED) return run_solve<float>(p, prm, s, res);
  return run_solve<double>(p, prm, s, res);
}

int lorads_solve(lorads_problem* p, const lorads_params* prm, void* stream, lorads_result* res) {
  if (res) std::memset(res, 0, sizeof(*res));
  const int st = solve_impl(p, prm, stream, res);
  if (res) res->status = st;
  return st;
}

int lorads_solve_batch(lorads_problem* const* ps, int32_t count, const lorads_params* prm,
                       void* stream, lorads_result* res, int32_t* tuned_threads,
                       int32_t* tuned_team_mult) {
  if (!ps || count <= 0) return LORADS_ERR_ARG;
  for (int32_t i = 0; i < count; ++i)
    if (!ps[i]) return LORADS_ERR_ARG;
  lorads_params defaults;
  if (!prm) {
    lorads_default_params(&defaults);
    prm = &defaults;
  }
  if (prm->precision != LORADS_PREC_FP64 && prm->precision != LORADS_PREC_MIXED)
    return LORADS_ERR_ARG;
  if (!(prm->tol > 0) || prm->max_admm_iter < 1 || prm->cg_max_iter < 1) return LORADS_ERR_ARG;
  if (!DevAlloc::from(prm, stream).valid()) return LORADS_ERR_ARG;
  if (res) std::memset(res, 0, sizeof(lorads_result) * count);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool mixed = prm->precision == LORADS_PREC_MIXED;
  int threads = prm->threads, mult = prm->team_mult;
  int st = LORADS_OK;
  // CTAs per problem: automatic = 2 when the largest problem has n >= 1024 (one CTA then
  // carries a long solve alone and sets the batch's makespan), else 1
  int64_t n_max = 0;
  for (int i = 0; i < count; ++i) n_max = std::max(n_max, ps[i]->n);
  const int group = prm->group > 0 ? prm->group : (n_max >= 1024 ? 2 : 1);
  if (group != 1 && group != 2 && group != 4) return LORADS_ERR_ARG;
  if (threads <= 0 || mult <= 0) {
    int th = SOLVER_THREADS, mu = 1;
    st = mixed ? autotune_batch<float>(ps, count, prm, s, group, &th, &mu)
               : autotune_batch<double>(ps, count, prm, s, group, &th, &mu);
    if (st != LORADS_OK) return st;
    if (threads <= 0) threads = th;
    if (mult <= 0) mult = mu;
  }
  if (threads % 32 != 0 || threads < SOLVER_THREADS_MIN || threads > BLOCK_THREADS_MAX)
    return LORADS_ERR_ARG;
  if (tuned_threads) *tuned_threads = threads;
  if (tuned_team_mult) *tuned_team_mult = mult;
  st = mixed ? run_batch_once<float>(ps, count, prm, s, threads, mult, group, res, nullptr)
             : run_batch_once<double>(ps, count, prm, s, threads, mult, group, res, nullptr);
  return st;
}

int lorads_get_solution(const lorads_problem* p, double* U, double* V, double* U_hat, double* y,
                        int32_t* r) {
  if (!p) return LORADS_ERR_ARG;
  if (!p->has_solution) return LORADS_ERR_STATE;
  if (r) *r = p->sol_r;
  const int rr = p->sol_r, ld = p->sol_ld;
  const int64_t n = p->n;
  std::vector<double> buf((size_t)n * ld);
  auto fetch = [&](const double* d, double* h) -> int {
    if (!h) return LORADS_OK;
    if (cudaMemcpy(buf.data(), d, buf.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return check_cuda(cudaGetLastError());
    for (int64_t j = 0; j < n; ++j)
      std::memcpy(h + (size_t)j * rr, buf.data() + (size_t)j * ld, rr * 8);
    return LORADS_OK;
  };
  int st;
  if ((st = fetch(p->dU, U)) != LORADS_OK) return st;
  if ((st = fetch(p->dV, V)) != LORADS_OK) return st;
  if ((st = fetch(p->dUh, U_hat)) != LORADS_OK) return st;
  if (y) {
    if (cudaMemcpy(y, p->dlam, p->m * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return check_cuda(cudaGetLastError());
    for (int64_t i = 0; i < p->m; ++i) y[i] = -y[i];
  }
  return LORADS_OK;
}

int lorads_get_state(const lorads_problem* p, lorads_state* st, double* U, double* V,
                     double* lambda) {
  if (!p) return LORADS_ERR_ARG;
  const SolveOut& o = p->last_out;
  if (!p->has_solution || o.phase != 2 ||
      (o.status != ST_OK && o.status != ST_MAXITER && o.status != ST_TIMEOUT))
    return LORADS_ERR_STATE;
  if (st) {
    *st = lorads_state{};
    st->n = p->n;
    st->m = p->m;
    st->phase = 2;
    st->rank = o.rank;
    st->admm_iters = o.admm_iters;
    st->next_dual_test = o.next_dual_test;
    st->cg_iters = o.cg_iters;
    st->hessian_applies = o.hess_applies;
    st->alm_outer = o.alm_outer;
    st->lbfgs_iters = o.lbfgs_iters;
    st->rank_growths = o.growths;
    st->rho = o.rho;
    st->gamma = o.gamma;
    st->sigma = o.sigma;
    st->prev_d_infeas = o.prev_dinf;
  }
  const size_t r = (size_t)p->sol_r, ld = (size_t)p->sol_ld;
  if (U) CU(cudaMemcpy2D(U, r * 8, p->dU, ld * 8, r * 8, (size_t)p->n, cudaMemcpyDeviceToHost));
  if (V) CU(cudaMemcpy2D(V, r * 8, p->dV, ld * 8, r * 8, (size_t)p->n, cudaMemcpyDeviceToHost));
  if (lambda) CU(cudaMemcpy(lambda, p->dlam, (size_t)p->m * 8, cudaMemcpyDeviceToHost));
  return LORADS_OK;
}

int lorads_set_state(lorads_problem* p, const lorads_state* st, const double* U, const double* V,
                     const double* lambda) {
  if (!p || !st || !U || !V) return LORADS_ERR_ARG;
  if (st->n != p->n || st->m != p->m || st->phase != 2) return LORADS_ERR_ARG;
  if (st->rank < 1 || st->rank > std::min<int64_t>(p->n, 256)) return LORADS_ERR_ARG;
  if (!(st->rho > 0) || !std::isfinite(st->rho) || !(st->gamma > 0) || !std::isfinite(st->gamma))
    return LORADS_ERR_ARG;
  if (!std::isfinite(st->sigma) || (!std::isnan(st->prev_d_infeas) && !(st->prev_d_infeas >= 0)))
    return LORADS_ERR_ARG;
  if (std::isinf(st->prev_d_infeas)) return LORADS_ERR_ARG;
  if (st->admm_iters < 0 || st->next_dual_test < 0 || st->cg_iters < 0 ||
      st->hessian_applies < 0 || st->alm_outer < 0 || st->lbfgs_iters < 0 || st->rank_growths < 0)
    return LORADS_ERR_ARG;
  const size_t nr = (size_t)p->n * st->rank;
  for (size_t t = 0; t < nr; ++t)
    if (!is_finite_value(U[t]) || !is_finite_value(V[t])) return LORADS_ERR_ARG;
  if (lambda)
    for (int64_t i = 0; i < p->m; ++i)
      if (!is_finite_value(lambda[i])) return LORADS_ERR_ARG;
  p->start_r = st->rank;
  p->start_nz = trailing_zero_from(U, V, p->n, st->rank);
  p->start_U.assign(U, U + nr);
  p->start_V.assign(V, V + nr);
  if (lambda)
    p->start_lam.assign(lambda, lambda + p->m);
  else
    p->start_lam.clear();
  p->start_rho = st->rho;
  p->start_state = *st;
  p->start_resume = true;
  p->has_start = true;
  return LORADS_OK;
}

void lorads_destroy(lorads_problem* p) {
  if (!p) return;
  p->prob_mem.release();
  p->state_mem.release();
  delete p;
}

const char* lorads_status_string(int code) {
  switch (code) {
    case LORADS_OK: return "ok";
    case LORADS_ERR_ARG: return "bad argument";
    case LORADS_ERR_STATE: return "call out of order";
    case LORADS_ERR_CUDA: return "CUDA runtime error";
    case LORADS_ERR_NOMEM: return "out of memory";
    case LORADS_ERR_MAXITER: return "iteration cap reached";
    case LORADS_ERR_TIMEOUT: return "time limit reached";
    case LORADS_ERR_NAN: return "NaN or Inf in the iterates";
    case LORADS_ERR_UNSUPPORTED: return "constraint structure not supported by the device path";
    case LORADS_ERR_DEVICE: return "device-side wait gave up";
    case LORADS_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of lorads_solve_static";
    default: return "unknown status";
  }
}

void lorads_struct_sizes(int64_t* params_bytes, int64_t* result_bytes, int64_t* state_bytes) {
  if (params_bytes) *params_bytes = (int64_t)sizeof(lorads_params);
  if (result_bytes) *result_bytes = (int64_t)sizeof(lorads_result);
  if (state_bytes) *state_bytes = (int64_t)sizeof(lorads_state);
}

// ---- operators -----------------------------------------------------------------------
static int op_prepare(lorads_problem* p, int32_t prec, int32_t r, int32_t ld) {
  if (!p || (prec != LORADS_PREC_FP64 && prec != LORADS_PREC_MIXED)) return LORADS_ERR_ARG;
  if (r <= 0 || ld < r || (ld % 4) != 0 || team_size_for(ld) * KMAX * CHUNK < ld)
    return LORADS_ERR_ARG;
  return assemble(p, DevAlloc{});
}

static int op_grid(const lorads_problem* p) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    cudaGetLastError();
    sms = 1;
  }
  return sms * 8;
}

int lorads_op_sddmm(lorads_problem* p, int32_t prec, int32_t r, int32_t ld, const void* U,
                    const void* V, double* q, void* stream) {
  int st = op_prepare(p, prec, r, ld);
  if (st != LORADS_OK) return st;
  if (!U || !V || !q) return LORADS_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (prec == LORADS_PREC_MIXED)
    return check_cuda(Launch<float>::op_sddmm(p->dp, ld, (const float*)U, (const float*)V, q,
                                              op_grid(p), s));
  return check_cuda(Launch<double>::op_sddmm(p->dp, ld, (const double*)U, (const double*)V, q,
                                             op_grid(p), s));
}

int lorads_op_spmm(lorads_problem* p, int32_t prec, int32_t r, int32_t ld, const double* w,
                   double gamma, const void* V, void* out, void* stream) {
  int st = op_prepare(p, prec, r, ld);
  if (st != LORADS_OK) return st;
  if (!w || !V || !out) return LORADS_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (prec == LORADS_PREC_MIXED)
    return check_cuda(Launch<float>::op_spmm(p->dp, ld, w, gamma, (const float*)V, (float*)out,
                                             op_grid(p), s));
  return check_cuda(Launch<double>::op_spmm(p->dp, ld, w, gamma, (const double*)V, (double*)out,
                                            op_grid(p), s));
}

int lorads_op_hessian(lorads_problem* p, int32_t prec, int32_t r, int32_t ld, double rho,
                      double gamma, const void* V, const void* P, void* out, void* stream) {
  int st = op_prepare(p, prec, r, ld);
  if (st != LORADS_OK) return st;
  if (!V || !P || !out) return LORADS_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (prec == LORADS_PREC_MIXED)
    return check_cuda(Launch<float>::op_hessian(p->dp, ld, rho, gamma, (const float*)V,
                                                (const float*)P, (float*)out, op_grid(p), s));
  return check_cuda(Launch<double>::op_hessian(p->dp, ld, rho, gamma, (const double*)V,
                                               (const double*)P, (double*)out, op_grid(p), s));
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// lorads_solve_static: the solver's working memory in a fixed file-scope device array
// ---------------------------------------------------------------------------------------
// The array is the only memory the call touches besides the problem's assembled device
// form (built earlier) and the caller's output buffers.  Host code must not use the
// symbol's name as an address: it is a host-side stand-in.  The device address is looked
// up once per device with cudaGetSymbolAddress and passed to the kernels.
static __device__ __align__(256) unsigned char g_static_scratch[LORADS_STATIC_SCRATCH_BYTES];

__global__ void static_negate_kernel(const double* lam, double* y, int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    y[i] = -lam[i];
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_addr[kMaxDevices] = {};

// device address of g_static_scratch on `device`, which must be current
int static_scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return LORADS_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_addr[device] == nullptr) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return LORADS_ERR_CUDA;
    }
    g_static_addr[device] = static_cast<unsigned char*>(ptr);
  }
  *out = g_static_addr[device];
  return LORADS_OK;
}

// bump carving of the fixed array; never allocates
struct StaticCarve {
  unsigned char* base;
  size_t cap;
  size_t used;
  template <typename X>
  X* take(size_t count) {
    const size_t bytes = ((count * sizeof(X) + 255) / 256) * 256;
    if (used + bytes > cap) return nullptr;
    X* q = reinterpret_cast<X*>(base + used);
    used += bytes;
    return q;
  }
};

// switches to the problem's device for the call and restores the caller's device after
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    if (!ok) cudaGetLastError();
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

// Set-up of lorads_solve_static on `device` (current), done when a problem is assembled:
// loads the modules of the solver kernels and of this file (CUDA loads modules lazily by
// default, and loading one allocates device memory for its code and its __device__ data,
// g_static_scratch included) and resolves the array's address.  Failures are left for the
// static call itself to report.
static void static_path_setup(int device) {
  unsigned char* base = nullptr;
  int per_sm = 0;
  for (int sub = 0; sub < 2; ++sub) {
    Launch<float>::block_capacity(sub, SOLVER_THREADS, &per_sm);
    Launch<float>::grid_capacity(sub, SOLVER_THREADS, &per_sm);
    Launch<double>::block_capacity(sub, SOLVER_THREADS, &per_sm);
    Launch<double>::grid_capacity(sub, SOLVER_THREADS, &per_sm);
  }
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, static_negate_kernel);
  cudaGetLastError();
  static_scratch_address(device, &base);
}

template <typename T>
static int run_solve_static(lorads_problem* p, const lorads_params* prm, cudaStream_t s,
                            double* U_hat, int64_t ldu, double* y, lorads_result* res) {
  const int64_t n = p->n, m = p->m;
  // The solve's state lives in the shared scratch array; p's own arena (and with it the
  // last lorads_solve's solution and checkpoint, which lorads_get_solution / get_state
  // read) is left as it is.
  DevParams dv;
  const int pst = fill_params(p, prm, dv);
  if (pst != LORADS_OK) return pst;
  const int cap = dv.rank_cap;
  if (!dv.phase1 && (!p->has_start || p->start_r > 256)) return LORADS_ERR_STATE;
  const int rmax = std::max(cap, dv.phase1 ? 0 : p->start_r);
  const long long ld_cap = round4(rmax);
  if (U_hat != nullptr && ldu < rmax) return LORADS_ERR_ARG;
  const size_t NS = (size_t)n * ld_cap;
  const int ring = dv.lbfgs_mem + 1;
  const bool mixed = sizeof(T) == 4;
  int dev_sms = 0;
  CU(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, p->device));
  bool whole = false;
  int grid = 1, threads = SOLVER_THREADS;
  int st = solve_geometry<T>(p, prm, dv, dev_sms, &whole, &grid, &threads);
  if (st != LORADS_OK) return st;
  unsigned char* base = nullptr;
  st = static_scratch_address(p->device, &base);
  if (st != LORADS_OK) return st;
  StaticCarve a{base, (size_t)LORADS_STATIC_SCRATCH_BYTES, 0};
  SolverArgs<T> h{};
  h.P = p->dp;
  h.prm = dv;
  h.U = a.take<double>(NS);
  h.V = a.take<double>(NS);
  if (mixed) {
    h.Ut = a.take<T>(NS);
    h.Vt = a.take<T>(NS);
  } else {
    h.Ut = reinterpret_cast<T*>(h.U);
    h.Vt = reinterpret_cast<T*>(h.V);
  }
  h.Dl = a.take<T>(NS);
  h.R = a.take<T>(NS);
  h.Pd = a.take<T>(NS);
  h.HP = a.take<T>(NS);
  h.Sv = a.take<T>(NS);
  h.lam = a.take<double>(m);
  h.e = a.take<double>(m);
  h.cq = a.take<double>(3 * (size_t)p->dp.nchunk + m);
  h.grad = a.take<double>(NS);
  h.grad_old = a.take<double>(NS);
  h.dir = a.take<double>(NS);
  h.tmp = a.take<double>(NS);
  h.CWn = a.take<double>(NS);
  h.S = a.take<double>(NS * ring);
  h.Y = a.take<double>(NS * ring);
  h.lz_store = nullptr;              // the escape vector by the second pass: no room here
  h.ld_cap = ld_cap;
  SolverArgs<T>* dargs = a.take<SolverArgs<T>>(1);
  SolveOut* dout = a.take<SolveOut>(1);
  GridCtl* dctl = a.take<GridCtl>(1);
  double* dpartials = a.take<double>((size_t)dev_sms * 8 * MAXRED * 3);
  int* dqueue = a.take<int>(4);
  if (!h.U || !h.V || !h.Ut || !h.Vt || !h.Dl || !h.R || !h.Pd || !h.HP || !h.Sv || !h.lam ||
      !h.e || !h.cq || !h.grad || !h.grad_old || !h.dir || !h.tmp || !h.CWn || !h.S || !h.Y ||
      !dargs || !dout || !dctl || !dpartials || !dqueue)
    return LORADS_ERR_TOO_LARGE;
  h.out = dout;
  if (!dv.phase1) {
    st = upload_start(p, h.U, h.V, h.lam, s);
    if (st != LORADS_OK) return st;
  }
  // what must start at zero: the report, the grid barrier and the CTA queue
  CU(cudaMemcpyAsync(dargs, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  SolveOut unreached{};
  unreached.status = ST_DEVICE;
  CU(cudaMemcpyAsync(dout, &unreached, sizeof(SolveOut), cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(dctl, 0, sizeof(GridCtl), s));
  CU(cudaMemsetAsync(dpartials, 0xFF, sizeof(double) * (size_t)dev_sms * 8 * MAXRED * 3, s));
  CU(cudaMemsetAsync(dqueue, 0, 16, s));
  cudaError_t le;
  if (!whole) {
    le = Launch<T>::solve_block(dv.subsolver, dargs, 1, dqueue, 1, threads, s);
  } else {
    le = Launch<T>::solve_grid(dv.subsolver, dargs, dctl, dpartials, barrier_polls(prm), grid,
                               threads, s);
  }
  CU(le);
  SolveOut out{};
  CU(cudaMemcpyAsync(&out, dout, sizeof(out), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (out.ld > 0) {
    if (U_hat != nullptr && out.rank > 0)
      CU(cudaMemcpy2DAsync(U_hat, (size_t)ldu * 8, h.tmp, (size_t)out.ld * 8,
                           (size_t)out.rank * 8, (size_t)n, cudaMemcpyDeviceToDevice, s));
    if (y != nullptr) {
      static_negate_kernel<<<std::max(1, std::min(dev_sms * 4, (int)((m + 255) / 256))), 256, 0,
                             s>>>(h.lam, y, (int)m);
      CU(cudaGetLastError());
    }
    CU(cudaStreamSynchronize(s));
  }
  if (res) {
    lorads_result r;
    to_result(out, r);
    *res = r;
  }
  return out.status;
}

extern "C" int lorads_solve_static(lorads_problem* p, const lorads_params* prm, void* stream,
                                   double* U_hat, int64_t ldu, double* y, lorads_result* res) {
  if (res) std::memset(res, 0, sizeof(*res));
  int st = LORADS_OK;
  if (!p || !prm) {
    st = LORADS_ERR_ARG;
  } else if (prm->precision != LORADS_PREC_FP64 && prm->precision != LORADS_PREC_MIXED) {
    st = LORADS_ERR_ARG;
  } else if (!(prm->tol > 0) || prm->max_admm_iter < 1 || prm->cg_max_iter < 1) {
    st = LORADS_ERR_ARG;
  } else if (!p->assembled || p->assemble_status != LORADS_OK) {
    st = LORADS_ERR_STATE;       // assembling would allocate
  } else {
    DeviceGuard guard(p->device);
    if (!guard.ok) {
      st = LORADS_ERR_CUDA;
    } else {
      cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
      st = prm->precision == LORADS_PREC_MIXED
               ? run_solve_static<float>(p, prm, s, U_hat, ldu, y, res)
               : run_solve_static<double>(p, prm, s, U_hat, ldu, y, res);
    }
  }
  if (res) res->status = st;
  return st;
}
