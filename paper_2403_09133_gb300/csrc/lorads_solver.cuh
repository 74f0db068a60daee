// Persistent device solver for LoRADS (Algorithm 2).
//
// The whole method runs inside one launch: Phase I (augmented Lagrangian on the BM
// problem, L-BFGS with exact quartic line search, dynamic rank), the switch, Phase II
// (Algorithm 1 with warm-started CG on eq. linU / eq. linV, dual step, penalty schedule)
// and the output step U_hat = (U + V)/2 with its residuals.  It is written once against a
// "scope": one CTA (BlockScope: small problems and batches, one CTA per problem) or the
// whole grid of a cooperative launch (GridScope: one large problem).  Every scalar decision
// is taken redundantly by all threads from reduced values, so control flow is uniform.
//
// Precision: T is the element type of the CG operators and vectors (double: plain FP64,
// float: mixed form).  The masters U, V, lambda, the CG scalars alpha/beta, all residual
// norms and the objective stay FP64; the CG of each subproblem solves for the correction
// delta of H delta = R_0, R_0 = G - H X_0 formed in FP64 from the warm start X_0.
#pragma once
#include "lorads_device.cuh"

namespace lorads {

struct DevParams {
  int r0, rank_cap;
  double rank_factor;
  double tol, switch_tol, h, rho_max, rho_growth;
  int rho_every;
  double gamma;
  int max_admm_iter, cg_max_iter;
  double cg_rel_tol, cg_abs_floor;
  int lbfgs_mem, inner_max_iter;
  double inner_tol_factor, inner_tol_max;
  int max_outer;
  double sigma_factor, sigma_decrease, sigma_max, new_col_std;
  unsigned long long seed;
  int phase1;
  int r_start;
  double rho0;
  long long time_limit_ns;
  double* iter_log;     // Phase II per-iteration log (NULL: off), iter_log_cap rows of 6
  int iter_log_cap;
  int team_mult;   // lanes per row = team_mult * the minimum for ld (autotuned for batches)
  int kkt_dinf;    // the Appendix B dual infeasibility is part of the final test
  int lanczos_steps;
  int dinf_every;
  double escape_scale;   // Phase II rank growth along the lambda_min eigenvector (0: off)
  int subsolver;         // 0: CG on eq. linU / linV; 1: exact row-block solve (the kernel's SUB)
  int polish;            // Phase III (Newton on the product of spheres) where it applies
  int newton_max, newton_cg_max;
  // continuation of a checkpointed Phase II (resume = 1): V is given apart from U, and the
  // iteration counter, the final-test schedule and the reported counters go on from here
  int resume;
  int nz0;               // Phase II start: columns nz0 .. r_start-1 of the start are zero
  int k0, next_test0, cg0, hess0, outer0, lbfgs0, growths0;
  double prev_dinf0, sigma0;
};

constexpr int LANCZOS_MAX = 2048;  // Lanczos steps of one lambda_min estimate, at most
constexpr int REFINE_CHUNK = 25;   // Phase III augmented-Lagrangian outer iterations between dual tests

struct SolveOut {
  int status, rank, ld, admm_iters, cg_iters, hess_applies, alm_outer, lbfgs_iters, growths;
  int phase;            // 2 once Phase II has started (U, V, lambda form a Phase II iterate)
  int next_dual_test;   // final-test schedule at exit (continued by a resume)
  int pad;
  double prev_dinf;
  double objective, dual_objective, r_P, r_P_split, r_stop, r_D, gap, rho, gamma, sigma;
  double p_infeas, d_infeas, lambda_min, dual_psd;
  long long t_phase1_ns, t_phase2_ns, t_phase3_ns;
  int polished, newton_steps, newton_cg, refine_outer, refine_lbfgs, lanczos_steps;
  long long t_lanczos_ns;
};

// status values written to SolveOut (mirror the public codes)
enum { ST_OK = 0, ST_MAXITER = -5, ST_TIMEOUT = -6, ST_NAN = -7, ST_DEVICE = -9 };

template <typename T>
struct SolverArgs {
  DevProblem P;
  DevParams prm;
  double* U;      // masters, capacity n * ld_cap
  double* V;
  T* Ut;          // shadows of U, V in T (alias U, V when T is double)
  T* Vt;
  T* Dl;          // CG correction delta
  T* R;
  T* Pd;
  T* HP;
  T* Sv;          // s = H p of the single-reduction CG (row-local form)
  double* lam;    // m
  double* e;      // m
  double* cq;     // multi-entry constraints: 3 * nchunk chunk sums, then m values q_i
  double* grad;   // n * ld_cap (Phase I)
  double* grad_old;
  double* dir;
  double* S;      // lbfgs_mem * n * ld_cap
  double* Y;
  double* tmp;    // n * ld_cap (rank growth, U_hat)
  double* CWn;    // n * ld_cap: -(C W) of the row-local Phase II pipeline
  // Phase II reuses grad / grad_old / dir as the three n x 4 Lanczos blocks and S as the
  // Lanczos coefficients (8 per step; S holds ring * n * ld_cap >= 8 n doubles)
  double* lz_store;   // null, or slots 0..Kmax of n x 4 doubles: every Lanczos block of a test
  long long ld_cap;
  SolveOut* out;
};

__device__ inline long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

__host__ __device__ inline int round4(int r) { return (r + 3) & ~3; }

// real roots of c3 t^3 + c2 t^2 + c1 t + c0 (c3 != 0) by the trigonometric / Cardano
// formulas, each polished by two Newton steps; returns the count
__device__ inline int cubic_roots(double c3, double c2, double c1, double c0, double* x) {
  const double B = c2 / c3, C = c1 / c3, D = c0 / c3;
  const double p = C - B * B / 3.0;
  const double q = 2.0 * B * B * B / 27.0 - B * C / 3.0 + D;
  const double disc = 0.25 * q * q + p * p * p / 27.0;
  int k = 0;
  if (disc > 0.0) {
    const double s = sqrt(disc);
    x[k++] = cbrt(-0.5 * q + s) + cbrt(-0.5 * q - s) - B / 3.0;
  } else if (p == 0.0) {
    x[k++] = -B / 3.0;
  } else {
    const double m = 2.0 * sqrt(-p / 3.0);
    double arg = 3.0 * q / (p * m);
    arg = fmin(1.0, fmax(-1.0, arg));
    const double th = acos(arg) / 3.0;
    for (int j = 0; j < 3; ++j) x[k++] = m * cos(th - 2.0 * M_PI * j / 3.0) - B / 3.0;
  }
  for (int j = 0; j < k; ++j) {
    for (int it = 0; it < 2; ++it) {
      const double t = x[j];
      const double f = ((t + B) * t + C) * t + D;
      const double df = (3.0 * t + 2.0 * B) * t + C;
      if (df != 0.0) x[j] = t - f / df;
    }
  }
  return k;
}

// argmin over t > 0 of a1 t + a2 t^2 + a3 t^3 + a4 t^4; 0 when nothing decreases
__device__ inline double quartic_step(double a1, double a2, double a3, double a4) {
  double roots[3];
  int k = 0;
  if (a4 != 0.0) {
    k = cubic_roots(4.0 * a4, 3.0 * a3, 2.0 * a2, a1, roots);
  } else if (a3 != 0.0) {
    const double A = 3.0 * a3, Bq = 2.0 * a2, Cq = a1;
    const double d = Bq * Bq - 4.0 * A * Cq;
    if (d >= 0.0) {
      roots[k++] = (-Bq + sqrt(d)) / (2.0 * A);
      roots[k++] = (-Bq - sqrt(d)) / (2.0 * A);
    }
  } else if (a2 != 0.0) {
    roots[k++] = -a1 / (2.0 * a2);
  }
  double best = 0.0, fbest = 0.0;
  for (int j = 0; j < k; ++j) {
    const double t = roots[j];
    if (!(t > 0.0)) continue;
    const double f = (((a4 * t + a3) * t + a2) * t + a1) * t;
    if (f < fbest) {
      fbest = f;
      best = t;
    }
  }
  return best;
}

// SUB selects the Phase II subproblem solver at compile time: 0 = CG (every constraint
// structure), 1 = the exact row-block solve (row-local problems only), so that neither
// kernel carries the other's code
template <typename T, class Scope, int SUB = 0>
struct Solver {
  const SolverArgs<T>& A;
  Scope& sc;
  const DevProblem& P;
  const DevParams& prm;
  int n, m, r, ld;
  Team tm;
  Team tmc;  // team geometry for constraint loops (same as tm)
  long long t_start;
  int status;
  // counters
  int cg_iters, hess, admm_iters, alm_outer, lbfgs_iters, growths;
  double last_rs;
  double last_lmin;   // latest lambda_min(C - A^T y) estimate ...
  int lmin_at;        // ... and the Phase II iteration count it belongs to (-1: none)
  double uh_norm2;    // ||U_hat||_F^2 from the latest gap test
  double rs_num, rs_den;   // ||V^{k+1} - V^k||^2, ||V^k||^2 of the row-local loop (< 0: unused)
  int ndt;            // first Phase II iteration at which the dual-infeasibility test may run
  double pdinf;       // dual measure of the latest failed test since the last growth
  double last_rd2;    // ||(C + A^T lambda) U_hat||_F^2 from the latest final test
  bool to_polish;     // Phase II handed its output to Phase III
  bool fp64_bulk;     // Phase I's bulk products read the FP64 masters (Phase III refinement)
  bool alm_done;      // the augmented Lagrangian loop met its stopping rule
  int refine_outer, refine_lbfgs;
  int newton_steps, newton_cg;
  int lz_steps;       // Lanczos steps (both passes) over the solve
  long long lz_ns;    // device time spent in lanczos_lambda_min
  int lz_len[4], lz_cs;  // the last first pass: recurrence lengths, column of the estimate
  double lz_qs0[4], lz_best;
  long long t_p3;     // start of Phase III (0: none)
  int nzc;            // columns nzc .. r-1 of U and V are zero (the padding of a rank growth)

  __device__ Solver(const SolverArgs<T>& a, Scope& s)
      : A(a), sc(s), P(a.P), prm(a.prm), n(a.P.n), m(a.P.m), r(0), ld(0), status(ST_OK),
        cg_iters(0), hess(0), admm_iters(0), alm_outer(0), lbfgs_iters(0), growths(0),
        last_rs(0.0), last_lmin(NAN), lmin_at(-1), uh_norm2(0.0), rs_num(-1.0), rs_den(0.0),
        ndt(0), pdinf(NAN), last_rd2(0.0), to_polish(false), fp64_bulk(false), alm_done(false),
        refine_outer(0), refine_lbfgs(0), newton_steps(0), newton_cg(0), lz_steps(0), lz_ns(0), t_p3(0), nzc(0) {}

  __device__ void set_rank(int rr) {
    r = rr;
    ld = round4(rr);
    tm = make_team(ld, sc.tid(), sc.nthreads(), prm.team_mult);
    tmc = tm;
  }

  // ----------------------------------------------------------------------------------
  // Phase I pieces.  Masters (U, the direction, gradients, L-BFGS pairs) and every scalar
  // are FP64; the bulk products (residual SDDMM, gradient SpMM, line-search products) read
  // T shadows of U (A.Ut) and of the direction (A.Dl, free until Phase II), so the mixed
  // form runs them in FP32.  For T = double the shadows alias the masters.
  // ----------------------------------------------------------------------------------
  __device__ T* dir_shadow() const {
    return ((const void*)A.Ut == (const void*)A.U) ? reinterpret_cast<T*>(A.dir) : A.Dl;
  }
  __device__ __forceinline__ void store_shadow(const Frag<double>& f, T* dst, int j) const {
    if ((const void*)dst == (const void*)A.U || (const void*)dst == (const void*)A.dir) return;
    Frag<T> t;
    frag_convert(t, f);
    frag_store(t, dst, j, ld, tm);
  }

  __device__ void init_factor() {
    const uint64_t key = stream_key(prm.seed, 0);
    const double inv = 1.0 / sqrt((double)r);
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> f;
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) {
          const int c = (tm.lane + k * tm.G) * CHUNK + e;
          f.v[k][e] = (c < r) ? normal_at(key, (uint64_t)j * r + c) * inv : 0.0;
        }
      if (P.row_norm != nullptr && P.row_norm[j] > 0.0) {
        const double nr = sqrt(frag_dot(f, f, tm));
        const double s = P.row_norm[j] / nr;
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
#pragma unroll
          for (int e = 0; e < CHUNK; ++e) f.v[k][e] *= s;
      }
      frag_store(f, A.U, j, ld, tm);
      store_shadow(f, A.Ut, j);
    }
  }

  // ----------------------------------------------------------------------------------
  // Multi-entry constraints: the products <A_i, X Y^T> are sums over each constraint's
  // entries.  One team per chunk of at most CON_CHUNK entries forms K per-entry sums
  // f(r, c, a, s) at once (so a long constraint such as tr X = 1 is spread over many teams);
  // after a barrier, con_total(i, k) adds constraint i's chunks in a fixed order.
  // ----------------------------------------------------------------------------------
  template <int K, typename F>
  __device__ bool con_chunks(F f) {
    const int nch = P.nchunk;
    for (int ch = tmc.id; ch < nch; ch += tmc.count) {
      double s[K];
#pragma unroll
      for (int k = 0; k < K; ++k) s[k] = 0.0;
      for (int e = P.chunk_ptr[ch]; e < P.chunk_ptr[ch + 1]; ++e)
        f(P.con_r[e], P.con_c[e], P.con_a[e], s);
      if (tmc.lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) A.cq[(long long)k * nch + ch] = s[k];
      }
    }
    return sc.sync();
  }

  __device__ double con_total(int i, int k) const {
    const double* part = A.cq + (long long)k * P.nchunk;
    double s = 0.0;
    for (int ch = P.con_chunk[i]; ch < P.con_chunk[i + 1]; ++ch) s += part[ch];
    return s;
  }

  // q_i = <A_i, X Y^T> for every constraint into A.cq + 3 nchunk, visible to the whole scope
  template <typename E>
  __device__ bool con_q(const E* X, const E* Y) {
    if (!con_chunks<1>([&](int r, int c, double a, double* s) {
          s[0] += sddmm_entry<E>(X, Y, ld, r, c, a, tmc);
        }))
      return false;
    double* q = A.cq + 3LL * P.nchunk;
    for (int i = sc.tid(); i < m; i += sc.nthreads()) q[i] = con_total(i, 0);
    return sc.sync();
  }

  // Phase II per-iteration log: row k = (k + 1, rho, r_P of U V^T, r_P of U_hat U_hat^T, CG
  // iterations so far, device time in s since the solve started), written by the leader
  __device__ void log_iter(int k, double rho, double e2, double eh2, double t_ns) const {
    if (prm.iter_log == nullptr || k >= prm.iter_log_cap || !sc.is_leader()) return;
    double* row = prm.iter_log + (size_t)k * 6;
    row[0] = (double)(k + 1);
    row[1] = rho;
    row[2] = sqrt(e2) / (1.0 + P.b_inf);
    row[3] = sqrt(eh2) / (1.0 + P.b_inf);
    row[4] = (double)cg_iters;
    row[5] = t_ns * 1e-9;
  }

  // e = A(U U^T) - b (stored), returns ||e||^2
  template <typename E>
  __device__ bool eval_residual_UU_e(const E* Ub, double& e2) {
    double v[1] = {0.0};
    if (P.a_multi) {
      if (!con_chunks<1>([&](int r, int c, double a, double* s) {
            s[0] += sddmm_entry<E>(Ub, Ub, ld, r, c, a, tmc);
          }))
        return false;
      for (int i = sc.tid(); i < m; i += sc.nthreads()) {
        const double ei = con_total(i, 0) - P.b[i];
        A.e[i] = ei;
        v[0] += ei * ei;
      }
    } else {
      for (int i = tmc.id; i < m; i += tmc.count) {
        const double q = sddmm_con<E>(P, Ub, Ub, ld, i, tmc);
        const double ei = q - P.b[i];
        if (tmc.lane == 0) {
          A.e[i] = ei;
          v[0] += ei * ei;
        }
      }
    }
    if (!sc.reduce(v, 1)) return false;
    e2 = v[0];
    return true;
  }

  __device__ bool eval_residual_UU(double& e2) {
    return fp64_bulk ? eval_residual_UU_e<double>(A.U, e2) : eval_residual_UU_e<T>(A.Ut, e2);
  }

  // grad = 2 (C + A^T(lambda + sigma e)) U, returns ||grad||_F^2
  template <typename E>
  __device__ bool eval_grad_e(const E* Ub, double sigma, double& g2) {
    double v[1] = {0.0};
    if (P.a_diag_only) {
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<E> ot;
        Frag<double> out;
        spmm_row<E>(P, Ub, ld, j, A.lam, A.e, 0.0, -1.0, -sigma, E(0), tm, ot);
        frag_convert(out, ot);
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
#pragma unroll
          for (int e = 0; e < CHUNK; ++e) out.v[k][e] *= -2.0;
        frag_store(out, A.grad, j, ld, tm);
        const double d = frag_dot(out, out, tm);
        if (tm.lane == 0) v[0] += d;
      }
    } else {
      // rows with many entries: one warp per row
      const WarpRow wr = make_warp_row(ld, sc.tid(), sc.nthreads(), prm.team_mult);
      for (int j = wr.warp; j < n; j += wr.nwarps) {
        Frag<E> ot;
        Frag<double> out;
        spmm_row_warp<E>(P, Ub, ld, j, A.lam, A.e, 0.0, -1.0, -sigma, E(0), wr, ot);
        frag_convert(out, ot);
        if (wr.sub == 0) {
#pragma unroll
          for (int k = 0; k < KMAX; ++k)
#pragma unroll
            for (int e = 0; e < CHUNK; ++e) out.v[k][e] *= -2.0;
          frag_store(out, A.grad, j, ld, wr.st);
          const double d = frag_dot(out, out, wr.st);
          if (wr.st.lane == 0) v[0] += d;
        }
      }
    }
    if (!sc.reduce(v, 1)) return false;
    g2 = v[0];
    return true;
  }

  __device__ bool eval_grad(double sigma, double& g2) {
    return fp64_bulk ? eval_grad_e<double>(A.U, sigma, g2) : eval_grad_e<T>(A.Ut, sigma, g2);
  }

  // L-BFGS two-loop recursion (Nocedal and Wright, Algorithm 7.4), passes fused with the
  // dot products they feed.  dir <- -H grad; returns <dir, grad>.  The pairs live in a
  // ring of lbfgs_mem + 1 slots: the cnt kept pairs end at head - 1 and slot head is free,
  // so a rejected candidate pair never overwrites a kept one.
  __device__ bool lbfgs_direction(int cnt, int head, const double* hrho, double H0,
                                  double& dg) {
    const int mem = prm.lbfgs_mem + 1;
    const long long NS = (long long)n * A.ld_cap;
    double alpha[MAXMEM + 1], beta_prev = 0.0;
    if (cnt == 0) {
      double v[1] = {0.0};
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<double> g;
        frag_load(g, A.grad, j, ld, tm);
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
#pragma unroll
          for (int e = 0; e < CHUNK; ++e) g.v[k][e] = -g.v[k][e];
        frag_store(g, A.dir, j, ld, tm);
        store_shadow(g, dir_shadow(), j);
        const double d = frag_dot(g, g, tm);
        if (tm.lane == 0) v[0] -= d;
      }
      if (!sc.reduce(v, 1)) return false;
      dg = v[0];
      return true;
    }
    // loop 1: newest -> oldest
    for (int i = 0; i < cnt; ++i) {
      const int slot = (head - 1 - i + 2 * mem) % mem;
      const int prev = (head - i + 2 * mem) % mem;   // slot of pair i-1
      double v[1] = {0.0};
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<double> q, s;
        if (i == 0) {
          frag_load(q, A.grad, j, ld, tm);
        } else {
          Frag<double> y;
          frag_load(q, A.dir, j, ld, tm);
          frag_load(y, A.Y + prev * NS, j, ld, tm);
          frag_axpy(q, -alpha[i - 1], y);
        }
        frag_store(q, A.dir, j, ld, tm);
        frag_load(s, A.S + slot * NS, j, ld, tm);
        const double d = frag_dot(s, q, tm);
        if (tm.lane == 0) v[0] += d;
      }
      if (!sc.reduce(v, 1)) return false;
      alpha[i] = hrho[slot] * v[0];
    }
    // loop 2: oldest -> newest, starting from H0 (q - alpha_last y_last)
    for (int i = 0; i < cnt; ++i) {
      const int slot = (head - cnt + i + 2 * mem) % mem;
      const int ai = cnt - 1 - i;
      double v[1] = {0.0};
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<double> q;
        frag_load(q, A.dir, j, ld, tm);
        if (i == 0) {
          Frag<double> y;
          frag_load(y, A.Y + slot * NS, j, ld, tm);
          frag_axpy(q, -alpha[cnt - 1], y);
#pragma unroll
          for (int k = 0; k < KMAX; ++k)
#pragma unroll
            for (int e = 0; e < CHUNK; ++e) q.v[k][e] *= H0;
        } else {
          const int ps = (slot - 1 + mem) % mem;
          Frag<double> s;
          frag_load(s, A.S + ps * NS, j, ld, tm);
          frag_axpy(q, alpha[ai + 1] - beta_prev, s);
        }
        frag_store(q, A.dir, j, ld, tm);
        Frag<double> y;
        frag_load(y, A.Y + slot * NS, j, ld, tm);
        const double d = frag_dot(y, q, tm);
        if (tm.lane == 0) v[0] += d;
      }
      if (!sc.reduce(v, 1)) return false;
      beta_prev = hrho[slot] * v[0];
    }
    {
      const int last = (head - 1 + 2 * mem) % mem;
      double v[1] = {0.0};
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<double> q, s, g;
        frag_load(q, A.dir, j, ld, tm);
        frag_load(s, A.S + last * NS, j, ld, tm);
        frag_axpy(q, alpha[0] - beta_prev, s);
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
#pragma unroll
          for (int e = 0; e < CHUNK; ++e) q.v[k][e] = -q.v[k][e];
        frag_store(q, A.dir, j, ld, tm);
        store_shadow(q, dir_shadow(), j);
        frag_load(g, A.grad, j, ld, tm);
        const double d = frag_dot(q, g, tm);
        if (tm.lane == 0) v[0] += d;
      }
      if (!sc.reduce(v, 1)) return false;
      dg = v[0];
    }
    return true;
  }

  // dir <- -grad (restart)
  __device__ bool steepest() {
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> g;
      frag_load(g, A.grad, j, ld, tm);
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) g.v[k][e] = -g.v[k][e];
      frag_store(g, A.dir, j, ld, tm);
      store_shadow(g, dir_shadow(), j);
    }
    return sc.sync();
  }

  // quartic coefficients of phi(U + t D) - phi(U)
  template <typename E>
  __device__ bool line_search_coeffs_e(const E* Ub, const E* Dt, double sigma, double* a) {
    double v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = 0.0;
    // <C, U D^T + D U^T> = 2 sum_j D_j . (C U)_j ;  <C, D D^T> = sum_j D_j . (C D)_j
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<E> mCU, mCD, Dj;
      spmm_row<E>(P, Ub, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, E(0), tm, mCU);
      spmm_row<E>(P, Dt, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, E(0), tm, mCD);
      frag_load(Dj, Dt, j, ld, tm);
      const double c1 = -2.0 * (double)frag_dot(Dj, mCU, tm);
      const double c2 = -(double)frag_dot(Dj, mCD, tm);
      if (tm.lane == 0) {
        v[7] += c1;
        v[8] += c2;
      }
    }
    // e1 = <A_i, U D^T + D U^T> = 2 <A_i, U D^T>, e2 = <A_i, D D^T>
    auto accumulate = [&](int i, double e1, double e2) {
      const double l = A.lam[i], e0 = A.e[i];
      v[0] += l * e1;
      v[1] += l * e2;
      v[2] += e0 * e1;
      v[3] += e0 * e2;
      v[4] += e1 * e1;
      v[5] += e1 * e2;
      v[6] += e2 * e2;
    };
    if (P.a_multi) {
      if (!con_chunks<2>([&](int r, int c, double a, double* s) {
            s[0] += 2.0 * sddmm_entry<E>(Ub, Dt, ld, r, c, a, tmc);
            s[1] += sddmm_entry<E>(Dt, Dt, ld, r, c, a, tmc);
          }))
        return false;
      for (int i = sc.tid(); i < m; i += sc.nthreads()) accumulate(i, con_total(i, 0), con_total(i, 1));
    } else {
      for (int i = tmc.id; i < m; i += tmc.count) {
        const int rr = P.con_r[i], cc = P.con_c[i];
        const double aa = P.con_a[i];
        Frag<E> Ur, Dc, Dr, Uc;
        frag_load(Ur, Ub, rr, ld, tmc);
        frag_load(Dc, Dt, cc, ld, tmc);
        frag_load(Dr, Dt, rr, ld, tmc);
        frag_load(Uc, Ub, cc, ld, tmc);
        double e1, e2;
        if (rr != cc) {
          e1 = 2.0 * aa * (double)team_sum(frag_dot_local(Ur, Dc) + frag_dot_local(Uc, Dr), tmc);
          e2 = 2.0 * aa * (double)frag_dot(Dr, Dc, tmc);
        } else {
          e1 = 2.0 * aa * (double)frag_dot(Ur, Dr, tmc);
          e2 = aa * (double)frag_dot(Dr, Dr, tmc);
        }
        if (tmc.lane == 0) accumulate(i, e1, e2);
      }
    }
    if (!sc.reduce(v, 9)) return false;
    a[0] = v[7] + v[0] + sigma * v[2];
    a[1] = v[8] + v[1] + 0.5 * sigma * (v[4] + 2.0 * v[3]);
    a[2] = sigma * v[5];
    a[3] = 0.5 * sigma * v[6];
    return true;
  }

  __device__ bool line_search_coeffs(double sigma, double* a) {
    return fp64_bulk ? line_search_coeffs_e<double>(A.U, A.dir, sigma, a)
                     : line_search_coeffs_e<T>(A.Ut, dir_shadow(), sigma, a);
  }

  // U <- U + t dir; S[head] = t dir; grad_old = grad
  __device__ bool take_step(double t, int head) {
    const long long NS = (long long)n * A.ld_cap;
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> u, d, g;
      frag_load(u, A.U, j, ld, tm);
      frag_load(d, A.dir, j, ld, tm);
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) d.v[k][e] *= t;
      frag_axpy(u, 1.0, d);
      frag_store(u, A.U, j, ld, tm);
      store_shadow(u, A.Ut, j);
      frag_store(d, A.S + head * NS, j, ld, tm);
      frag_load(g, A.grad, j, ld, tm);
      frag_store(g, A.grad_old, j, ld, tm);
    }
    return sc.sync();
  }

  // Y[head] = grad - grad_old; returns s.y and y.y
  __device__ bool history_pair(int head, double& sy, double& yy) {
    const long long NS = (long long)n * A.ld_cap;
    double v[2] = {0.0, 0.0};
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> g, go, s;
      frag_load(g, A.grad, j, ld, tm);
      frag_load(go, A.grad_old, j, ld, tm);
      frag_axpy(g, -1.0, go);
      frag_store(g, A.Y + head * NS, j, ld, tm);
      frag_load(s, A.S + head * NS, j, ld, tm);
      const double a = frag_dot(s, g, tm), b = frag_dot(g, g, tm);
      if (tm.lane == 0) {
        v[0] += a;
        v[1] += b;
      }
    }
    if (!sc.reduce(v, 2)) return false;
    sy = v[0];
    yy = v[1];
    return true;
  }

  // append columns r..r_new-1 drawn N(0, std^2) from sub-stream g (Section 4.3)
  __device__ bool grow_rank(int r_new, int g) {
    const int r_old = r, ld_old = ld;
    const Team t_old = tm;
    for (int j = t_old.id; j < n; j += t_old.count) {
      Frag<double> u;
      frag_load(u, A.U, j, ld_old, t_old);
      frag_store(u, A.tmp, j, ld_old, t_old);
    }
    if (!sc.sync()) return false;
    set_rank(r_new);
    const uint64_t key = stream_key(prm.seed, (uint64_t)g);
    const int extra = r_new - r_old;
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> u;
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) {
          const int c = (tm.lane + k * tm.G) * CHUNK + e;
          double x = 0.0;
          if (c < r_old)
            x = A.tmp[(long long)j * ld_old + c];
          else if (c < r_new)
            x = prm.new_col_std * normal_at(key, (uint64_t)j * extra + (c - r_old));
          u.v[k][e] = x;
        }
      frag_store(u, A.U, j, ld, tm);
      store_shadow(u, A.Ut, j);
    }
    return sc.sync();
  }

  // ----------------------------------------------------------------------------------
  // Phase I: LRALM (Section 4.1) with dynamic rank (Section 4.3)
  // ----------------------------------------------------------------------------------
  __device__ bool phase1(double& sigma_out) { return alm(sigma_out, false, prm.max_outer); }

  // The augmented Lagrangian method of Phase I.  refine = false: from U_0 (init_factor),
  // lambda = 0, sigma_0 = 1/(1+||b||_inf), until r_P <= switch_tol.  refine = true (Phase III
  // outside the product-of-spheres class): from the U in A.U, lambda in A.lam and sigma_io, with
  // the bulk products on the FP64 masters, until r_P <= tol and r_D <= tol, where r_D of the
  // multiplier-updated pair is ||grad phi|| / (2 (1 + ||C||_F)) at the end of an inner solve.
  // alm_done tells whether the stopping rule was met (else max_outer ran out).
  __device__ bool alm(double& sigma_io, bool refine, int max_outer) {
    double sigma;
    if (!refine) {
      for (int i = sc.tid(); i < m; i += sc.nthreads()) A.lam[i] = 0.0;
      init_factor();
      if (!sc.sync()) return false;
      sigma = 1.0 / (1.0 + P.b_inf);
    } else {
      sigma = sigma_io;
      fp64_bulk = true;
    }
    alm_done = false;
    const double tol_g2 = 4.0 * prm.tol * (1.0 + P.C_fro) * prm.tol * (1.0 + P.C_fro);
    double rp_prev = INFINITY, rp = 0.0;
    double hrho[MAXMEM + 1], hsy[MAXMEM + 1], hyy[MAXMEM + 1];
    const int ring = prm.lbfgs_mem + 1;
    for (int outer = 1; outer <= max_outer; ++outer) {
      if (refine) ++refine_outer;
      else alm_outer = outer;
      int cnt = 0, head = 0;
      double e2, g2;
      if (!eval_residual_UU(e2)) return false;
      if (!eval_grad(sigma, g2)) return false;
      int it = 0;
      bool stalled = false;
      for (;;) {
        rp = sqrt(e2) / (1.0 + P.b_inf);
        const double grel = sqrt(g2) / (1.0 + P.C_fro);
        if (!(grel == grel)) { status = ST_NAN; return true; }
        if (grel <= fmax(1e-12, fmin(prm.inner_tol_max, prm.inner_tol_factor * rp))) break;
        if (it >= prm.inner_max_iter) { stalled = true; break; }
        double dg;
        const int newest = (head - 1 + ring) % ring;
        const double H0 = cnt > 0 ? hsy[newest] / hyy[newest] : 1.0;
        if (!lbfgs_direction(cnt, head, hrho, H0, dg)) return false;
        if (dg >= 0.0) {
          if (!steepest()) return false;
          cnt = 0;
          head = 0;
        }
        double a[4];
        if (!line_search_coeffs(sigma, a)) return false;
        const double t = quartic_step(a[0], a[1], a[2], a[3]);
        if (!(t > 0.0)) {
          if (cnt > 0) { cnt = 0; head = 0; continue; }
          break;
        }
        if (!take_step(t, head)) return false;
        if (!eval_residual_UU(e2)) return false;
        if (!eval_grad(sigma, g2)) return false;
        double sy, yy;
        if (!history_pair(head, sy, yy)) return false;
        if (sy > 0.0) {
          hrho[head] = 1.0 / sy;
          hsy[head] = sy;
          hyy[head] = yy;
          head = (head + 1) % ring;
          cnt = cnt < prm.lbfgs_mem ? cnt + 1 : prm.lbfgs_mem;
        }
        ++it;
      }
      if (refine) refine_lbfgs += it;
      else lbfgs_iters += it;
      if (refine ? (rp <= prm.tol && g2 <= tol_g2) : (rp <= prm.switch_tol)) {
        for (int i = sc.tid(); i < m; i += sc.nthreads()) A.lam[i] += sigma * A.e[i];
        if (!sc.sync()) return false;
        alm_done = true;
        break;
      }
      if (stalled && r < prm.rank_cap) {
        ++growths;
        int r_new = (int)ceil(prm.rank_factor * r - 1e-9);
        if (r_new > prm.rank_cap) r_new = prm.rank_cap;
        if (!grow_rank(r_new, growths)) return false;
        nzc = r;
        continue;
      }
      for (int i = sc.tid(); i < m; i += sc.nthreads()) A.lam[i] += sigma * A.e[i];
      if (!sc.sync()) return false;
      if (rp > prm.sigma_decrease * rp_prev) sigma = fmin(sigma * prm.sigma_factor, prm.sigma_max);
      rp_prev = rp;
    }
    sigma_io = sigma;
    return true;
  }

  // ----------------------------------------------------------------------------------
  // Phase II: one CG solve of eq. linU / eq. linV with fixed factor W, warm start X_0 = W
  // ----------------------------------------------------------------------------------
  // R_0 = G - H W with G = (A^T(rho b - lambda) - C) W + gamma W, computed in FP64:
  //   R_0j = sum_{entries} a (rho b_i - lambda_i - rho q_i) W_k - (C W)_j,
  //   q_i = <A_i, W W^T>  (the gamma terms cancel because X_0 = W).
  __device__ bool cg_solve(const double* Wm, const T* Wt, double* Xm, T* Xt, double rho,
                           double gamma, bool want_dv, double* dv) {
    double v[2] = {0.0, 0.0};
    // one warp per row (entries split across sub-teams): rows with many entries
    const WarpRow wr = make_warp_row(ld, sc.tid(), sc.nthreads(), prm.team_mult);
    const Team& st = wr.st;
    // multi-entry constraints: q_i = <A_i, W W^T> for every constraint first
    const bool multi = P.a_multi != 0;
    const double* qv = A.cq + 3LL * P.nchunk;
    if (multi && !con_q<double>(Wm, Wm)) return false;
    for (int j = wr.warp; j < n; j += wr.nwarps) {
      Frag<double> Wj, accR, accG;
      frag_load(Wj, Wm, j, ld, st);
      frag_zero(accR);
      frag_zero(accG);
      for (int q = P.A_rp[j] + wr.sub; q < P.A_rp[j + 1]; q += wr.S) {
        const int k = P.A_col[q], i = P.A_con[q];
        const double a = P.A_val[q];
        double qi;
        Frag<double> Wk;
        if (k == j)
          Wk = Wj;
        else
          frag_load(Wk, Wm, k, ld, st);
        if (multi)
          qi = qv[i];
        else
          qi = (k == j ? 1.0 : 2.0) * a * frag_dot(Wj, Wk, st);
        const double w = rho * P.b[i] - A.lam[i];
        frag_axpy(accG, a * w, Wk);
        frag_axpy(accR, a * (w - rho * qi), Wk);
      }
      for (int q = P.C_rp[j] + wr.sub; q < P.C_rp[j + 1]; q += wr.S) {
        Frag<double> Wk;
        frag_load(Wk, Wm, P.C_col[q], ld, st);
        frag_axpy(accR, -P.C_val[q], Wk);
        frag_axpy(accG, -P.C_val[q], Wk);
      }
      frag_warp_combine(accR, st.G);
      frag_warp_combine(accG, st.G);
      frag_axpy(accG, gamma, Wj);
      if (wr.sub == 0) {
        Frag<T> Rt, Zt;
        frag_convert(Rt, accR);
        frag_zero(Zt);
        frag_store(Rt, A.R, j, ld, st);
        frag_store(Rt, A.Pd, j, ld, st);
        frag_store(Zt, A.Dl, j, ld, st);
        Frag<double> Rd;
        frag_convert(Rd, Rt);
        const double a1 = frag_dot(Rd, Rd, st), a2 = frag_dot(accG, accG, st);
        if (st.lane == 0) {
          v[0] += a1;
          v[1] += a2;
        }
      }
    }
    if (!sc.reduce(v, 2)) return false;
    ++hess;
    double rr = v[0];
    const double target = fmax(prm.cg_rel_tol * sqrt(rr), prm.cg_abs_floor * sqrt(v[1]));
    const T rho_t = (T)rho, gamma_t = (T)gamma;
    int it = 0;
    while (sqrt(rr) > target && it < prm.cg_max_iter) {
      // HP = H P, p.Hp
      double w[1] = {0.0};
      if (multi && !con_q<T>(A.Pd, Wt)) return false;
      for (int j = wr.warp; j < n; j += wr.nwarps) {
        Frag<T> Pj, Hj;
        frag_load(Pj, A.Pd, j, ld, st);
        if (multi)
          hessian_row_q_warp<T>(P, Wt, ld, j, Pj, qv, rho_t, gamma_t, wr, Hj);
        else
          hessian_row_warp<T>(P, Wt, A.Pd, ld, j, Pj, rho_t, gamma_t, wr, Hj);
        if (wr.sub == 0) {
          frag_store(Hj, A.HP, j, ld, st);
          const double d = (double)team_sum(frag_dot_local(Pj, Hj), st);
          if (st.lane == 0) w[0] += d;
        }
      }
      if (!sc.reduce(w, 1)) return false;
      ++hess;
      const double pHp = w[0];
      if (!(pHp > 0.0)) {
        if (!(pHp == pHp)) status = ST_NAN;
        break;
      }
      const double alpha = rr / pHp;
      const T alpha_t = (T)alpha;
      double z[1] = {0.0};
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<T> Dj, Pj, Rj, Hj;
        frag_load(Dj, A.Dl, j, ld, tm);
        frag_load(Pj, A.Pd, j, ld, tm);
        frag_load(Rj, A.R, j, ld, tm);
        frag_load(Hj, A.HP, j, ld, tm);
        frag_axpy(Dj, alpha_t, Pj);
        frag_axpy(Rj, -alpha_t, Hj);
        frag_store(Dj, A.Dl, j, ld, tm);
        frag_store(Rj, A.R, j, ld, tm);
        Frag<double> Rd;
        frag_convert(Rd, Rj);
        const double d = frag_dot(Rd, Rd, tm);
        if (tm.lane == 0) z[0] += d;
      }
      if (!sc.reduce(z, 1)) return false;
      ++it;
      const double rr_new = z[0];
      if (sqrt(rr_new) <= target) { rr = rr_new; break; }
      const T beta_t = (T)(rr_new / rr);
      rr = rr_new;
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<T> Pj, Rj;
        frag_load(Pj, A.Pd, j, ld, tm);
        frag_load(Rj, A.R, j, ld, tm);
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
#pragma unroll
          for (int e = 0; e < CHUNK; ++e) Pj.v[k][e] = fma(beta_t, Pj.v[k][e], Rj.v[k][e]);
        frag_store(Pj, A.Pd, j, ld, tm);
      }
      if (!sc.sync()) return false;
    }
    cg_iters += it;
    // X = W + delta (FP64 master and T shadow)
    dv[0] = 0.0;
    dv[1] = 0.0;
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> Wj, Xj;
      Frag<T> Dj;
      frag_load(Wj, Wm, j, ld, tm);
      frag_load(Dj, A.Dl, j, ld, tm);
      frag_convert(Xj, Dj);
      frag_axpy(Xj, 1.0, Wj);
      if (want_dv) {
        Frag<double> Xo;
        frag_load(Xo, Xm, j, ld, tm);
        const double o2 = frag_dot(Xo, Xo, tm);
        frag_axpy(Xo, -1.0, Xj);
        const double d2 = frag_dot(Xo, Xo, tm);
        if (tm.lane == 0) {
          dv[0] += d2;
          dv[1] += o2;
        }
      }
      frag_store(Xj, Xm, j, ld, tm);
      if ((const void*)Xt != (const void*)Xm) {
        Frag<T> Xs;
        frag_convert(Xs, Xj);
        frag_store(Xs, Xt, j, ld, tm);
      }
    }
    return sc.sync();
  }

  // ----------------------------------------------------------------------------------
  // Row-local form (every constraint a diagonal entry, e.g. MaxCut): eq. linU's matrix is
  // block diagonal, (H x)_j = rho a_j^2 (x_j . W_j) W_j + gamma x_j.  CG runs as the
  // Chronopoulos-Gear recurrence (one grid reduction of r.r and r.Hr per iteration; the
  // same iterates as textbook CG in exact arithmetic), each iteration one pass whose loads
  // are independent (phase2_local below).
  // ----------------------------------------------------------------------------------
  __device__ __forceinline__ void local_h(const Frag<T>& x, const Frag<T>& Wj, T a, T rho,
                                          T gamma, Frag<T>& out) const {
    const T q = rho * a * a * frag_dot(x, Wj, tm);
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
#pragma unroll
      for (int e = 0; e < CHUNK; ++e) out.v[k][e] = fma(q, Wj.v[k][e], gamma * x.v[k][e]);
  }

  // dual step lambda += rho (A(U V^T) - b); partial sums of ||e||^2 and of the output
  // infeasibility ||A(U_hat U_hat^T) - b||^2, U_hat = (U + V)/2
  // entry (r, c, a) of a constraint: its terms of <A_i, U V^T> and <A_i, U_hat U_hat^T>
  __device__ __forceinline__ void dual_entry(int rr, int cc, double a, double& q,
                                             double& qh) const {
    Frag<double> Ur, Vc, Uc, Vr;
    frag_load(Ur, A.U, rr, ld, tmc);
    frag_load(Vc, A.V, cc, ld, tmc);
    frag_load(Uc, A.U, cc, ld, tmc);
    frag_load(Vr, A.V, rr, ld, tmc);
    Frag<double> Hr = Ur, Hc = Uc;
    frag_axpy(Hr, 1.0, Vr);
    frag_axpy(Hc, 1.0, Vc);
    if (rr != cc) {
      q = a * team_sum(frag_dot_local(Ur, Vc) + frag_dot_local(Uc, Vr), tmc);
      qh = 0.5 * a * frag_dot(Hr, Hc, tmc);      // 2 (Hr/2).(Hc/2)
    } else {
      q = a * frag_dot(Ur, Vr, tmc);
      qh = 0.25 * a * frag_dot(Hr, Hr, tmc);
    }
  }

  __device__ bool dual_step(double rho, double* v) {
    auto update = [&](int i, double q, double qh) {
      const double e = q - P.b[i], eh = qh - P.b[i];
      A.lam[i] += rho * e;
      v[0] += e * e;
      v[1] += eh * eh;
    };
    if (P.a_multi) {
      if (!con_chunks<2>([&](int r, int c, double a, double* s) {
            double q, qh;
            dual_entry(r, c, a, q, qh);
            s[0] += q;
            s[1] += qh;
          }))
        return false;
      for (int i = sc.tid(); i < m; i += sc.nthreads()) update(i, con_total(i, 0), con_total(i, 1));
      return true;
    }
    for (int i = tmc.id; i < m; i += tmc.count) {
      double q, qh;
      dual_entry(P.con_r[i], P.con_c[i], P.con_a[i], q, qh);
      if (tmc.lane == 0) update(i, q, qh);
    }
    return true;
  }

  // the dual measure of the final test: max(0, -lambda_min(C - A^T y)) / (1 + ||C||_inf).
  // Appendix B divides the same eigenvalue by 1 + ||vec C||_1, which grows with n.
  __device__ double dual_psd(double lmin) const { return fmax(0.0, -lmin) / (1.0 + P.C_inf); }

  // Phase III applies: every row carries exactly one diagonal constraint with b/a > 0
  __device__ bool polish_applies() const {
    return prm.polish && P.polish_ok && P.row_norm != nullptr;
  }

  // Final test on X = U_hat U_hat^T, y = -lambda^{k+1} once the primal test has passed: the
  // Appendix B gap and the stationarity r_D = ||(C - A^T y) U_hat||_F / (1 + ||C||_F) of
  // eq. def:eKKT (one pass); where Phase III applies, an output that passes the gap with
  // r_D > tol is handed over to it; otherwise the dual measure (rate-limited Lanczos) and r_D
  // must both pass.  A dual measure that fell by less than 10% since the previous failed test
  // (a stationary point of the rank-r problem) grows the rank along the eigenvector of
  // lambda_min.  Returns 1 (done), 0 (continue), 2 (rank grown: U, V changed), 3 (hand over to
  // Phase III), -1 (device error).
  __device__ int final_test() {
    double gap;
    if (!gap_check(gap)) return -1;
    if (!(fabs(gap) <= prm.tol)) return 0;
    const double tol_rd2 = prm.tol * (1.0 + P.C_fro) * prm.tol * (1.0 + P.C_fro);
    const bool rd_ok = last_rd2 <= tol_rd2;
    if (!rd_ok && prm.polish) return 3;
    if (!prm.kkt_dinf) return rd_ok ? 1 : 0;
    if (admm_iters < ndt) return 0;
    if (!lanczos_lambda_min(last_lmin)) return -1;
    lmin_at = admm_iters;
    const double d = dual_psd(last_lmin);
    if (d <= prm.tol && rd_ok) return 1;
    ndt = admm_iters + max(prm.dinf_every, admm_iters / 10);
    if (d <= prm.tol) return 0;
    if (pdinf == pdinf && d > 0.9 * pdinf && escape_possible()) {
      if (!escape_grow()) return -1;
      pdinf = NAN;
      return 2;
    }
    pdinf = d;
    return 0;
  }

  // The escape from a point where lambda_min(C - A^T y) < 0 (Section 4.3's rank rule where the
  // rank-r problem has stalled): the first zero column of U and V (the padding a growth left,
  // which every step keeps at zero) takes tau z, z the Ritz vector of lambda_min, tau =
  // escape_scale ||U_hat||_F / sqrt(r) (uh_norm2 = ||U_hat||_F^2); with no zero column left the
  // rank grows to ceil(1.5 r) (at least r + 1, at most the cap) with new columns [tau z, 0, ...].
  // The caller checks escape_possible() first, right after the failed dual test whose Lanczos
  // coefficients give z.
  __device__ bool escape_possible() const {
    return prm.escape_scale > 0.0 && (nzc < r || r < prm.rank_cap);
  }
  __device__ bool escape_grow() {
    double zn2 = 0.0;
    if (!lanczos_ritz_vector(zn2)) return false;
    const int Kmax = min(min(prm.lanczos_steps, LANCZOS_MAX), n);
    const double* zv = A.Y + 2 * Kmax;
    if (nzc < r) {
      const double tau = zn2 > 0.0 ? prm.escape_scale * sqrt(uh_norm2 / (double)r / zn2) : 0.0;
      const bool shadow = (const void*)A.Ut != (const void*)A.U;
      const int c = nzc;
      for (int j = sc.tid(); j < n; j += sc.nthreads()) {
        const double x = tau * zv[j];
        const long long o = (long long)j * ld + c;
        A.U[o] = x;
        A.V[o] = x;
        if (shadow) {
          A.Ut[o] = (T)x;
          A.Vt[o] = (T)x;
        }
      }
      ++nzc;
      return sc.sync();
    }
    const int r_old = r;
    int r_new = (int)ceil(prm.rank_factor * r - 1e-9);
    if (r_new <= r) r_new = r + 1;
    if (r_new > prm.rank_cap) r_new = prm.rank_cap;
    if (!grow_rank_phase2(r_new, zv, zn2)) return false;
    nzc = r_old + 1;
    ++growths;
    return true;
  }

  __device__ bool phase2(double rho, double& rho_out) {
    if constexpr (SUB == 1) {
      // launched by the host for row-local problems only
      if (!P.a_diag_only) return false;
      return phase2_local_direct(rho, rho_out);
    } else {
      return phase2_cg(rho, rho_out);
    }
  }

  __device__ bool phase2_cg(double rho, double& rho_out) {
    if (P.a_diag_only) return phase2_local(rho, rho_out);
    const double gamma = prm.gamma;
    for (int k = admm_iters; k < prm.max_admm_iter; ++k) {
      double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      double dv[2];
      // U-step: eq. linU with W = V^k, CG warm-started from V^k
      if (!cg_solve(A.V, A.Vt, A.U, A.Ut, rho, gamma, false, dv)) return false;
      if (status != ST_OK) break;
      // V-step: eq. linV with W = U^{k+1}, CG warm-started from U^{k+1}
      if (!cg_solve(A.U, A.Ut, A.V, A.Vt, rho, gamma, true, dv)) return false;
      if (status != ST_OK) break;
      if (!dual_step(rho, v)) return false;
      v[2] = dv[0];
      v[3] = dv[1];
      if (sc.is_leader()) v[4] = (double)(globaltimer_ns() - t_start);
      if (!sc.reduce(v, 5)) return false;
      admm_iters = k + 1;
      log_iter(k, rho, v[0], v[1], v[4]);
      const double rp = sqrt(v[0]) / (1.0 + P.b_inf);
      const double rph = sqrt(v[1]) / (1.0 + P.b_inf);
      const double rs = gamma * sqrt(v[2]) / (1.0 + sqrt(v[3]));
      last_rs = rs;
      if (!(rp == rp) || !(rs == rs)) { status = ST_NAN; break; }
      if (rph <= prm.tol) {
        const int t = final_test();
        if (t < 0) return false;
        if (t == 1 || t == 3) {
          to_polish = t == 3;
          rho_out = rho;
          return true;
        }
      }
      if ((long long)v[4] > prm.time_limit_ns) { status = ST_TIMEOUT; break; }
      if ((k + 1) % prm.rho_every == 0) rho = fmin(rho * prm.rho_growth, prm.rho_max);
    }
    if (status == ST_OK) status = ST_MAXITER;
    rho_out = rho;
    return true;
  }

  // ----------------------------------------------------------------------------------
  // Phase II, row-local form (every constraint a diagonal entry): the subproblems' Hessians
  // are block diagonal, so a CG solve needs no neighbour data; only the warm-start residual
  // R_0 = G - H W reads neighbours, through (C W)_j.  The loop is pipelined: -(C W) is kept
  // per row in FP64 (A.CWn) and advanced with -(C delta) of each CG correction (in T, read
  // from the neighbours' delta after the CG's last barrier), recomputed exactly in FP64 every
  // 32 iterations; so the pass that forms X = W + delta also forms the next subproblem's R_0
  // (U-step finish + V-step R_0; V-step finish + dual step + next U-step R_0), one grid
  // reduction each.  The T shadows of U^{k+1} and V^{k+1} are advanced as shadow(W) + delta
  // and re-rounded from the FP64 masters at the same exact steps.  Same iterates as the
  // unpipelined form up to rounding.
  // ----------------------------------------------------------------------------------
  // row j's constraint (the row-local form has at most one per row): its index (-1: none),
  // a, b and lambda, loaded before a pass stores anything (loads after a store to memory
  // that might alias wait behind it)
  struct RowCon {
    int i;
    double a, b, lam;
  };
  __device__ __forceinline__ RowCon row_con_of(int j) const {
    RowCon c;
    c.i = P.row_con[j];
    c.a = P.row_a[j];
    c.b = c.i >= 0 ? P.b[c.i] : 0.0;
    c.lam = c.i >= 0 ? A.lam[c.i] : 0.0;
    return c;
  }

  // R_0 and w_0 = H r_0 of the local subproblem with fixed factor W on row j, given
  // mCWj = -(C W)_j:  R_0j = -(C W)_j + a (rho b_i - lambda_i - rho q_i) W_j, q_i = a W_j.W_j;
  // ||G||^2 with G_j = R_0j + (a rho q_i + gamma) W_j (only its norm is used) in T
  // (lam_i: lambda of row j's constraint, when it has one)
  // Returns q_i = a ||W_j||^2 (0 without a constraint).
  // With dout (the direct subproblem solve) it stores delta_j = H_j^{-1} R_0j instead of R_0
  // and H R_0: H_j = gamma I + rho a_j^2 W_j W_j^T is inverted by Sherman-Morrison,
  // delta_j = (R_0j - c (W_j.R_0j) W_j) / gamma, c = rho a_j^2 / (gamma + rho a_j^2 ||W_j||^2)
  // (a_j = 0 without a constraint), in T with the shadow of W like the CG it replaces.
  __device__ __forceinline__ double local_r0_row(int j, const Frag<double>& Wj, const Frag<T>& Wjt,
                                                 const Frag<double>& mCWj, const RowCon& c,
                                                 double lam_i, double rho, double gamma,
                                                 double* g3, T* dout = nullptr) {
    Frag<double> accR = mCWj;
    double cg = gamma, qi = 0.0;
    if (c.i >= 0) {
      qi = c.a * frag_dot(Wj, Wj, tm);
      frag_axpy(accR, c.a * (rho * c.b - lam_i - rho * qi), Wj);
      cg += c.a * rho * qi;
    }
    Frag<T> rt, wt, gt;
    frag_convert(rt, accR);
    const T at = (T)c.a;                          // = rowa<T>(P)[j] (0 without a constraint)
    if (dout != nullptr) {
      const T sa = (T)rho * at * at;
      const T c = sa / ((T)gamma + sa * frag_dot(Wjt, Wjt, tm));
      const T cw = -c * frag_dot(Wjt, rt, tm);
      const T ig = T(1) / (T)gamma;
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) wt.v[k][e] = fma(cw, Wjt.v[k][e], rt.v[k][e]) * ig;
      frag_store(wt, dout, j, ld, tm);
      return qi;
    }
    local_h(rt, Wjt, at, (T)rho, (T)gamma, wt);
    frag_store(rt, A.R, j, ld, tm);
    frag_store(wt, A.HP, j, ld, tm);
    gt = rt;
    frag_axpy(gt, (T)cg, Wjt);
    const double d1 = (double)frag_dot(rt, rt, tm), d2 = (double)frag_dot(wt, rt, tm);
    const double d3 = (double)frag_dot(gt, gt, tm);
    if (tm.lane == 0) {
      g3[0] += d1;
      g3[1] += d2;
      g3[2] += d3;
    }
    return qi;
  }

  // -(C X)_j for X = W + delta (delta = D when have_delta): exact FP64 sum over the
  // neighbours' W and delta when exact, else mCWj - (C delta)_j with the product in T
  __device__ __forceinline__ void local_mcx_row(int j, const double* Wm, const T* D,
                                                bool have_delta, bool exact,
                                                const Frag<double>& mCWj, Frag<double>& out) {
    if (exact) {
      Frag<double> acc;
      frag_zero(acc);
      for (int q = P.C_rp[j]; q < P.C_rp[j + 1]; ++q) {
        const int k = P.C_col[q];
        Frag<double> Wk;
        frag_load(Wk, Wm, k, ld, tm);
        if (have_delta) {
          Frag<T> dk;
          Frag<double> dd;
          frag_load(dk, D, k, ld, tm);
          frag_convert(dd, dk);
          frag_axpy(Wk, 1.0, dd);
        }
        frag_axpy(acc, -P.C_val[q], Wk);
      }
      out = acc;
      return;
    }
    out = mCWj;
    if (!have_delta) return;
    Frag<T> mcd;
    spmm_row<T>(P, D, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, T(0), tm, mcd);
    Frag<double> md;
    frag_convert(md, mcd);
    frag_axpy(out, 1.0, md);
  }

  // the U-step's R_0 from W = V with -(C V) computed exactly (start, and after rank growth);
  // with dout the U-step's direct solution delta instead (the reduction is then a barrier)
  __device__ bool local_prologue(double rho, double gamma, double* g3, T* dout = nullptr) {
    g3[0] = g3[1] = g3[2] = 0.0;
    const bool shadow = (const void*)A.Vt != (const void*)A.V;
    for (int j = tm.id; j < n; j += tm.count) {
      const RowCon c = row_con_of(j);
      Frag<double> Wj, mCW;
      Frag<T> Wjt;
      frag_load(Wj, A.V, j, ld, tm);
      if (shadow) frag_load(Wjt, A.Vt, j, ld, tm);
      else frag_convert(Wjt, Wj);
      local_mcx_row(j, A.V, A.Dl, false, true, Wj, mCW);
      frag_store(mCW, A.CWn, j, ld, tm);
      local_r0_row(j, Wj, Wjt, mCW, c, c.lam, rho, gamma, g3, dout);
    }
    if (!sc.reduce(g3, 3)) return false;
    ++hess;
    return true;
  }

  // CG-CG iterations on H delta = r_0 from the R / HP left by the R_0 pass (row-local H).
  // The FP64 scalar recurrence after each reduction is evaluated by thread 0 of every CTA
  // and shared through shared memory (every CTA computes the same values from the same
  // reduced sums), and the stop test compares squares: FP64 divides issue at a small
  // fraction of the FP32 rate on this part, and evaluated in every warp they would queue on
  // each SM's FP64 unit.
  // row j of the in-memory row-local CG step: its r, p, x (p, x zero on the first step) and W
  __device__ __forceinline__ void cg7_load(int j, bool have_px, Frag<T>& r, Frag<T>& pp,
                                           Frag<T>& x, Frag<T>& Wjt, T& aj, const T* Wt,
                                           const T* ra) const {
    frag_load(r, A.R, j, ld, tm);
    frag_load(Wjt, Wt, j, ld, tm);
    aj = ra[j];
    if (have_px) {
      frag_load(pp, A.Pd, j, ld, tm);
      frag_load(x, A.Dl, j, ld, tm);
    } else {
      frag_zero(pp);
      frag_zero(x);
    }
  }
  // p = r + b p, s = H p, x += a p, r -= a s, w = H r; stores p, x, r; z += (r.r, w.r)
  __device__ __forceinline__ void cg7_step(int j, Frag<T>& r, Frag<T>& pp, Frag<T>& x,
                                           const Frag<T>& Wjt, T aj, T a_t, T b_t, T rho_t,
                                           T gamma_t, double* z) const {
    Frag<T> ss, w;
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
#pragma unroll
      for (int e = 0; e < CHUNK; ++e) pp.v[k][e] = fma(b_t, pp.v[k][e], r.v[k][e]);
    local_h(pp, Wjt, aj, rho_t, gamma_t, ss);
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
#pragma unroll
      for (int e = 0; e < CHUNK; ++e) {
        x.v[k][e] = fma(a_t, pp.v[k][e], x.v[k][e]);
        r.v[k][e] = fma(-a_t, ss.v[k][e], r.v[k][e]);
      }
    local_h(r, Wjt, aj, rho_t, gamma_t, w);
    frag_store(pp, A.Pd, j, ld, tm);
    frag_store(x, A.Dl, j, ld, tm);
    frag_store(r, A.R, j, ld, tm);
    const T d1 = frag_dot(r, r, tm), d2 = frag_dot(w, r, tm);
    if (tm.lane == 0) {
      z[0] += (double)d1;
      z[1] += (double)d2;
    }
  }

  __device__ bool cg_local_loop(const T* Wt, double rho, double gamma, const double* g3,
                                int& it) {
    const T rho_t = (T)rho, gamma_t = (T)gamma;
    const T* ra = rowa<T>(P);
    const bool lead = threadIdx.x == 0;
    double* shs = sc.scratch() + 4;   // state (0 go on, 1 stop, 2 NaN), alpha, beta
    // thread 0 carries gamma = r.r and ga = gamma * alpha: with D = delta_new ga - gamma_new^2
    // the Chronopoulos-Gear update alpha_new = gamma_new / (delta_new - beta gamma_new / alpha)
    // is gamma_new ga / D and beta = gamma_new / gamma = gamma_new D / (gamma D), both from the
    // one reciprocal 1 / (gamma D) (the denominator is positive exactly when D is)
    double gam = 0.0, ga = 0.0, target2 = 0.0;
    if (lead) {
      gam = g3[0];
      const double del = g3[1];
      target2 = fmax(prm.cg_rel_tol * prm.cg_rel_tol * gam,
                     prm.cg_abs_floor * prm.cg_abs_floor * g3[2]);
      const double alpha = del > 0.0 ? gam / del : 0.0;
      ga = gam * alpha;
      shs[0] = (gam > target2 && del > 0.0) ? 0.0 : 1.0;
      shs[1] = alpha;
      shs[2] = 0.0;
    }
    __syncthreads();
    int go = shs[0] == 0.0;
    T a_t = (T)shs[1], b_t = T(0);
    __syncthreads();
    it = 0;
    if (tm.count >= n) {
      // at most one row per team: its CG state stays in registers across the iterations
      // (same arithmetic in the same order as below), and only delta is stored at the end
      const int j = tm.id;
      const bool have = j < n;
      Frag<T> r, w, pp, ss, x, Wjt;
      T aj = T(0);
      frag_zero(pp);
      frag_zero(ss);
      frag_zero(x);
      if (have) {
        frag_load(r, A.R, j, ld, tm);
        frag_load(w, A.HP, j, ld, tm);
        frag_load(Wjt, Wt, j, ld, tm);
        aj = ra[j];
      } else {
        frag_zero(r);
        frag_zero(w);
        frag_zero(Wjt);
      }
      while (go && it < prm.cg_max_iter) {
        double z[2] = {0.0, 0.0};
        if (have) {
#pragma unroll
          for (int k = 0; k < KMAX; ++k)
#pragma unroll
            for (int e = 0; e < CHUNK; ++e) {
              pp.v[k][e] = fma(b_t, pp.v[k][e], r.v[k][e]);
              ss.v[k][e] = fma(b_t, ss.v[k][e], w.v[k][e]);
              x.v[k][e] = fma(a_t, pp.v[k][e], x.v[k][e]);
              r.v[k][e] = fma(-a_t, ss.v[k][e], r.v[k][e]);
            }
          local_h(r, Wjt, aj, rho_t, gamma_t, w);
          const T d1 = frag_dot(r, r, tm), d2 = frag_dot(w, r, tm);
          if (tm.lane == 0) {
            z[0] += (double)d1;
            z[1] += (double)d2;
          }
        }
        if (!sc.reduce(z, 2)) return false;
        ++hess;
        ++it;
        if (!cg_scalars(lead, shs, z, target2, gam, ga, go, a_t, b_t)) break;
      }
      if (have && it > 0) frag_store(x, A.Dl, j, ld, tm);
      cg_iters += it;
      return true;
    }
    // Rows in memory (a team owns several): the matrix is row-local, so s = H p and w = H r are
    // formed from p and r in the pass instead of being carried (s = w + beta s) in two more
    // arrays; a CG step reads r, p, x and W and writes r, p and x (7 arrays instead of 11).
    // In exact arithmetic these are the iterates of the recurrence above.
    // (Two rows per trip, their loads issued together, measured slower on the 2048^2 torus:
    // the second row's fragments went to local memory.)
    while (go && it < prm.cg_max_iter) {
      double z[2] = {0.0, 0.0};
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<T> r, pp, x, Wjt;
        T aj = T(0);
        cg7_load(j, it > 0, r, pp, x, Wjt, aj, Wt, ra);
        cg7_step(j, r, pp, x, Wjt, aj, a_t, b_t, rho_t, gamma_t, z);
      }
      if (!sc.reduce(z, 2)) return false;
      ++hess;
      ++it;
      if (!cg_scalars(lead, shs, z, target2, gam, ga, go, a_t, b_t)) break;
    }
    cg_iters += it;
    return true;
  }

  // the Chronopoulos-Gear scalars after a reduction z = (r.r, w.r): thread 0 of the CTA
  // evaluates them (one division) and shares them through shared memory; false when the
  // CG stops (converged, a non-positive denominator, or NaN, which sets the status)
  template <typename S>
  __device__ __forceinline__ bool cg_scalars(bool lead, double* shs, const double* z,
                                             double target2, double& gam, double& ga, int& go,
                                             S& a_t, S& b_t) {
    if (lead) {
      int state = 0;                 // 0: go on, 1: stop, 2: NaN
      const double gam_new = z[0], del_new = z[1];
      double alpha = 0.0, beta = 0.0;
      if (!(gam_new == gam_new) || !(del_new == del_new)) {
        state = 2;
      } else if (gam_new <= target2) {
        state = 1;
      } else {
        const double D = del_new * ga - gam_new * gam_new;
        if (D > 0.0) {
          const double inv = 1.0 / (gam * D);
          beta = gam_new * D * inv;
          alpha = gam_new * ga * gam * inv;
          ga = gam_new * alpha;
          gam = gam_new;
        } else {
          state = 1;                     // rounding made the denominator non-positive
        }
      }
      shs[0] = (double)state;
      shs[1] = alpha;
      shs[2] = beta;
    }
    __syncthreads();
    const int state = (int)shs[0];
    a_t = (S)shs[1];
    b_t = (S)shs[2];
    __syncthreads();
    if (state == 2) status = ST_NAN;
    go = state == 0;
    return state == 0;
  }

  __device__ bool phase2_local(double rho, double& rho_out) {
    const double gamma = prm.gamma;
    const double tol2_primal = prm.tol * (1.0 + P.b_inf) * prm.tol * (1.0 + P.b_inf);
    const bool shadow = (const void*)A.Ut != (const void*)A.U;
    double g3[3];
    if (!local_prologue(rho, gamma, g3)) return false;
    for (int k = admm_iters; k < prm.max_admm_iter; ++k) {
      const bool exact = (k + 1) % 32 == 0;
      // U-step: CG on eq. linU (W = V^k) from the R_0 of the previous pass
      int it;
      if (!cg_local_loop(A.Vt, rho, gamma, g3, it)) return false;
      if (status != ST_OK) break;
      // U^{k+1} = V^k + delta, -(C U^{k+1}), and the V-step's R_0 (W = U^{k+1})
      g3[0] = g3[1] = g3[2] = 0.0;
      for (int j = tm.id; j < n; j += tm.count) {
        const RowCon c = row_con_of(j);
        Frag<double> Wj, Xj, mCW, mCX;
        Frag<T> Xt;
        frag_load(Wj, A.V, j, ld, tm);
        frag_load(mCW, A.CWn, j, ld, tm);
        frag_load(Xt, A.Vt, j, ld, tm);           // (the master itself in the FP64 form)
        Xj = Wj;
        if (it > 0) {
          Frag<T> x;
          Frag<double> xd;
          frag_load(x, A.Dl, j, ld, tm);
          frag_convert(xd, x);
          frag_axpy(Xj, 1.0, xd);
          frag_axpy(Xt, T(1), x);                 // shadow of U^{k+1} = shadow(V^k) + delta
        }
        if (exact) frag_convert(Xt, Xj);          // re-rounded from the master every 32
        local_mcx_row(j, A.V, A.Dl, it > 0, exact, mCW, mCX);
        frag_store(Xj, A.U, j, ld, tm);
        if (shadow) frag_store(Xt, A.Ut, j, ld, tm);
        frag_store(mCX, A.CWn, j, ld, tm);
        const double qU = local_r0_row(j, Xj, Xt, mCX, c, c.lam, rho, gamma, g3);
        if (c.i >= 0 && tm.lane == 0) A.e[c.i] = qU;  // a ||U_j^{k+1}||^2 for the output residual
      }
      if (!sc.reduce(g3, 3)) return false;
      ++hess;
      // V-step: CG on eq. linV (W = U^{k+1})
      if (!cg_local_loop(A.Ut, rho, gamma, g3, it)) return false;
      if (status != ST_OK) break;
      // V^{k+1} = U^{k+1} + delta, the dual step, -(C V^{k+1}) and the next U-step's R_0
      const double rho_next =
          ((k + 1) % prm.rho_every == 0) ? fmin(rho * prm.rho_growth, prm.rho_max) : rho;
      double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int j = tm.id; j < n; j += tm.count) {
        const RowCon c = row_con_of(j);
        const double qU = c.i >= 0 ? A.e[c.i] : 0.0;   // a ||U_j^{k+1}||^2 from pass A
        Frag<double> Wj, Xj, mCW, mCX;
        Frag<T> x, Wt, Vot;
        frag_load(Wj, A.U, j, ld, tm);
        frag_load(mCW, A.CWn, j, ld, tm);
        frag_load(Wt, A.Ut, j, ld, tm);           // (the masters themselves in the FP64 form)
        frag_load(Vot, A.Vt, j, ld, tm);
        Xj = Wj;
        if (it > 0) {
          Frag<double> xd;
          frag_load(x, A.Dl, j, ld, tm);
          frag_convert(xd, x);
          frag_axpy(Xj, 1.0, xd);
        } else {
          frag_zero(x);
        }
        // eq. stop's second term (reported only): ||V^{k+1} - V^k||, ||V^k|| from the shadows
        Frag<T> Xt = Wt, dV = Wt;
        frag_axpy(Xt, T(1), x);                   // shadow of V^{k+1} = shadow(U^{k+1}) + delta
        frag_axpy(dV, T(-1), Vot);
        frag_axpy(dV, T(1), x);
        const double d2 = (double)frag_dot(dV, dV, tm), o2 = (double)frag_dot(Vot, Vot, tm);
        if (exact) frag_convert(Xt, Xj);          // re-rounded from the master every 32
        // dual step lambda_i += rho (a U_j.V_j - b_i)
        double e = 0.0, lam_new = 0.0;
        if (c.i >= 0) {
          e = c.a * frag_dot(Wj, Xj, tm) - c.b;
          lam_new = c.lam + rho * e;        // every lane of the team holds the same value
        }
        local_mcx_row(j, A.U, A.Dl, it > 0, exact, mCW, mCX);
        frag_store(Xj, A.V, j, ld, tm);
        if (shadow) frag_store(Xt, A.Vt, j, ld, tm);
        frag_store(mCX, A.CWn, j, ld, tm);
        const double qV = local_r0_row(j, Xj, Xt, mCX, c, lam_new, rho_next, gamma, v + 5);
        // the output's row residual a ||(U_j + V_j)/2||^2 - b_i from a||U_j||^2 (pass A),
        // a U_j.V_j = e + b_i and a||V_j||^2
        double eh = 0.0;
        if (c.i >= 0) eh = 0.25 * (qU + 2.0 * (e + c.b) + qV) - c.b;
        if (tm.lane == 0) {
          if (c.i >= 0) A.lam[c.i] = lam_new;
          v[0] += e * e;
          v[1] += eh * eh;
          v[2] += d2;
          v[3] += o2;
        }
      }
      if (sc.is_leader()) v[4] = (double)(globaltimer_ns() - t_start);
      if (!sc.reduce(v, 8)) return false;
      ++hess;
      g3[0] = v[5];
      g3[1] = v[6];
      g3[2] = v[7];
      admm_iters = k + 1;
      log_iter(k, rho, v[0], v[1], v[4]);
      // squared forms of the tests (no per-thread square roots); eq. stop's second term is
      // formed once, when the result is written
      rs_num = v[2];
      rs_den = v[3];
      if (!(v[0] == v[0]) || !(v[2] == v[2])) { status = ST_NAN; break; }
      if (v[1] <= tol2_primal) {
        const int t = final_test();
        if (t < 0) return false;
        if (t == 1 || t == 3) {
          to_polish = t == 3;
          rho_out = rho;
          return true;
        }
        if (t == 2) {
          // U, V and the rank changed: the pipelined R_0 is stale
          if ((long long)v[4] > prm.time_limit_ns) { status = ST_TIMEOUT; break; }
          rho = rho_next;
          if (!local_prologue(rho, gamma, g3)) return false;
          continue;
        }
      }
      if ((long long)v[4] > prm.time_limit_ns) { status = ST_TIMEOUT; break; }
      rho = rho_next;
    }
    if (status == ST_OK) status = ST_MAXITER;
    rho_out = rho;
    return true;
  }

  // ----------------------------------------------------------------------------------
  // Phase II, row-local form with the direct subproblem solve (subsolver 1).  Section 1
  // allows direct methods for the subproblems; here each row block of eq. linU / linV is
  // inverted by Sherman-Morrison (local_r0_row with dout), so a subproblem costs no CG
  // iteration and no reduction: the pass that forms a subproblem's R_0 also forms its
  // solution delta.  Two passes per iteration:
  //   A: U^{k+1} = V^k + delta_U, -(C U^{k+1}), and delta_V from the V-step's R_0; barrier
  //   B: V^{k+1} = U^{k+1} + delta_V, the dual step, -(C V^{k+1}), and delta_U from the next
  //      U-step's R_0; one grid reduction of the test sums.
  // delta_U lives in A.Dl and delta_V in A.Pd, so no pass writes what its neighbours read.
  // -(C W) and the T shadows are kept and refreshed every 32 iterations as in phase2_local.
  // ----------------------------------------------------------------------------------
  __device__ bool phase2_local_direct(double rho, double& rho_out) {
    const double gamma = prm.gamma;
    const double tol2_primal = prm.tol * (1.0 + P.b_inf) * prm.tol * (1.0 + P.b_inf);
    const bool shadow = (const void*)A.Ut != (const void*)A.U;
    T* const dU = A.Dl;
    T* const dV = A.Pd;
    double g3[3];
    if (!local_prologue(rho, gamma, g3, dU)) return false;
    for (int k = admm_iters; k < prm.max_admm_iter; ++k) {
      const bool exact = (k + 1) % 32 == 0;
      // pass A: U-step finish and the V-step's solution
      for (int j = tm.id; j < n; j += tm.count) {
        const RowCon c = row_con_of(j);
        Frag<double> Wj, Xj, mCW, mCX, xd;
        Frag<T> Xt, x;
        frag_load(Wj, A.V, j, ld, tm);
        frag_load(mCW, A.CWn, j, ld, tm);
        frag_load(Xt, A.Vt, j, ld, tm);           // (the master itself in the FP64 form)
        frag_load(x, dU, j, ld, tm);
        frag_convert(xd, x);
        Xj = Wj;
        frag_axpy(Xj, 1.0, xd);
        frag_axpy(Xt, T(1), x);                   // shadow of U^{k+1} = shadow(V^k) + delta
        if (exact) frag_convert(Xt, Xj);          // re-rounded from the master every 32
        local_mcx_row(j, A.V, dU, true, exact, mCW, mCX);
        frag_store(Xj, A.U, j, ld, tm);
        if (shadow) frag_store(Xt, A.Ut, j, ld, tm);
        frag_store(mCX, A.CWn, j, ld, tm);
        const double qU = local_r0_row(j, Xj, Xt, mCX, c, c.lam, rho, gamma, g3, dV);
        if (c.i >= 0 && tm.lane == 0) A.e[c.i] = qU;  // a ||U_j^{k+1}||^2 for the output residual
      }
      if (!sc.sync()) return false;
      ++hess;
      // pass B: V-step finish, dual step, and the next U-step's solution
      const double rho_next =
          ((k + 1) % prm.rho_every == 0) ? fmin(rho * prm.rho_growth, prm.rho_max) : rho;
      double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int j = tm.id; j < n; j += tm.count) {
        const RowCon c = row_con_of(j);
        const double qU = c.i >= 0 ? A.e[c.i] : 0.0;   // a ||U_j^{k+1}||^2 from pass A
        Frag<double> Wj, Xj, mCW, mCX, xd;
        Frag<T> x, Wt, Vot;
        frag_load(Wj, A.U, j, ld, tm);
        frag_load(mCW, A.CWn, j, ld, tm);
        frag_load(Wt, A.Ut, j, ld, tm);           // (the masters themselves in the FP64 form)
        frag_load(Vot, A.Vt, j, ld, tm);
        frag_load(x, dV, j, ld, tm);
        frag_convert(xd, x);
        Xj = Wj;
        frag_axpy(Xj, 1.0, xd);
        // eq. stop's second term (reported only): ||V^{k+1} - V^k||, ||V^k|| from the shadows
        Frag<T> Xt = Wt, dVk = Wt;
        frag_axpy(Xt, T(1), x);                   // shadow of V^{k+1} = shadow(U^{k+1}) + delta
        frag_axpy(dVk, T(-1), Vot);
        frag_axpy(dVk, T(1), x);
        const double d2 = (double)frag_dot(dVk, dVk, tm), o2 = (double)frag_dot(Vot, Vot, tm);
        if (exact) frag_convert(Xt, Xj);          // re-rounded from the master every 32
        // dual step lambda_i += rho (a U_j.V_j - b_i)
        double e = 0.0, lam_new = 0.0;
        if (c.i >= 0) {
          e = c.a * frag_dot(Wj, Xj, tm) - c.b;
          lam_new = c.lam + rho * e;        // every lane of the team holds the same value
        }
        local_mcx_row(j, A.U, dV, true, exact, mCW, mCX);
        frag_store(Xj, A.V, j, ld, tm);
        if (shadow) frag_store(Xt, A.Vt, j, ld, tm);
        frag_store(mCX, A.CWn, j, ld, tm);
        const double qV = local_r0_row(j, Xj, Xt, mCX, c, lam_new, rho_next, gamma, g3, dU);
        // the output's row residual a ||(U_j + V_j)/2||^2 - b_i from a||U_j||^2 (pass A),
        // a U_j.V_j = e + b_i and a||V_j||^2
        double eh = 0.0;
        if (c.i >= 0) eh = 0.25 * (qU + 2.0 * (e + c.b) + qV) - c.b;
        if (tm.lane == 0) {
          if (c.i >= 0) A.lam[c.i] = lam_new;
          v[0] += e * e;
          v[1] += eh * eh;
          v[2] += d2;
          v[3] += o2;
        }
      }
      if (sc.is_leader()) v[4] = (double)(globaltimer_ns() - t_start);
      if (!sc.reduce(v, 5)) return false;
      ++hess;
      admm_iters = k + 1;
      log_iter(k, rho, v[0], v[1], v[4]);
      rs_num = v[2];
      rs_den = v[3];
      if (!(v[0] == v[0]) || !(v[2] == v[2])) { status = ST_NAN; break; }
      if (v[1] <= tol2_primal) {
        const int t = final_test();
        if (t < 0) return false;
        if (t == 1 || t == 3) {
          to_polish = t == 3;
          rho_out = rho;
          return true;
        }
        if (t == 2) {
          // U, V and the rank changed: the pipelined delta_U is stale
          if ((long long)v[4] > prm.time_limit_ns) { status = ST_TIMEOUT; break; }
          rho = rho_next;
          if (!local_prologue(rho, gamma, g3, dU)) return false;
          continue;
        }
      }
      if ((long long)v[4] > prm.time_limit_ns) { status = ST_TIMEOUT; break; }
      rho = rho_next;
    }
    if (status == ST_OK) status = ST_MAXITER;
    rho_out = rho;
    return true;
  }

  // ----------------------------------------------------------------------------------
  // Phase III (not in the paper): Newton's method for eq. prob:BM on the product of spheres.
  // When every row carries one diagonal constraint a U_j.U_j = b (b/a > 0), the feasible set
  // of eq. prob:BM is the product of the spheres ||U_j|| = rad_j = sqrt(b/a) (P.row_norm), the
  // projection onto it is a row scaling, and for U on it the multiplier minimising
  // ||(C + A^T lambda) U||_F is a_j lambda_i = -mu_j, mu_j = (C U)_j.U_j / ||U_j||^2.  Then
  //   Riemannian gradient  g_j = 2 ((C U)_j - mu_j U_j)            (= 2 ((C + A^T lambda) U)_j)
  //   Riemannian Hessian   (H Z)_j = 2 P_j((C Z)_j - mu_j Z_j),  P_j(W) = W - (W.U_j/||U_j||^2) U_j
  // (Absil, Mahony and Sepulchre 2008, Ch. 6), and r_D = ||g|| / (2 (1 + ||C||_F)); on the
  // manifold A(U U^T) = b holds and the gap with y = -lambda(U) is zero.  The method is the
  // Riemannian trust-region Newton method (ibid., Algorithm 10), which reaches second-order
  // critical points: each step minimises the model g.d + d.H d / 2 over ||d|| <= Delta by
  // truncated CG (Steihaug-Toint, ibid. Algorithm 11: stop at ||H d + g|| <= eta ||g||,
  // eta = min(0.5, sqrt(||g||)), or on the boundary along a direction of non-positive curvature
  // or one that leaves the region), run as the Chronopoulos-Gear recurrence (one reduction and one
  // barrier per iteration: the Hessian reads the neighbours' residual); the step R(U + d), R the
  // row scaling, is taken when rho = (f(U) - f(R(U + d))) / (model decrease) > 0.1; Delta shrinks
  // by 4 when rho < 1/4 and doubles (up to ||U||_F) when rho > 3/4 on the boundary, from
  // ||U||_F / 8.  Once r_D <= tol the dual measure is tested (Lanczos); a failure escapes along
  // the eigenvector of lambda_min (escape_grow).
  // The gradient, the multipliers, the line search and the retraction are FP64; the CG of a
  // Newton step runs in the form's element type T (FP32 in the mixed form: the step is an
  // inexact solve to a relative residual of at least sqrt(||g||), far above FP32 rounding).
  // Arrays: U (iterate, FP64; Ut its T shadow), V (trial), grad (g), e (mu, by row), and in T the
  // CG's R (residual), Pd (direction), Sv (H p), HP (H r) and Dl (the Newton direction d).
  // ----------------------------------------------------------------------------------
  // (H Z)_j for the tangent field Z (neighbours' rows of Z must be visible); Zj is row j of Z,
  // Uj row j of the iterate; in T (the CG of a Newton step runs in the form's element type)
  __device__ __forceinline__ void sphere_hess_row(int j, const T* Z, const Frag<T>& Zj,
                                                  const Frag<T>& Uj, T u2, T mu,
                                                  Frag<T>& out) const {
    Frag<T> mCZ;
    spmm_row<T>(P, Z, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, T(0), tm, mCZ);
    // W = (C Z)_j - mu Z_j
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
#pragma unroll
      for (int e = 0; e < CHUNK; ++e) out.v[k][e] = -mCZ.v[k][e] - mu * Zj.v[k][e];
    const T c = frag_dot(out, Uj, tm) / u2;
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
#pragma unroll
      for (int e = 0; e < CHUNK; ++e) out.v[k][e] = T(2) * (out.v[k][e] - c * Uj.v[k][e]);
  }

  // g, mu, lambda(U) and C U at the iterate in A.U; v = (||g||^2, <C, U U^T>, ||U||_F^2, time)
  __device__ bool sphere_gradient(double* v) {
    v[0] = v[1] = v[2] = v[3] = 0.0;
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> Uj, mCU, g;
      frag_load(Uj, A.U, j, ld, tm);
      spmm_row<double>(P, A.U, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, 0.0, tm, mCU);
      const double u2 = frag_dot(Uj, Uj, tm);
      const double cu = -frag_dot(mCU, Uj, tm);
      const double mu = cu / u2;
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) g.v[k][e] = 2.0 * (-mCU.v[k][e] - mu * Uj.v[k][e]);
      frag_store(g, A.grad, j, ld, tm);
      const double g2 = frag_dot(g, g, tm);
      if (tm.lane == 0) {
        A.e[j] = mu;
        const int ci = P.row_con[j];
        A.lam[ci] = -mu / P.row_a[j];
        v[0] += g2;
        v[1] += cu;
        v[2] += u2;
      }
    }
    if (sc.is_leader()) v[3] = (double)(globaltimer_ns() - t_start);
    return sc.reduce(v, 4);
  }

  // One pass of the truncated CG for row j: with the scalars (a, b) of the step, p = r + b p,
  // s = w + b s, d += a p, r' = r - a s (the Chronopoulos-Gear recurrence), and with want_h also
  // w' = Hess r' and the row's shares of r'.r' and w'.r'.  Hess r' needs the neighbours' r',
  // which the pass recomputes from their r, w and s of the previous step (the same operations
  // as the rows' owners, so the same values): r, w and s are double-buffered (read from the
  // *c buffers, written to the *n ones) and one barrier per CG step remains, the reduction.
  __device__ __forceinline__ void sphere_tcg_row(int j, const T* Rc, const T* Wc, const T* Sc,
                                                 T* Rn, T* Wn, T* Sn, T a_t, T b_t, bool have_ps,
                                                 bool want_h, double* z) {
    Frag<T> r, w, pd, ss, x;
    frag_load(r, Rc, j, ld, tm);
    frag_load(w, Wc, j, ld, tm);
    if (have_ps) {
      frag_load(pd, A.Pd, j, ld, tm);
      frag_load(ss, Sc, j, ld, tm);
      frag_load(x, A.Dl, j, ld, tm);
    } else {
      frag_zero(pd);
      frag_zero(ss);
      frag_zero(x);
    }
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
#pragma unroll
      for (int e = 0; e < CHUNK; ++e) {
        pd.v[k][e] = fma(b_t, pd.v[k][e], r.v[k][e]);
        ss.v[k][e] = fma(b_t, ss.v[k][e], w.v[k][e]);
        x.v[k][e] = fma(a_t, pd.v[k][e], x.v[k][e]);
        r.v[k][e] = fma(-a_t, ss.v[k][e], r.v[k][e]);
      }
    frag_store(pd, A.Pd, j, ld, tm);
    frag_store(ss, Sn, j, ld, tm);
    frag_store(x, A.Dl, j, ld, tm);
    frag_store(r, Rn, j, ld, tm);
    if (!want_h) return;
    // (C r')_j with the neighbours' r' = r - a (w + b s) formed from the previous step's rows
    Frag<T> acc;
    frag_zero(acc);
    const T* cv = cval<T>(P);
    for (int q = P.C_rp[j]; q < P.C_rp[j + 1]; ++q) {
      const int k = P.C_col[q];
      const T c = cv[q];
      if (k == j) {
        frag_axpy(acc, c, r);
        continue;
      }
      Frag<T> rk, wk, sk;
      frag_load(rk, Rc, k, ld, tm);
      frag_load(wk, Wc, k, ld, tm);
      if (have_ps) frag_load(sk, Sc, k, ld, tm);
      else frag_zero(sk);
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) {
          const T sv = fma(b_t, sk.v[kk][e], wk.v[kk][e]);
          acc.v[kk][e] = fma(c, fma(-a_t, sv, rk.v[kk][e]), acc.v[kk][e]);
        }
    }
    // w' = 2 P_U((C r')_j - mu_j r'_j)
    Frag<T> Uj;
    frag_load(Uj, A.Ut, j, ld, tm);
    const T u2 = frag_dot(Uj, Uj, tm);
    const T mu = (T)A.e[j];
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
#pragma unroll
      for (int e = 0; e < CHUNK; ++e) acc.v[k][e] = acc.v[k][e] - mu * r.v[k][e];
    const T cp = frag_dot(acc, Uj, tm) / u2;
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
#pragma unroll
      for (int e = 0; e < CHUNK; ++e) acc.v[k][e] = T(2) * (acc.v[k][e] - cp * Uj.v[k][e]);
    frag_store(acc, Wn, j, ld, tm);
    const double d1 = (double)frag_dot(r, r, tm), d2 = (double)frag_dot(acc, r, tm);
    if (tm.lane == 0) {
      z[0] += d1;
      z[1] += d2;
    }
  }

  // Steihaug-Toint truncated CG (Absil, Mahony and Sepulchre 2008, Algorithm 11) for the
  // trust-region model at U with gradient g (A.grad, ||g||^2 = g2) and radius delta, as the
  // single-reduction Chronopoulos-Gear recurrence (the iterates of textbook CG in exact
  // arithmetic): stops at ||r|| <= min(0.5, sqrt ||g||) ||g||, where p.Hp <= 0 (to the boundary
  // along p) or where the next iterate would leave the region (to the boundary).  Thread 0 of
  // each CTA evaluates the scalar recurrence, including ||d||^2, d.p and ||p||^2 for the
  // boundary tests.  The vectors are in T (the mixed form runs this CG in FP32; the gradient,
  // the model test and the retraction stay FP64) at the iterate's T shadow A.Ut.  d ends in
  // A.Dl; it = CG steps (Hessian products after the first).
  __device__ bool sphere_tcg(double g2, double delta, int& it, bool& on_boundary) {
    // double-buffered r, w, s (free in Phase III: the FP64 scratch of Phase I / II viewed as T)
    T* Rb[2] = {A.R, reinterpret_cast<T*>(A.CWn)};
    T* Wb[2] = {A.HP, reinterpret_cast<T*>(A.grad_old)};
    T* Sb[2] = {A.Sv, reinterpret_cast<T*>(A.dir)};
    const T* const Us = A.Ut;
    // r_0 = -g, w_0 = H r_0
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> gj;
      Frag<T> r;
      frag_load(gj, A.grad, j, ld, tm);
      frag_convert(r, gj);
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) r.v[k][e] = -r.v[k][e];
      frag_store(r, Rb[0], j, ld, tm);
    }
    if (!sc.sync()) return false;
    double g3[2] = {0.0, 0.0};
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<T> Uj, r, w;
      frag_load(Uj, Us, j, ld, tm);
      frag_load(r, Rb[0], j, ld, tm);
      const T u2 = frag_dot(Uj, Uj, tm);
      sphere_hess_row(j, Rb[0], r, Uj, u2, (T)A.e[j], w);
      frag_store(w, Wb[0], j, ld, tm);
      const double d1 = (double)frag_dot(r, r, tm), d2 = (double)frag_dot(w, r, tm);
      if (tm.lane == 0) {
        g3[0] += d1;
        g3[1] += d2;
      }
    }
    if (!sc.reduce(g3, 2)) return false;
    const bool lead = threadIdx.x == 0;
    double* shs = sc.scratch() + 4;     // state (0 go on, 1 stop, 2 NaN, 3 last step), a, b
    const double eta = fmin(0.5, sqrt(sqrt(g2)));
    const double target2 = eta * eta * g2;
    const double dl2 = delta * delta;
    // thread 0: gam = r.r, ga = gam * alpha, a_prev = alpha, pp = ||p||^2, dp = d.p,
    // dd = ||d||^2 (of the direction / iterate the next pass forms)
    double gam = 0.0, ga = 0.0, a_prev = 0.0, pp = 0.0, dp = 0.0, dd = 0.0;
    if (lead) {
      gam = g3[0];
      const double del = g3[1];
      pp = gam;
      int state = 0;
      double alpha = 0.0;
      if (!(gam == gam) || !(del == del)) {
        state = 2;
      } else if (gam <= target2) {
        state = 1;
      } else if (!(del > 0.0) || gam * (gam / del) * (gam / del) >= dl2) {
        alpha = delta / sqrt(gam);       // to the boundary along p_0 = -g
        state = 3;
      } else {
        alpha = gam / del;
      }
      ga = gam * alpha;
      a_prev = alpha;
      shs[0] = (double)state;
      shs[1] = alpha;
      shs[2] = 0.0;
    }
    __syncthreads();
    int state = (int)shs[0];
    T a_t = (T)shs[1], b_t = T(0);
    __syncthreads();
    if (state == 2) status = ST_NAN;
    it = 0;
    on_boundary = state == 3;
    bool wrote = false;
    int cur = 0;
    // FP64: recomputing the neighbours' r' costs two DFMAs per element and neighbour (FP64 issues
    // at 1/64 of FP32 here), more than the barrier it saves; that form takes a second pass
    constexpr bool fuse = sizeof(T) == 4;
    while ((state == 0 || state == 3) && it < prm.newton_cg_max) {
      const bool want_h = state == 0;
      double z[2] = {0.0, 0.0};
      for (int j = tm.id; j < n; j += tm.count)
        sphere_tcg_row(j, Rb[cur], Wb[cur], Sb[cur], Rb[cur ^ 1], Wb[cur ^ 1], Sb[cur ^ 1], a_t,
                       b_t, wrote, want_h && fuse, z);
      wrote = true;
      cur ^= 1;
      if (!want_h) break;                // the boundary step: d is final
      if (!fuse) {
        if (!sc.sync()) return false;
        for (int j = tm.id; j < n; j += tm.count) {
          Frag<T> Uj, r, w;
          frag_load(Uj, Us, j, ld, tm);
          frag_load(r, Rb[cur], j, ld, tm);
          const T u2 = frag_dot(Uj, Uj, tm);
          sphere_hess_row(j, Rb[cur], r, Uj, u2, (T)A.e[j], w);
          frag_store(w, Wb[cur], j, ld, tm);
          const double d1 = (double)frag_dot(r, r, tm), d2 = (double)frag_dot(w, r, tm);
          if (tm.lane == 0) {
            z[0] += d1;
            z[1] += d2;
          }
        }
      }
      if (!sc.reduce(z, 2)) return false;
      ++it;
      if (lead) {
        // the pass just made: d += alpha p (the alpha of the previous step), so d.p and ||d||^2
        // move on
        const double alpha_prev = a_prev;
        dd += 2.0 * alpha_prev * dp + alpha_prev * alpha_prev * pp;
        dp += alpha_prev * pp;           // d_k+1 . p_k
        const double gam_new = z[0], del_new = z[1];
        int st = 0;
        double alpha = 0.0, beta = 0.0;
        if (!(gam_new == gam_new) || !(del_new == del_new)) {
          st = 2;
        } else if (gam_new <= target2) {
          st = 1;
        } else {
          // with D = del_new ga - gam_new^2 (p.Hp = D / ga), beta = gam_new / gam and
          // alpha = gam_new ga / D both come from the one reciprocal 1 / (gam D) when D > 0
          const double D = del_new * ga - gam_new * gam_new;
          bool to_boundary = !(D > 0.0);
          if (!to_boundary) {
            const double inv = 1.0 / (gam * D);
            beta = gam_new * D * inv;
            alpha = gam_new * ga * gam * inv;
          } else {
            beta = gam_new / gam;
          }
          pp = gam_new + beta * beta * pp;          // ||p_k+1||^2
          dp = beta * dp;                           // d_k+1 . p_k+1
          if (!to_boundary)
            to_boundary = dd + 2.0 * alpha * dp + alpha * alpha * pp >= dl2;
          if (to_boundary) {
            const double qa = pp, qb = 2.0 * dp, qc = dd - dl2;
            alpha = (-qb + sqrt(fmax(qb * qb - 4.0 * qa * qc, 0.0))) / (2.0 * qa);
            st = 3;
          }
          ga = gam_new * alpha;
          gam = gam_new;
          a_prev = alpha;
        }
        shs[0] = (double)st;
        shs[1] = alpha;
        shs[2] = beta;
      }
      __syncthreads();
      state = (int)shs[0];
      a_t = (T)shs[1];
      b_t = (T)shs[2];
      __syncthreads();
      if (state == 2) status = ST_NAN;
      if (state == 3) on_boundary = true;
    }
    if (!wrote) {
      // no step taken (the gradient already small, or a NaN): d = 0
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<T> x;
        frag_zero(x);
        frag_store(x, A.Dl, j, ld, tm);
      }
    }
    return sc.sync();
  }

  // the model's decrease -(g.d + d.H d / 2) for the d in A.Dl (neighbours' d visible)
  __device__ bool sphere_model_decrease(double& pred) {
    double v[2] = {0.0, 0.0};
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<T> Uj, dj, w;
      Frag<double> gj, dd;
      frag_load(Uj, A.Ut, j, ld, tm);
      frag_load(dj, A.Dl, j, ld, tm);
      const T u2 = frag_dot(Uj, Uj, tm);
      sphere_hess_row(j, A.Dl, dj, Uj, u2, (T)A.e[j], w);
      frag_load(gj, A.grad, j, ld, tm);
      frag_convert(dd, dj);
      const double a1 = frag_dot(gj, dd, tm), a2 = (double)frag_dot(dj, w, tm);
      if (tm.lane == 0) {
        v[0] += a1;
        v[1] += a2;
      }
    }
    if (!sc.reduce(v, 2)) return false;
    pred = -(v[0] + 0.5 * v[1]);
    return true;
  }

  // trial point R(U + t d) into A.V (row scaling onto the spheres); with want_slope also g.d
  __device__ bool sphere_trial(double t, bool want_slope, double& slope) {
    double v[1] = {0.0};
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> Uj, dj;
      Frag<T> dt;
      frag_load(Uj, A.U, j, ld, tm);
      frag_load(dt, A.Dl, j, ld, tm);
      frag_convert(dj, dt);
      if (want_slope) {
        Frag<double> gj;
        frag_load(gj, A.grad, j, ld, tm);
        const double gd = frag_dot(gj, dj, tm);
        if (tm.lane == 0) v[0] += gd;
      }
      frag_axpy(Uj, t, dj);
      const double sc2 = P.row_norm[j] / sqrt(frag_dot(Uj, Uj, tm));
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) Uj.v[k][e] *= sc2;
      frag_store(Uj, A.V, j, ld, tm);
    }
    if (!sc.reduce(v, 1)) return false;
    if (want_slope) slope = v[0];
    return true;
  }

  // <C, W W^T> for W = A.V (neighbours visible)
  __device__ bool trial_objective(double& f) {
    double v[1] = {0.0};
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> Wj, mCW;
      frag_load(Wj, A.V, j, ld, tm);
      spmm_row<double>(P, A.V, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, 0.0, tm, mCW);
      const double o = -frag_dot(Wj, mCW, tm);
      if (tm.lane == 0) v[0] += o;
    }
    if (!sc.reduce(v, 1)) return false;
    f = v[0];
    return true;
  }

  // copies src into dst (both n x ld FP64), and into the T shadow tdst unless it aliases the
  // masters (nullptr: none), then a barrier
  __device__ bool copy_rows(const double* src, double* dst, T* tdst = nullptr) {
    const bool sh = tdst != nullptr && (const void*)tdst != (const void*)A.U &&
                    (const void*)tdst != (const void*)A.V;
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> x;
      frag_load(x, src, j, ld, tm);
      frag_store(x, dst, j, ld, tm);
      if (sh) {
        Frag<T> t;
        frag_convert(t, x);
        frag_store(t, tdst, j, ld, tm);
      }
    }
    return sc.sync();
  }

  // U <- rows of U scaled onto the spheres (at the start, after a rank growth), V = U, and the
  // T shadow of U
  __device__ bool sphere_retract_u() {
    const bool sh = (const void*)A.Ut != (const void*)A.U;
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> Uj;
      frag_load(Uj, A.U, j, ld, tm);
      const double sc2 = P.row_norm[j] / sqrt(frag_dot(Uj, Uj, tm));
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) Uj.v[k][e] *= sc2;
      frag_store(Uj, A.U, j, ld, tm);
      frag_store(Uj, A.V, j, ld, tm);
      if (sh) {
        Frag<T> t;
        frag_convert(t, Uj);
        frag_store(t, A.Ut, j, ld, tm);
      }
    }
    return sc.sync();
  }

  __device__ bool phase3() {
    t_p3 = globaltimer_ns();
    // start: U = R(U_hat), U_hat = (U + V)/2 of Phase II's output
    if (!form_u_hat()) return false;
    if (!copy_rows(A.tmp, A.U)) return false;
    if (!sphere_retract_u()) return false;
    const double tol_g2 = 4.0 * prm.tol * (1.0 + P.C_fro) * prm.tol * (1.0 + P.C_fro);
    double delta_max = -1.0, delta = 0.0;
    for (;;) {
      double v[4];
      if (!sphere_gradient(v)) return false;
      const double g2 = v[0], f0 = v[1];
      if (!(g2 == g2) || !(f0 == f0)) { status = ST_NAN; return true; }
      if (delta_max < 0.0) {
        delta_max = sqrt(v[2]);          // ||U||_F
        delta = delta_max / 8.0;
      }
      if (g2 <= tol_g2) {
        if (!prm.kkt_dinf) return true;
        if (!lanczos_lambda_min(last_lmin)) return false;
        lmin_at = admm_iters;
        if (dual_psd(last_lmin) <= prm.tol) return true;
        if (!escape_possible()) { status = ST_MAXITER; return true; }
        uh_norm2 = v[2];
        if (!copy_rows(A.U, A.V)) return false;
        if (!escape_grow()) return false;
        if (!sphere_retract_u()) return false;
        continue;
      }
      if ((long long)v[3] > prm.time_limit_ns) { status = ST_TIMEOUT; return true; }
      if (newton_steps >= prm.newton_max) { status = ST_MAXITER; return true; }
      int it = 0;
      bool on_boundary = false;
      if (!sphere_tcg(g2, delta, it, on_boundary)) return false;
      if (status != ST_OK) return true;
      double pred = 0.0, slope = 0.0, f = 0.0;
      if (!sphere_model_decrease(pred)) return false;
      newton_cg += it + 2;                 // the CG's Hessian products, its first, the model's
      if (!sphere_trial(1.0, false, slope)) return false;
      if (!trial_objective(f)) return false;
      const double ratio = pred > 0.0 ? (f0 - f) / pred : -1.0;
      if (ratio < 0.25) delta *= 0.25;
      else if (ratio > 0.75 && on_boundary) delta = fmin(2.0 * delta, delta_max);
      if (ratio > 0.1) {
        if (!copy_rows(A.V, A.U, A.Ut)) return false;
      }
      ++newton_steps;
    }
  }

  // ||U||_F^2 of the masters
  __device__ bool u_norm2(double& u2) {
    double v[1] = {0.0};
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> Uj;
      frag_load(Uj, A.U, j, ld, tm);
      const double d = frag_dot(Uj, Uj, tm);
      if (tm.lane == 0) v[0] += d;
    }
    if (!sc.reduce(v, 1)) return false;
    u2 = v[0];
    return true;
  }

  // Phase III outside the product-of-spheres class: the augmented Lagrangian method of Phase I
  // continued from Phase II's output (U = U_hat, lambda, sigma = Phase I's last penalty) until
  // r_P <= tol, r_D <= tol and the dual measure <= tol, in chunks of REFINE_CHUNK outer
  // iterations with the dual measure taken after each.  Above tol after a chunk that
  // converged, or after one that did not but left it less than 10% below the previous chunk's,
  // the rank is too small: the escape (tau z into a zero column or a grown rank) follows.  At
  // most max_outer outer iterations in all; V = U at the end.
  __device__ bool phase3_alm(double sigma) {
    t_p3 = globaltimer_ns();
    if (!form_u_hat()) return false;
    if (!copy_rows(A.tmp, A.U)) return false;
    int outer = 0;
    double prev = -1.0;
    bool converged = false;
    while (outer < prm.max_outer) {
      const int before = refine_outer;
      if (!alm(sigma, true, min(REFINE_CHUNK, prm.max_outer - outer))) return false;
      if (status != ST_OK) break;
      outer += refine_outer - before;
      if (!prm.kkt_dinf) {
        if (alm_done) { converged = true; break; }
        continue;
      }
      if (!lanczos_lambda_min(last_lmin)) return false;
      lmin_at = admm_iters;
      const double d = dual_psd(last_lmin);
      if (alm_done && d <= prm.tol) { converged = true; break; }
      if (d <= prm.tol || (!alm_done && (prev < 0.0 || d < 0.9 * prev))) {
        prev = d;
        continue;
      }
      if (!escape_possible()) break;
      if (!u_norm2(uh_norm2)) return false;
      if (!copy_rows(A.U, A.V)) return false;
      if (!escape_grow()) return false;
      prev = -1.0;
    }
    if (status == ST_OK && !converged) status = ST_MAXITER;
    return copy_rows(A.U, A.V);
  }

  // U_hat = (U + V)/2 into tmp
  __device__ bool form_u_hat() {
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> u, w;
      frag_load(u, A.U, j, ld, tm);
      frag_load(w, A.V, j, ld, tm);
      frag_axpy(u, 1.0, w);
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) u.v[k][e] *= 0.5;
      frag_store(u, A.tmp, j, ld, tm);
    }
    return sc.sync();
  }

  // Appendix B primal-dual gap of X = U_hat U_hat^T, y = -lambda:
  // (<C, X> - b^T y) / (1 + |<C, X>| + |b^T y|), in FP64 from the masters
  // Appendix B primal-dual gap of X = U_hat U_hat^T, y = -lambda:
  // (<C, X> - b^T y) / (1 + |<C, X>| + |b^T y|), in FP64 from the masters; in the same pass
  // last_rd2 = ||(C + A^T lambda) U_hat||_F^2 (eq. def:eKKT's stationarity with y = -lambda)
  __device__ bool gap_check(double& gap) {
    if (!form_u_hat()) return false;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (P.a_diag_only) {
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<double> Uh, mCU;
        frag_load(Uh, A.tmp, j, ld, tm);
        spmm_row<double>(P, A.tmp, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, 0.0, tm, mCU);
        const double o = -frag_dot(Uh, mCU, tm), u2 = frag_dot(Uh, Uh, tm);
        // -(C + A^T lambda) U_hat on row j: -(C U_hat)_j - a lambda_i U_hat_j
        const int ci = P.row_con[j];
        if (ci >= 0) frag_axpy(mCU, -P.row_a[j] * A.lam[ci], Uh);
        const double s2 = frag_dot(mCU, mCU, tm);
        if (tm.lane == 0) {
          v[0] += o;
          v[2] += u2;
          v[3] += s2;
        }
      }
    } else {
      const WarpRow wr = make_warp_row(ld, sc.tid(), sc.nthreads(), prm.team_mult);
      for (int j = wr.warp; j < n; j += wr.nwarps) {
        Frag<double> Uh, mCU, mSU;
        frag_load(Uh, A.tmp, j, ld, wr.st);
        spmm_row_warp<double>(P, A.tmp, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, 0.0, wr, mCU);
        spmm_row_warp<double>(P, A.tmp, ld, j, A.lam, nullptr, 0.0, -1.0, 0.0, 0.0, wr, mSU);
        if (wr.sub == 0) {
          const double o = -frag_dot(Uh, mCU, wr.st), u2 = frag_dot(Uh, Uh, wr.st);
          const double s2 = frag_dot(mSU, mSU, wr.st);
          if (wr.st.lane == 0) {
            v[0] += o;
            v[2] += u2;
            v[3] += s2;
          }
        }
      }
    }
    for (int i = sc.tid(); i < m; i += sc.nthreads()) v[1] += P.b[i] * A.lam[i];
    if (!sc.reduce(v, 4)) return false;
    uh_norm2 = v[2];
    last_rd2 = v[3];
    const double pobj = v[0], dobj = -v[1];
    gap = (pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
    return true;
  }

  // Largest eigenvalue of each Lanczos tridiagonal T_c (alpha at hist[8k + c], beta at
  // hist[8k + 4 + c], L[c] steps) by Sturm counts: the LDL^T pivots of T_c - x I,
  //   d_0 = alpha_0 - x,   d_i = (alpha_i - x) - beta_{i-1}^2 / d_{i-1},
  // have as many negative entries as T_c has eigenvalues below x.  The multisection spreads its
  // points over the whole scope: in each round lane l of warp c in the CTA of rank q takes point
  // g = 32 q + l of Np = 32 (CTAs in the scope) evenly spaced interior points of chain c's
  // bracket, one reduction counts the points at or below the top eigenvalue, and the bracket
  // shrinks to the two points around it (a factor Np + 1; the first bracket is Gershgorin's).
  // Rounds continue until the factors reach 2^46 (4 rounds over 152 CTAs, 10 in one CTA).
  // Every CTA takes the same sums and so the same brackets.  The pivot's reciprocal is the
  // FP32 reciprocal refined by one Newton step in FP64, r <- r + r (1 - d r), relative error
  // about 2^-48: the count is then that of T_c with its beta^2 perturbed by as much.  Pivots
  // below 1e-30 in magnitude become -1e-30 (a shift of x by at most that, and inside the range
  // of the FP32 seed).  best is the largest over the columns (-inf when none has a step), cs
  // its column.  Called by every thread of the scope.
  __device__ bool ritz_top(const double* hist, const int* L, double& best, int& cs) {
    constexpr int NC = 4;
    double* sh = sc.scratch();     // 2 NC entries: the Gershgorin brackets
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < NC) {
      const int c = warp, Lc = L[c];
      double lo = INFINITY, hi = -INFINITY;
      for (int i = lane; i < Lc; i += 32) {
        const double ai = hist[8 * i + c];
        const double bl = i > 0 ? fabs(hist[8 * (i - 1) + 4 + c]) : 0.0;
        const double br = i + 1 < Lc ? fabs(hist[8 * i + 4 + c]) : 0.0;
        lo = fmin(lo, ai - bl - br);
        hi = fmax(hi, ai + bl + br);
      }
      for (int off = 16; off > 0; off >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, off));
      }
      if (lane == 0) {
        sh[c] = lo;
        sh[NC + c] = hi;
      }
    }
    __syncthreads();
    double lo[NC], hi[NC];
    int Ls[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      lo[c] = sh[c];
      hi[c] = sh[NC + c];
      Ls[c] = L[c];
    }
    __syncthreads();
    const int Np = 32 * (sc.nthreads() / (int)blockDim.x);
    const double span = (double)(Np + 1);
    int rounds = 0;
    for (double f = 1.0; f < 70368744177664.0; f *= span) ++rounds;     // 2^46
    const int g = 32 * (sc.tid() / (int)blockDim.x) + lane;
    for (int round = 0; round < rounds; ++round) {
      double v[NC] = {0.0, 0.0, 0.0, 0.0};
      if (warp < NC) {
        double clo = lo[0], chi = hi[0];
        int Lc = Ls[0];
#pragma unroll
        for (int c = 1; c < NC; ++c)
          if (c == warp) {
            clo = lo[c];
            chi = hi[c];
            Lc = Ls[c];
          }
        if (Lc > 0) {
          const double x = clo + (chi - clo) * (double)(g + 1) / span;
          const int c = warp;
          int below = 0;
          double d = 1.0;
          for (int i = 0; i < Lc; ++i) {
            const double ai = hist[8 * i + c];
            if (i == 0) {
              d = ai - x;
            } else {
              const double bi = hist[8 * (i - 1) + 4 + c];
              double r = (double)__frcp_rn((float)d);
              r = fma(r, fma(-d, r, 1.0), r);
              d = (ai - x) - (bi * bi) * r;
            }
            if (fabs(d) < 1e-30) d = -1e-30;
            below += d < 0.0;
          }
#pragma unroll
          for (int k = 0; k < NC; ++k) v[k] = (k == warp && below < Lc) ? 1.0 : 0.0;
        }
      }
      if (!sc.reduce(v, NC)) return false;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (Ls[c] <= 0) continue;
        const int F = (int)v[c];      // points at or below the top eigenvalue
        const double w = hi[c] - lo[c];
        const double nlo = F == 0 ? lo[c] : lo[c] + w * (double)F / span;
        const double nhi = F >= Np ? hi[c] : lo[c] + w * (double)(F + 1) / span;
        lo[c] = nlo;
        hi[c] = nhi;
      }
    }
    best = -INFINITY;
    cs = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double th = Ls[c] > 0 ? 0.5 * (lo[c] + hi[c]) : -INFINITY;
      if (th > best) {
        best = th;
        cs = c;
      }
    }
    return true;
  }

  // lambda_min(C - A^T y), y = -lambda: Lanczos on M = -(C + A^T(lambda)) from four random
  // start columns at once (an n x 4 block in the factor layout of width 4), at most Kmax =
  // min(lanczos_steps, 2048, n) steps each (fewer once the estimate settles, see below), no
  // reorthogonalisation; the estimate is -max_c theta_c, theta_c the largest eigenvalue of
  // column c's tridiagonal (Sturm-count multisection).  A clustered bottom of the spectrum
  // (the dual slack of a degenerate SDP) needs many steps: on the 141 x 141 torus the estimate
  // moves from +6e-5 (128 steps) to -3.6e-6 (2048).  Column c stops early when its beta
  // vanishes (its Krylov space is exhausted).
  // With want_vec the Ritz vector of the estimate is rebuilt too: the eigenvector s of the
  // chosen T_c by inverse iteration, then z = sum_k s_k q_k into A.Y + 2 Kmax (n entries),
  // from the blocks kept in A.lz_store when the state has room for them, else by a second
  // pass of the same recurrence (the stored alpha / beta, the same start); zn2 receives
  // ||z||^2.
  __device__ bool lanczos_lambda_min(double& lmin) {
    const long long t0 = globaltimer_ns();
    const bool ok = lanczos_run(lmin);
    lz_ns += globaltimer_ns() - t0;
    return ok;
  }

  // the Ritz vector of the last lanczos_lambda_min into A.Y + 2 Kmax (squared norm zn2)
  __device__ bool lanczos_ritz_vector(double& zn2) {
    const long long t0 = globaltimer_ns();
    const bool ok = lanczos_vector(zn2);
    lz_ns += globaltimer_ns() - t0;
    return ok;
  }

  __device__ __noinline__ bool lanczos_run(double& lmin) {
    constexpr int NC = 4;
    const int Kmax = min(min(prm.lanczos_steps, LANCZOS_MAX), n);
    if (Kmax <= 0) {
      lmin = NAN;
      return true;
    }
    // steps taken: Kmax, or fewer once the estimate settles (checked at 128, 256, 512, ...
    // steps: the largest Ritz value of M grows with the step count, and the recurrence stops
    // when it rose by at most 0.05 tol (1 + ||C||_inf) over the last doubling), or once it
    // proves the dual test failed: a Ritz value of M never exceeds lambda_max(M), so an
    // estimate of lambda_min(C - A^T y) that already fails the test fails it for the true value
    int K = Kmax;
    int next_check = min(128, Kmax);
    double theta_prev = -INFINITY;
    const double settle = 0.05 * prm.tol * (1.0 + P.C_inf);
    double* Qp = A.dir;     // raw q_{k-1} (true vector: qps * Qp)
    double* Q = A.grad;     // raw q_k     (true vector: qs * Q)
    double* W = A.grad_old;
    double* const store = A.lz_store;     // raw q_k in slot k, when kept
    const long long slot = (long long)n * NC;
    if (store) {
      Q = store;
      W = store + slot;
    }
    double* hist = A.S;     // alpha_k[c] at hist[8k + c], beta_k[c] at hist[8k + 4 + c]
    const Team t4 = make_team(NC, sc.tid(), sc.nthreads(), 1);     // one thread per row
    const WarpRow w4 = make_warp_row(NC, sc.tid(), sc.nthreads(), 1);
    const uint64_t key = stream_key(prm.seed, 4000);
    double v[NC] = {0.0, 0.0, 0.0, 0.0};
    for (int j = sc.tid(); j < n; j += sc.nthreads())
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double x = normal_at(key, (uint64_t)j * NC + c);
        Q[(long long)j * NC + c] = x;
        Qp[(long long)j * NC + c] = 0.0;
        v[c] += x * x;
      }
    if (!sc.reduce(v, NC)) return false;
    double qs[NC], qps[NC], bp[NC], qs0[NC];
    int len[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      qs[c] = v[c] > 0.0 ? 1.0 / sqrt(v[c]) : 0.0;
      qs0[c] = qs[c];
      qps[c] = 0.0;
      bp[c] = 0.0;
      len[c] = v[c] > 0.0 ? K : 0;
    }
    for (int k = 0; k < Kmax; ++k) {
      ++lz_steps;
      // W = M q_k - beta_{k-1} q_{k-1};  alpha_k = q_k . W
      double a[NC] = {0.0, 0.0, 0.0, 0.0};
      const bool diag = P.a_diag_only != 0;
      const int j0 = diag ? t4.id : w4.warp, js = diag ? t4.count : w4.nwarps;
      for (int j = j0; j < n; j += js) {
        Frag<double> mq;
        if (diag) {
          spmm_row<double>(P, Q, NC, j, A.lam, nullptr, 0.0, -1.0, 0.0, 0.0, t4, mq);
        } else {
          spmm_row_warp<double>(P, Q, NC, j, A.lam, nullptr, 0.0, -1.0, 0.0, 0.0, w4, mq);
          if (w4.sub != 0) continue;
        }
        const long long o = (long long)j * NC;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const double w = qs[c] * mq.v[0][c] - bp[c] * qps[c] * Qp[o + c];
          W[o + c] = w;
          a[c] += qs[c] * Q[o + c] * w;
        }
      }
      if (!sc.reduce(a, NC)) return false;
      // W -= alpha_k q_k;  beta_k = ||W||
      double b2[NC] = {0.0, 0.0, 0.0, 0.0};
      for (int j = sc.tid(); j < n; j += sc.nthreads()) {
        const long long o = (long long)j * NC;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const double w = W[o + c] - a[c] * qs[c] * Q[o + c];
          W[o + c] = w;
          b2[c] += w * w;
        }
      }
      if (!sc.reduce(b2, NC)) return false;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double beta = sqrt(b2[c]);
        if (sc.is_leader()) {
          hist[8 * k + c] = a[c];
          hist[8 * k + 4 + c] = beta;
        }
        const bool live = len[c] > k + 1;
        const bool breakdown = !(beta > 1e-12 * (fabs(a[c]) + bp[c]) && beta > 1e-300);
        if (live && breakdown) len[c] = k + 1;
        qps[c] = qs[c];
        qs[c] = len[c] > k + 1 ? 1.0 / beta : 0.0;
        bp[c] = len[c] > k + 1 ? beta : 0.0;
      }
      double* t = Qp;
      Qp = Q;
      Q = W;
      W = store ? store + (long long)min(k + 2, Kmax) * slot : t;
      if (k + 1 == next_check && k + 1 < Kmax) {
        if (!sc.sync()) return false;   // the coefficients written by the leader
        double th;
        int cc;
        int lc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) lc[c] = min(len[c], k + 1);
        if (!ritz_top(hist, lc, th, cc)) return false;
        if (th - theta_prev <= settle || dual_psd(-th) > prm.tol) {
          K = k + 1;
          break;
        }
        theta_prev = th;
        next_check *= 2;
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) len[c] = min(len[c], K);
    if (!sc.sync()) return false;       // the coefficients written by the leader
    double best;
    int cs;
    if (!ritz_top(hist, len, best, cs)) return false;
    lmin = best > -INFINITY ? -best : NAN;
    // what the Ritz vector pass needs (the coefficients stay in hist)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      lz_len[c] = len[c];
      lz_qs0[c] = qs0[c];
    }
    lz_best = best;
    lz_cs = cs;
    return true;
  }

  // Second pass of the last first pass (same start, same recurrence with its stored
  // coefficients): the Ritz vector of its estimate.  Callers run it right after a failed dual
  // test, before anything else touches the Lanczos blocks or the multiplier.
  __device__ __noinline__ bool lanczos_vector(double& zn2_out) {
    constexpr int NC = 4;
    const int Kmax = min(min(prm.lanczos_steps, LANCZOS_MAX), n);
    double* hist = A.S;
    const Team t4 = make_team(NC, sc.tid(), sc.nthreads(), 1);     // one thread per row
    const WarpRow w4 = make_warp_row(NC, sc.tid(), sc.nthreads(), 1);
    const uint64_t key = stream_key(prm.seed, 4000);
    int len[NC];
    double qs[NC], qps[NC], bp[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) len[c] = lz_len[c];
    const double best = lz_best;
    const int cs = lz_cs;
    double* Qp;
    double* Q;
    double* W;
    double* zn2 = &zn2_out;
    // eigenvector of T_cs for theta by two steps of inverse iteration (Thomas elimination of
    // T_cs - theta I; pivots below 1e-300 are nudged), one thread
    const int L = len[cs];
    double* sv = A.Y;          // s (L entries)
    double* cp = A.Y + Kmax;   // elimination scratch
    double* zv = A.Y + 2 * Kmax;  // the Ritz vector (where escape_grow reads it)
    if (sc.is_leader() && L > 0) {
      for (int i = 0; i < L; ++i) sv[i] = 1.0;
      for (int it = 0; it < 2; ++it) {
        double piv = hist[c8(0, cs)] - best;
        if (fabs(piv) < 1e-300) piv = 1e-300;
        cp[0] = L > 1 ? hist[c8(0, cs) + 4] / piv : 0.0;
        sv[0] = sv[0] / piv;
        for (int i = 1; i < L; ++i) {
          const double bl = hist[c8(i - 1, cs) + 4];
          piv = (hist[c8(i, cs)] - best) - bl * cp[i - 1];
          if (fabs(piv) < 1e-300) piv = 1e-300;
          cp[i] = i + 1 < L ? hist[c8(i, cs) + 4] / piv : 0.0;
          sv[i] = (sv[i] - bl * sv[i - 1]) / piv;
        }
        for (int i = L - 2; i >= 0; --i) sv[i] -= cp[i] * sv[i + 1];
        double nrm = 0.0;
        for (int i = 0; i < L; ++i) nrm += sv[i] * sv[i];
        nrm = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
        for (int i = 0; i < L; ++i) sv[i] *= nrm;
      }
    }
    if (A.lz_store) {
      // z_j = sum_k (s_k qs_k) Q_k[j, cs], the raw blocks of the first pass and their scales
      // (qs_0 the start's, qs_k = 1 / beta_{k-1}), in the order the second pass adds them;
      // the leader folds the scales into s
      if (sc.is_leader())
        for (int k = 0; k < L; ++k)
          sv[k] = sv[k] * (k == 0 ? lz_qs0[cs] : 1.0 / hist[c8(k - 1, cs) + 4]);
      if (!sc.sync()) return false;       // s, written by the leader
      const long long slot = (long long)n * NC;
      for (int j = sc.tid(); j < n; j += sc.nthreads()) {
        double z = 0.0;
        for (int k = 0; k < L; ++k) z += sv[k] * A.lz_store[k * slot + (long long)j * NC + cs];
        zv[j] = z;
      }
    } else {
    // second pass: the same start and recurrence with the stored coefficients
    Qp = A.dir;
    Q = A.grad;
    W = A.grad_old;
    for (int j = sc.tid(); j < n; j += sc.nthreads()) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        Q[(long long)j * NC + c] = normal_at(key, (uint64_t)j * NC + c);
        Qp[(long long)j * NC + c] = 0.0;
      }
      zv[j] = 0.0;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      qs[c] = lz_qs0[c];
      qps[c] = 0.0;
      bp[c] = 0.0;
    }
    if (!sc.sync()) return false;
    for (int k = 0; k < L; ++k) {
      ++lz_steps;
      double a[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) a[c] = hist[c8(k, c)];
      const double sk = sv[k];
      const bool diag = P.a_diag_only != 0;
      const int j0 = diag ? t4.id : w4.warp, js = diag ? t4.count : w4.nwarps;
      for (int j = j0; j < n; j += js) {
        Frag<double> mq;
        if (diag) {
          spmm_row<double>(P, Q, NC, j, A.lam, nullptr, 0.0, -1.0, 0.0, 0.0, t4, mq);
        } else {
          spmm_row_warp<double>(P, Q, NC, j, A.lam, nullptr, 0.0, -1.0, 0.0, 0.0, w4, mq);
          if (w4.sub != 0) continue;
        }
        const long long o = (long long)j * NC;
        zv[j] += sk * qs[cs] * Q[o + cs];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const double w1 = qs[c] * mq.v[0][c] - bp[c] * qps[c] * Qp[o + c];
          W[o + c] = w1 - a[c] * qs[c] * Q[o + c];
        }
      }
      if (!sc.sync()) return false;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double beta = hist[c8(k, c) + 4];
        qps[c] = qs[c];
        qs[c] = len[c] > k + 1 ? 1.0 / beta : 0.0;
        bp[c] = len[c] > k + 1 ? beta : 0.0;
      }
      double* t = Qp;
      Qp = Q;
      Q = W;
      W = t;
    }
    }
    double z2[1] = {0.0};
    for (int j = sc.tid(); j < n; j += sc.nthreads()) z2[0] += zv[j] * zv[j];
    if (!sc.reduce(z2, 1)) return false;
    *zn2 = z2[0];
    return true;
  }

  __device__ static int c8(int k, int c) { return 8 * k + c; }

  // Phase II rank growth: U, V -> [U, tau z, 0], [V, tau z, 0] at rank r_new, z the Ritz
  // vector of lambda_min(C - A^T y) (in A.Y + 2 Kmax, squared norm zn2), tau = escape_scale *
  // ||U_hat||_F / sqrt(r) (the size of an average column); the T shadows follow
  __device__ bool grow_rank_phase2(int r_new, const double* zv, double zn2) {
    const int r_old = r, ld_old = ld;
    const Team t_old = tm;
    for (int j = t_old.id; j < n; j += t_old.count) {
      Frag<double> u, w;
      frag_load(u, A.U, j, ld_old, t_old);
      frag_store(u, A.tmp, j, ld_old, t_old);
      frag_load(w, A.V, j, ld_old, t_old);
      frag_store(w, A.grad, j, ld_old, t_old);
    }
    if (!sc.sync()) return false;
    set_rank(r_new);
    const double tau = zn2 > 0.0 ? prm.escape_scale * sqrt(uh_norm2 / (double)r_old / zn2) : 0.0;
    const bool shadow = (const void*)A.Ut != (const void*)A.U;
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> u, w;
      const double zj = tau * zv[j];
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) {
          const int c = (tm.lane + k * tm.G) * CHUNK + e;
          const long long o = (long long)j * ld_old + c;
          u.v[k][e] = c < r_old ? A.tmp[o] : (c == r_old ? zj : 0.0);
          w.v[k][e] = c < r_old ? A.grad[o] : (c == r_old ? zj : 0.0);
        }
      frag_store(u, A.U, j, ld, tm);
      frag_store(w, A.V, j, ld, tm);
      if (shadow) {
        Frag<T> ut, wt;
        frag_convert(ut, u);
        frag_convert(wt, w);
        frag_store(ut, A.Ut, j, ld, tm);
        frag_store(wt, A.Vt, j, ld, tm);
      }
    }
    return sc.sync();
  }

  // U_hat, objective, dual stationarity, output infeasibility, b^T lambda
  __device__ bool output(double* res) {
    if (prm.lanczos_steps > 0 && lmin_at != admm_iters) {
      if (!lanczos_lambda_min(last_lmin)) return false;
      lmin_at = admm_iters;
    }
    if (!form_u_hat()) return false;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (P.a_diag_only) {
      for (int j = tm.id; j < n; j += tm.count) {
        Frag<double> Uh, mCU, mSU;
        frag_load(Uh, A.tmp, j, ld, tm);
        spmm_row<double>(P, A.tmp, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, 0.0, tm, mCU);
        spmm_row<double>(P, A.tmp, ld, j, A.lam, nullptr, 0.0, -1.0, 0.0, 0.0, tm, mSU);
        const double o = -frag_dot(Uh, mCU, tm), d = frag_dot(mSU, mSU, tm);
        if (tm.lane == 0) {
          v[0] += o;
          v[1] += d;
        }
      }
    } else {
      const WarpRow wr = make_warp_row(ld, sc.tid(), sc.nthreads(), prm.team_mult);
      for (int j = wr.warp; j < n; j += wr.nwarps) {
        Frag<double> Uh, mCU, mSU;
        frag_load(Uh, A.tmp, j, ld, wr.st);
        spmm_row_warp<double>(P, A.tmp, ld, j, nullptr, nullptr, 0.0, 0.0, 0.0, 0.0, wr, mCU);
        spmm_row_warp<double>(P, A.tmp, ld, j, A.lam, nullptr, 0.0, -1.0, 0.0, 0.0, wr, mSU);
        if (wr.sub == 0) {
          const double o = -frag_dot(Uh, mCU, wr.st), d = frag_dot(mSU, mSU, wr.st);
          if (wr.st.lane == 0) {
            v[0] += o;
            v[1] += d;
          }
        }
      }
    }
    auto add = [&](int i, double q, double qs) {
      const double eh = q - P.b[i], es = qs - P.b[i];
      v[2] += eh * eh;
      v[3] += P.b[i] * A.lam[i];
      v[4] += es * es;
    };
    if (P.a_multi) {
      if (!con_chunks<2>([&](int r, int c, double a, double* s) {
            s[0] += sddmm_entry<double>(A.tmp, A.tmp, ld, r, c, a, tmc);
            s[1] += sddmm_entry<double>(A.U, A.V, ld, r, c, a, tmc);
          }))
        return false;
      for (int i = sc.tid(); i < m; i += sc.nthreads()) add(i, con_total(i, 0), con_total(i, 1));
    } else {
      for (int i = tmc.id; i < m; i += tmc.count) {
        const double q = sddmm_con<double>(P, A.tmp, A.tmp, ld, i, tmc);
        const double qs = sddmm_con<double>(P, A.U, A.V, ld, i, tmc);
        if (tmc.lane == 0) add(i, q, qs);
      }
    }
    if (!sc.reduce(v, 5)) return false;
    for (int i = 0; i < 5; ++i) res[i] = v[i];
    return true;
  }

  __device__ void run() {
    t_start = globaltimer_ns();
    double sigma = 0.0, rho = 0.0;
    set_rank(prm.phase1 ? prm.r0 : prm.r_start);
    nzc = prm.phase1 ? r : min(max(prm.nz0, 0), r);
    if (prm.phase1) {
      if (!phase1(sigma)) { finish_error(); return; }
      if (status != ST_OK) { finish(sigma, rho, nullptr, 0, 0); return; }
      rho = fmin(prm.h * sigma, prm.rho_max);
    } else {
      rho = prm.rho0;
      sigma = 1.0 / (1.0 + P.b_inf);     // the penalty a Phase III refinement starts from
      if (prm.resume) {
        admm_iters = prm.k0;
        ndt = prm.next_test0;
        pdinf = prm.prev_dinf0;
        cg_iters = prm.cg0;
        hess = prm.hess0;
        alm_outer = prm.outer0;
        lbfgs_iters = prm.lbfgs0;
        growths = prm.growths0;
        sigma = prm.sigma0;
      }
    }
    // switch: V = U (Algorithm 2), or the checkpointed V of a resume; shadows
    for (int j = tm.id; j < n; j += tm.count) {
      Frag<double> u, w;
      frag_load(u, A.U, j, ld, tm);
      if (prm.resume) frag_load(w, A.V, j, ld, tm);
      else {
        w = u;
        frag_store(u, A.V, j, ld, tm);
      }
      if ((const void*)A.Ut != (const void*)A.U) {
        Frag<T> s;
        frag_convert(s, u);
        frag_store(s, A.Ut, j, ld, tm);
        frag_convert(s, w);
        frag_store(s, A.Vt, j, ld, tm);
      }
    }
    if (!sc.sync()) { finish_error(); return; }
    const long long t1 = globaltimer_ns();
    double rho_out = rho;
    if (!phase2(rho, rho_out)) { finish_error(); return; }
    if (to_polish && status == ST_OK) {
      if (!(polish_applies() ? phase3() : phase3_alm(sigma))) { finish_error(); return; }
    }
    double res[5];
    if (!output(res)) { finish_error(); return; }
    finish(sigma, rho_out, res, t1, 1);
  }

  __device__ void finish_error() {
    if (sc.is_leader()) A.out->status = ST_DEVICE;
  }

  __device__ void finish(double sigma, double rho, const double* res, long long t1, int have) {
    if (!sc.is_leader()) return;
    SolveOut* o = A.out;
    const long long t2 = globaltimer_ns();
    o->status = status;
    o->rank = r;
    o->ld = ld;
    o->admm_iters = admm_iters;
    o->cg_iters = cg_iters;
    o->hess_applies = hess;
    o->alm_outer = alm_outer;
    o->lbfgs_iters = lbfgs_iters;
    o->growths = growths;
    o->phase = have ? 2 : 1;
    o->next_dual_test = ndt;
    o->prev_dinf = pdinf;
    o->rho = rho;
    o->gamma = prm.gamma;
    o->sigma = sigma;
    o->t_phase1_ns = have ? t1 - t_start : t2 - t_start;
    o->t_phase2_ns = have ? (t_p3 > 0 ? t_p3 : t2) - t1 : 0;
    o->t_phase3_ns = (have && t_p3 > 0) ? t2 - t_p3 : 0;
    o->polished = to_polish ? (polish_applies() ? 1 : 2) : 0;
    o->newton_steps = newton_steps;
    o->newton_cg = newton_cg;
    o->lanczos_steps = lz_steps;
    o->t_lanczos_ns = lz_ns;
    o->refine_outer = refine_outer;
    o->refine_lbfgs = refine_lbfgs;
    if (have) {
      const double obj = res[0], dobj = -res[3];
      o->objective = obj;
      o->dual_objective = dobj;
      o->r_D = sqrt(res[1]) / (1.0 + P.C_fro);
      o->r_P = sqrt(res[2]) / (1.0 + P.b_inf);
      o->r_P_split = sqrt(res[4]) / (1.0 + P.b_inf);
      o->gap = (obj - dobj) / (1.0 + fabs(obj) + fabs(dobj));
      o->r_stop = rs_num >= 0.0 ? prm.gamma * sqrt(rs_num) / (1.0 + sqrt(rs_den)) : last_rs;
      o->p_infeas = sqrt(res[2]) / (1.0 + P.b_one);
      o->lambda_min = last_lmin;
      o->d_infeas = last_lmin == last_lmin ? fmax(0.0, -last_lmin) / (1.0 + P.c_one) : NAN;
      o->dual_psd = last_lmin == last_lmin ? dual_psd(last_lmin) : NAN;
    } else {
      o->p_infeas = NAN;
      o->lambda_min = NAN;
      o->d_infeas = NAN;
      o->dual_psd = NAN;
    }
  }
};

template <typename T, int SUB, class Scope>
__device__ void run_solver(const SolverArgs<T>& a, Scope& sc) {
  Solver<T, Scope, SUB> s(a, sc);
  s.run();
}

}  // namespace lorads
