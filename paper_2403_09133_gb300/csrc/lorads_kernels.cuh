// Kernel entry points of the solver and of the operator calls, instantiated per element
// type by lorads_f64.cu / lorads_f32.cu.
#pragma once
#include "lorads_solver.cuh"

namespace lorads {

constexpr int SOLVER_THREADS = 256;       // one-CTA solver: default CTA size ...
constexpr int BLOCK_THREADS_MAX = 384;    // ... and the largest (batches autotune 128..384)
constexpr int GRID_THREADS_MAX = 320;     // grid solver: CTA size chosen per problem
constexpr int SOLVER_THREADS_MIN = 128;   // every solver CTA: four warps, one per Lanczos chain

// one CTA per problem; CTAs take problems from a queue (batches), or a single problem
template <typename T, int SUB>
__global__ void __launch_bounds__(BLOCK_THREADS_MAX, 1)
solve_block_kernel(const SolverArgs<T>* args, int count, int* queue) {
  __shared__ double red[34 * MAXRED];
  __shared__ SolverArgs<T> sa;
  __shared__ int inst;
  for (;;) {
    if (threadIdx.x == 0) inst = atomicAdd(queue, 1);
    __syncthreads();
    const int i = inst;
    if (i >= count) return;
    if (threadIdx.x == 0) sa = args[i];
    __syncthreads();
    BlockScope sc{red};
    run_solver<T, SUB>(sa, sc);
    __syncthreads();
  }
}

// one problem over the whole grid (cooperative launch: all CTAs co-resident)
template <typename T, int SUB>
__global__ void __launch_bounds__(GRID_THREADS_MAX, 1)
solve_grid_kernel(const SolverArgs<T>* args, GridCtl* ctl, double* partials, long long spin) {
  __shared__ double red[34 * MAXRED];
  __shared__ SolverArgs<T> sa;
  if (threadIdx.x == 0) sa = *args;
  __syncthreads();
  GridScope sc{red, ctl, partials, spin, 0, (int)gridDim.x};
  run_solver<T, SUB>(sa, sc);
}

// batches with several CTAs per problem: CTAs [g * group, (g + 1) * group) form group g,
// which takes problems from the queue (largest first) and solves each with a scope spanning
// the group (ctls[g] is its barrier, slots[g] the index its leader fetched).  The launch is
// cooperative, so every CTA of a group is resident and the group's bounded barriers never
// wait on a CTA that has not started.
template <typename T, int SUB>
__global__ void __launch_bounds__(BLOCK_THREADS_MAX, 1)
solve_group_kernel(const SolverArgs<T>* args, int count, int* queue, GridCtl* ctls,
                   double* partials, int* slots, int group, long long spin) {
  __shared__ double red[34 * MAXRED];
  __shared__ SolverArgs<T> sa;
  const int g = blockIdx.x / group;
  GroupScope sc{{red, ctls + g, partials, spin, g * group, group}};
  for (;;) {
    if (sc.is_leader()) slots[g] = atomicAdd(queue, 1);
    if (!sc.sync()) return;
    const int i = __ldcg(slots + g);
    if (i >= count) return;
    if (threadIdx.x == 0) sa = args[i];
    __syncthreads();
    run_solver<T, SUB>(sa, sc);
    __syncthreads();
  }
}

// ---- operators on caller-owned device arrays ----
template <typename T>
__global__ void op_sddmm_kernel(DevProblem P, int ld, const T* U, const T* V, double* q) {
  const Team t = make_team(ld, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  for (int i = t.id; i < P.m; i += t.count) {
    const double v = sddmm_con<T>(P, U, V, ld, i, t);
    if (t.lane == 0) q[i] = v;
  }
}

template <typename T>
__global__ void op_spmm_kernel(DevProblem P, int ld, const double* w, double gamma, const T* V,
                               T* out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  if (P.a_diag_only) {
    const Team t = make_team(ld, tid, nt);
    for (int j = t.id; j < P.n; j += t.count) {
      Frag<T> o;
      spmm_row<T>(P, V, ld, j, w, nullptr, 0.0, 1.0, 0.0, (T)gamma, t, o);
      frag_store(o, out, j, ld, t);
    }
  } else {
    const WarpRow wr = make_warp_row(ld, tid, nt);
    for (int j = wr.warp; j < P.n; j += wr.nwarps) {
      Frag<T> o;
      spmm_row_warp<T>(P, V, ld, j, w, nullptr, 0.0, 1.0, 0.0, (T)gamma, wr, o);
      if (wr.sub == 0) frag_store(o, out, j, ld, wr.st);
    }
  }
}

template <typename T>
__global__ void op_hessian_kernel(DevProblem P, int ld, T rho, T gamma, const T* V, const T* Pm,
                                  T* out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  if (P.a_diag_only) {
    const Team t = make_team(ld, tid, nt);
    for (int j = t.id; j < P.n; j += t.count) {
      Frag<T> Pj, H;
      frag_load(Pj, Pm, j, ld, t);
      hessian_row<T>(P, V, Pm, ld, j, Pj, rho, gamma, t, H);
      frag_store(H, out, j, ld, t);
    }
  } else {
    const WarpRow wr = make_warp_row(ld, tid, nt);
    for (int j = wr.warp; j < P.n; j += wr.nwarps) {
      Frag<T> Pj, H;
      frag_load(Pj, Pm, j, ld, wr.st);
      hessian_row_warp<T>(P, V, Pm, ld, j, Pj, rho, gamma, wr, H);
      if (wr.sub == 0) frag_store(H, out, j, ld, wr.st);
    }
  }
}

// Hessian of eq. linU for multi-entry constraints from q_i = <A_i, P V^T> (op_sddmm_kernel)
template <typename T>
__global__ void op_hessian_q_kernel(DevProblem P, int ld, T rho, T gamma, const T* V,
                                    const T* Pm, const double* q, T* out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  const WarpRow wr = make_warp_row(ld, tid, nt);
  for (int j = wr.warp; j < P.n; j += wr.nwarps) {
    Frag<T> Pj, H;
    frag_load(Pj, Pm, j, ld, wr.st);
    hessian_row_q_warp<T>(P, V, ld, j, Pj, q, rho, gamma, wr, H);
    if (wr.sub == 0) frag_store(H, out, j, ld, wr.st);
  }
}

// host-side launchers of the solver kernels, per element type and subproblem solver
// (defined in lorads_f64.cu / lorads_f32.cu for SUB 0 and lorads_f64_direct.cu /
// lorads_f32_direct.cu for SUB 1, compiled in parallel)
template <typename T, int SUB>
struct SolveLaunch {
  static cudaError_t solve_block(const SolverArgs<T>* args, int count, int* queue, int grid,
                                 int threads, cudaStream_t s);
  static cudaError_t block_capacity(int threads, int* blocks_per_sm);
  static cudaError_t solve_grid(const SolverArgs<T>* args, GridCtl* ctl, double* partials,
                                long long spin, int grid, int threads, cudaStream_t s);
  static cudaError_t grid_capacity(int threads, int* blocks_per_sm);
  static cudaError_t solve_group(const SolverArgs<T>* args, int count, int* queue, GridCtl* ctls,
                                 double* partials, int* slots, int group, long long spin,
                                 int grid, int threads, cudaStream_t s);
  static cudaError_t group_capacity(int threads, int* blocks_per_sm);
};

#define LORADS_DECLARE_SOLVE_LAUNCH(T, SUB)                                                    \
  template <> cudaError_t SolveLaunch<T, SUB>::solve_block(const SolverArgs<T>*, int, int*,    \
                                                           int, int, cudaStream_t);            \
  template <> cudaError_t SolveLaunch<T, SUB>::block_capacity(int, int*);                      \
  template <> cudaError_t SolveLaunch<T, SUB>::solve_grid(const SolverArgs<T>*, GridCtl*,      \
                                                          double*, long long, int, int,        \
                                                          cudaStream_t);                       \
  template <> cudaError_t SolveLaunch<T, SUB>::grid_capacity(int, int*);                       \
  template <> cudaError_t SolveLaunch<T, SUB>::solve_group(const SolverArgs<T>*, int, int*,    \
                                                           GridCtl*, double*, int*, int,       \
                                                           long long, int, int, cudaStream_t); \
  template <> cudaError_t SolveLaunch<T, SUB>::group_capacity(int, int*);
LORADS_DECLARE_SOLVE_LAUNCH(double, 0)
LORADS_DECLARE_SOLVE_LAUNCH(float, 0)
LORADS_DECLARE_SOLVE_LAUNCH(double, 1)
LORADS_DECLARE_SOLVE_LAUNCH(float, 1)

#define LORADS_DEFINE_SOLVE_LAUNCH_BLOCK(T, SUB)                                               \
  template <>                                                                                  \
  cudaError_t SolveLaunch<T, SUB>::solve_block(const SolverArgs<T>* args, int count,           \
                                               int* queue, int grid, int threads,              \
                                               cudaStream_t s) {                               \
    solve_block_kernel<T, SUB><<<grid, threads, 0, s>>>(args, count, queue);                   \
    return cudaGetLastError();                                                                 \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t SolveLaunch<T, SUB>::block_capacity(int threads, int* blocks_per_sm) {           \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,                        \
                                                         solve_block_kernel<T, SUB>, threads,  \
                                                         0);                                   \
  }

#define LORADS_DEFINE_SOLVE_LAUNCH_MULTI(T, SUB)                                               \
  template <>                                                                                  \
  cudaError_t SolveLaunch<T, SUB>::solve_grid(const SolverArgs<T>* args, GridCtl* ctl,         \
                                              double* partials, long long spin, int grid,      \
                                              int threads, cudaStream_t s) {                   \
    void* kargs[] = {(void*)&args, (void*)&ctl, (void*)&partials, (void*)&spin};               \
    return cudaLaunchCooperativeKernel((const void*)solve_grid_kernel<T, SUB>, dim3(grid),     \
                                       dim3(threads), kargs, 0, s);                            \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t SolveLaunch<T, SUB>::grid_capacity(int threads, int* blocks_per_sm) {            \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,                        \
                                                         solve_grid_kernel<T, SUB>, threads,   \
                                                         0);                                   \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t SolveLaunch<T, SUB>::solve_group(const SolverArgs<T>* args, int count,           \
                                               int* queue, GridCtl* ctls, double* partials,    \
                                               int* slots, int group, long long spin,          \
                                               int grid, int threads, cudaStream_t s) {        \
    void* kargs[] = {(void*)&args,     (void*)&count, (void*)&queue, (void*)&ctls,             \
                     (void*)&partials, (void*)&slots, (void*)&group, (void*)&spin};            \
    return cudaLaunchCooperativeKernel((const void*)solve_group_kernel<T, SUB>, dim3(grid),    \
                                       dim3(threads), kargs, 0, s);                            \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t SolveLaunch<T, SUB>::group_capacity(int threads, int* blocks_per_sm) {           \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,                        \
                                                         solve_group_kernel<T, SUB>, threads,  \
                                                         0);                                   \
  }

#define LORADS_DEFINE_SOLVE_LAUNCH(T, SUB) \
  LORADS_DEFINE_SOLVE_LAUNCH_BLOCK(T, SUB) \
  LORADS_DEFINE_SOLVE_LAUNCH_MULTI(T, SUB)

// the solver launchers by run-time subproblem solver, and the operator launchers
template <typename T>
struct Launch {
  static cudaError_t solve_block(int sub, const SolverArgs<T>* args, int count, int* queue,
                                 int grid, int threads, cudaStream_t s) {
    return sub ? SolveLaunch<T, 1>::solve_block(args, count, queue, grid, threads, s)
               : SolveLaunch<T, 0>::solve_block(args, count, queue, grid, threads, s);
  }
  static cudaError_t block_capacity(int sub, int threads, int* blocks_per_sm) {
    return sub ? SolveLaunch<T, 1>::block_capacity(threads, blocks_per_sm)
               : SolveLaunch<T, 0>::block_capacity(threads, blocks_per_sm);
  }
  static cudaError_t solve_grid(int sub, const SolverArgs<T>* args, GridCtl* ctl,
                                double* partials, long long spin, int grid, int threads,
                                cudaStream_t s) {
    return sub ? SolveLaunch<T, 1>::solve_grid(args, ctl, partials, spin, grid, threads, s)
               : SolveLaunch<T, 0>::solve_grid(args, ctl, partials, spin, grid, threads, s);
  }
  static cudaError_t grid_capacity(int sub, int threads, int* blocks_per_sm) {
    return sub ? SolveLaunch<T, 1>::grid_capacity(threads, blocks_per_sm)
               : SolveLaunch<T, 0>::grid_capacity(threads, blocks_per_sm);
  }
  static cudaError_t solve_group(int sub, const SolverArgs<T>* args, int count, int* queue,
                                 GridCtl* ctls, double* partials, int* slots, int group,
                                 long long spin, int grid, int threads, cudaStream_t s) {
    return sub ? SolveLaunch<T, 1>::solve_group(args, count, queue, ctls, partials, slots,
                                                group, spin, grid, threads, s)
               : SolveLaunch<T, 0>::solve_group(args, count, queue, ctls, partials, slots,
                                                group, spin, grid, threads, s);
  }
  static cudaError_t group_capacity(int sub, int threads, int* blocks_per_sm) {
    return sub ? SolveLaunch<T, 1>::group_capacity(threads, blocks_per_sm)
               : SolveLaunch<T, 0>::group_capacity(threads, blocks_per_sm);
  }
  static cudaError_t op_sddmm(const DevProblem& P, int ld, const T* U, const T* V, double* q,
                              int grid, cudaStream_t s);
  static cudaError_t op_spmm(const DevProblem& P, int ld, const double* w, double gamma,
                             const T* V, T* out, int grid, cudaStream_t s);
  static cudaError_t op_hessian(const DevProblem& P, int ld, double rho, double gamma, const T* V,
                                const T* Pm, T* out, int grid, cudaStream_t s);
};

#define LORADS_DECLARE_LAUNCH(T)                                                               \
  template <> cudaError_t Launch<T>::op_sddmm(const DevProblem&, int, const T*, const T*,      \
                                              double*, int, cudaStream_t);                      \
  template <> cudaError_t Launch<T>::op_spmm(const DevProblem&, int, const double*, double,    \
                                             const T*, T*, int, cudaStream_t);                  \
  template <> cudaError_t Launch<T>::op_hessian(const DevProblem&, int, double, double,        \
                                                const T*, const T*, T*, int, cudaStream_t);
LORADS_DECLARE_LAUNCH(double)
LORADS_DECLARE_LAUNCH(float)

#define LORADS_DEFINE_LAUNCH(T)                                                                \
  template <>                                                                                  \
  cudaError_t Launch<T>::op_sddmm(const DevProblem& P, int ld, const T* U, const T* V,         \
                                  double* q, int grid, cudaStream_t s) {                       \
    op_sddmm_kernel<T><<<grid, 256, 0, s>>>(P, ld, U, V, q);                                   \
    return cudaGetLastError();                                                                 \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t Launch<T>::op_spmm(const DevProblem& P, int ld, const double* w, double gamma,   \
                                 const T* V, T* out, int grid, cudaStream_t s) {               \
    op_spmm_kernel<T><<<grid, 256, 0, s>>>(P, ld, w, gamma, V, out);                           \
    return cudaGetLastError();                                                                 \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t Launch<T>::op_hessian(const DevProblem& P, int ld, double rho, double gamma,     \
                                    const T* V, const T* Pm, T* out, int grid,                 \
                                    cudaStream_t s) {                                          \
    if (P.a_multi) {                                                                           \
      op_sddmm_kernel<T><<<grid, 256, 0, s>>>(P, ld, Pm, V, P.op_q);                           \
      op_hessian_q_kernel<T><<<grid, 256, 0, s>>>(P, ld, (T)rho, (T)gamma, V, Pm, P.op_q, out); \
    } else {                                                                                   \
      op_hessian_kernel<T><<<grid, 256, 0, s>>>(P, ld, (T)rho, (T)gamma, V, Pm, out);          \
    }                                                                                          \
    return cudaGetLastError();                                                                 \
  }

}  // namespace lorads
