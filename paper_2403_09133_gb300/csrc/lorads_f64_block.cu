// Plain FP64 form of the one-CTA solver kernel (small problems and batches).  build.py compiles
// this unit with ptxas at -O1: at -O3 (CUDA 13.0, sm_103a) this kernel gave non-deterministic,
// diverging CG iterations on problems with off-diagonal constraints (matrix completion), while
// the same source at -O1, the FP32 form and the whole-GPU FP64 kernel gave the same iterates.
#include "lorads_kernels.cuh"
namespace lorads {
LORADS_DEFINE_SOLVE_LAUNCH_BLOCK(double, 0)
}
