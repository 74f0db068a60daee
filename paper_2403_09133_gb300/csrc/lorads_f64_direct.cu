// Plain FP64 form with the exact row-block subproblem solve (its own translation unit, so
// that it compiles in parallel with the CG kernels).
#include "lorads_kernels.cuh"
namespace lorads {
LORADS_DEFINE_SOLVE_LAUNCH(double, 1)
}
