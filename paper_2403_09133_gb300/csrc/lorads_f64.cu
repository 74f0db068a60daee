// Plain FP64 form of the solver and operators.
#include "lorads_kernels.cuh"
namespace lorads {
LORADS_DEFINE_LAUNCH(double)
LORADS_DEFINE_SOLVE_LAUNCH(double, 0)
}
