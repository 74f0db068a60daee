// Mixed form: FP32 CG operators and vectors, FP64 masters and scalars.
#include "lorads_kernels.cuh"
namespace lorads {
LORADS_DEFINE_LAUNCH(float)
LORADS_DEFINE_SOLVE_LAUNCH(float, 0)
}
