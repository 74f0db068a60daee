// Plain FP64 form of the solver (whole-GPU and CTA-group kernels) and operators.  The one-CTA
// kernel of this form is in lorads_f64_block.cu.
#include "lorads_kernels.cuh"
namespace lorads {
LORADS_DEFINE_LAUNCH(double)
LORADS_DEFINE_SOLVE_LAUNCH_MULTI(double, 0)
}
