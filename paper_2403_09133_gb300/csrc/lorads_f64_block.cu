// Plain FP64 form of the one-CTA solver kernel (small problems and batches), a unit of its own
// so that the units compile in parallel.  This kernel has twice diverged on matrix completion
// (CG iterations growing without bound in Phase II) after code changes elsewhere in the solver:
// once at ptxas -O3, later at -O1, each time passing again at the other level; the FP32 form
// and the whole-GPU FP64 kernel of the same source never did.  The cause is not identified.
// The GPU tests repeat FP64 one-CTA matrix-completion solves, require identical results and
// compare them with the whole-GPU kernel and the oracle.
#include "lorads_kernels.cuh"
namespace lorads {
LORADS_DEFINE_SOLVE_LAUNCH_BLOCK(double, 0)
}
