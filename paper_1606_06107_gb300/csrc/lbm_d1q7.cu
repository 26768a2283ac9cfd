// Kernel instantiations for the D1Q7 lattice.
#include "lbm_step.cuh"

namespace lbm {
cudaError_t launch_d1q7(Op op, const Args &a, cudaStream_t s) { return launch_lattice<1>(op, a, s); }
}  // namespace lbm
