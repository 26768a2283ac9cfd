// Kernel instantiations for the D2Q49 lattice.
#include "lbm_step.cuh"

namespace lbm {
cudaError_t launch_d2q49(Op op, const Args &a, cudaStream_t s) { return launch_lattice<3>(op, a, s); }
}  // namespace lbm
