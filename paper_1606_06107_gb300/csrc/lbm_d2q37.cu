// Kernel instantiations for the D2Q37 lattice.
#include "lbm_step.cuh"

namespace lbm {
cudaError_t launch_d2q37(Op op, const Args &a, cudaStream_t s) { return launch_lattice<2>(op, a, s); }
}  // namespace lbm
