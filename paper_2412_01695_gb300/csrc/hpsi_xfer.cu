// Instantiation of the fused H|psi> kernel: arithmetic double, io complex of double, complex dv (DFPT right-hand side).
#include "fused_kernel.cuh"

namespace pwk {
int launch_fused_xfer(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  return launch_fused<double, double, true, false>(N, a, nblocks, s, st);
}
}  // namespace pwk
