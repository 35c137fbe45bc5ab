// Instantiation of the fused H|psi> kernels with the projector terms applied inside them
// (nl_fused.cuh): arithmetic double, io complex of double.
#include "fused_kernel.cuh"
#include "fused_window.cuh"

namespace pwk {
int launch_fused_f64_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  return launch_fused<double, double, false, true>(N, a, nblocks, s, st);
}
int launch_window_f64_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  return launch_window<double, double, true>(N, a, nblocks, s, st);
}
}  // namespace pwk
