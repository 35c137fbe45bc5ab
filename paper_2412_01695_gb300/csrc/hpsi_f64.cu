// Instantiation of the fused H|psi> kernels without the projector terms: arithmetic double, io complex of double.
#include "fused_kernel.cuh"
#include "fused_window.cuh"

namespace pwk {
int launch_fused_f64(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  return launch_fused<double, double, false, false>(N, a, nblocks, s, st);
}
int launch_window_f64(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  return launch_window<double, double, false>(N, a, nblocks, s, st);
}
}  // namespace pwk
