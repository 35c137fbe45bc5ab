// Instantiation of the fused H|psi> kernels without the projector terms: arithmetic float, io complex of double.
#include "fused_kernel.cuh"
#include "fused_window.cuh"

namespace pwk {
int launch_fused_f32c128(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  return launch_fused<float, double, false, false>(N, a, nblocks, s, st);
}
int launch_window_f32c128(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  return launch_window<float, double, false>(N, a, nblocks, s, st);
}
}  // namespace pwk
