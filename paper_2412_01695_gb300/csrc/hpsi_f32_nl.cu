// Instantiation of the fused H|psi> kernels with the projector terms applied inside them
// (nl_fused.cuh): arithmetic float, io complex of float.
#include "fused_kernel.cuh"
#include "fused_window.cuh"

namespace pwk {
int launch_fused_f32_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  return launch_fused<float, float, false, true>(N, a, nblocks, s, st);
}
int launch_window_f32_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  return launch_window<float, float, true>(N, a, nblocks, s, st);
}
}  // namespace pwk
