// Instantiation of the window kernel over work lists that span several plans of one grid
// (pwk_hpsi_multi), for every precision; the projector terms are applied inside the kernel.
#include "fused_window.cuh"

namespace pwk {
int launch_window_multi_prec(int precision, int N, const FusedArgs& a, int nblocks, const LaunchShape& s,
                             cudaStream_t st) {
  switch (precision) {
    case PWK_FP64: return launch_window_multi<double, double>(N, a, nblocks, s, st);
    case PWK_FP32: return launch_window_multi<float, float>(N, a, nblocks, s, st);
    default: return launch_window_multi<float, double>(N, a, nblocks, s, st);
  }
}
}  // namespace pwk
