// Solver workspaces and entry points (filled in by davidson.cu / sternheimer.cu).
#include "solvers.h"

namespace pwk {
void destroy_solver_work(pwk_plan*) {}
}  // namespace pwk

extern "C" {
int pwk_davidson_batched(pwk_plan*, int, void*, double*, int, double, double, int, int, int*, int*,
                         long long*, void*) {
  pwk::set_error("not built yet");
  return PWK_ERR_UNSUPPORTED;
}
int pwk_sternheimer_cg_batched(pwk_plan*, pwk_plan*, int, const void*, const double*, const void*,
                               int, const double*, const void*, void*, double, int, int*, double*,
                               void*) {
  pwk::set_error("not built yet");
  return PWK_ERR_UNSUPPORTED;
}
}
