// Workspace teardown shared by the solvers.
#include "solvers.h"

namespace pwk {
void destroy_solver_work(pwk_plan* p) {
  destroy_dav_work(p);
  destroy_cg_work(p);
}
}  // namespace pwk
