// Internal interface between the plan code and the solver translation units.
#pragma once
#include "pwk_internal.h"

namespace pwk {
// Free the Davidson and CG workspaces held by a plan (called by pwk_plan_destroy).
void destroy_solver_work(pwk_plan* p);
}  // namespace pwk
