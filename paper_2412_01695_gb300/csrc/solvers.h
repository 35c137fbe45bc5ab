// Internal interface between the plan code and the solver translation units.
#pragma once
#include "pwk_internal.h"

namespace pwk {
constexpr int kMaxBasis = 160;   // largest Davidson basis (reduced problem size)

// Free the Davidson and CG workspaces held by a plan (called by pwk_plan_destroy).
void destroy_solver_work(pwk_plan* p);
void destroy_dav_work(pwk_plan* p);
void destroy_cg_work(pwk_plan* p);

// batched generalized eigensolver of the reduced problem (rr.cu)
// drop_out (optional, [nk][ld]): 1 for each basis vector left out as numerically dependent
int launch_rr(int nk, int ld, int nb, const int* nbase, const int* active, const double2* Hr,
              const double2* Sr, double2* W, double2* ev, double* eps, int* status,
              cudaStream_t st, unsigned char* drop_out = nullptr);
}  // namespace pwk
