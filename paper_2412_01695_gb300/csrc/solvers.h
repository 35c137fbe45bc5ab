// Internal interface between the plan code and the solver translation units.
#pragma once
#include <vector>

#include "pwk_internal.h"

namespace pwk {
constexpr int kMaxBasis = 160;   // largest Davidson basis (reduced problem size)

// Free the Davidson and CG workspaces held by a plan (called by pwk_plan_destroy).
void destroy_solver_work(pwk_plan* p);
void destroy_dav_work(pwk_plan* p);
void destroy_cg_work(pwk_plan* p);

// batched generalized eigensolver of the reduced problem (rr.cu)
// drop_out (optional, [nk][ld]): 1 for each basis vector left out as numerically dependent
// flops (optional, device): the algorithmic FP64 operation count of every problem solved is
// added to it
int launch_rr(int nk, int ld, int nb, const int* nbase, const int* active, const double2* Hr,
              const double2* Sr, double2* W, double2* ev, double* eps, int* status,
              cudaStream_t st, unsigned char* drop_out = nullptr, double* flops = nullptr);

// Device time of the phases of a solver call (pwk_plan_set_solver_timing): CUDA events are
// recorded around each phase on the solver's stream and read after the stream synchronises
// (the solvers synchronise once per iteration anyway), so timing adds no synchronisation.
// Phases: 0 H (and S) applications, 1 reduced eigensolves, 2 the rest of the vector kernels
// is the call's total minus these.
struct PhaseTimer {
  pwk_plan* p = nullptr;
  cudaStream_t st = nullptr;
  bool on = false;
  cudaEvent_t first = nullptr;
  std::vector<cudaEvent_t> pool;
  struct Open { int phase; cudaEvent_t a, b; };
  std::vector<Open> open;
  double ms[2] = {0.0, 0.0};
  PhaseTimer(pwk_plan* plan, cudaStream_t stream);
  ~PhaseTimer();
  cudaEvent_t mark();                         // an event recorded on the stream now
  void close(int phase, cudaEvent_t a);       // the phase that began at a ends now
  void harvest();                             // after a synchronisation: add the elapsed times
  void finish();                              // synchronise, store the call's figures in the plan
};

}  // namespace pwk
