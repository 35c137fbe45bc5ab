// Workspace teardown shared by the solvers, and the phase timer of a solver call.
#include "solvers.h"

namespace pwk {
void destroy_solver_work(pwk_plan* p) {
  destroy_dav_work(p);
  destroy_cg_work(p);
}

PhaseTimer::PhaseTimer(pwk_plan* plan, cudaStream_t stream) : p(plan), st(stream), on(plan->solver_timing) {
  if (!on) return;
  if (p->d_flops != nullptr) cudaMemsetAsync(p->d_flops, 0, sizeof(double), st);
  first = mark();
}

PhaseTimer::~PhaseTimer() {
  for (auto& o : open) {
    pool.push_back(o.a);
    pool.push_back(o.b);
  }
  if (first) pool.push_back(first);
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

cudaEvent_t PhaseTimer::mark() {
  if (!on) return nullptr;
  cudaEvent_t e = nullptr;
  if (!pool.empty()) {
    e = pool.back();
    pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    on = false;   // no events: the call goes on untimed
    return nullptr;
  }
  cudaEventRecord(e, st);
  return e;
}

void PhaseTimer::close(int phase, cudaEvent_t a) {
  if (!on || a == nullptr) return;
  cudaEvent_t b = mark();
  if (b != nullptr) open.push_back({phase, a, b});
}

void PhaseTimer::harvest() {
  if (!on) return;
  for (auto& o : open) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, o.a, o.b) == cudaSuccess) ms[o.phase] += t;
    else cudaGetLastError();
    pool.push_back(o.a);
    pool.push_back(o.b);
  }
  open.clear();
}

void PhaseTimer::finish() {
  if (!on) return;
  cudaEvent_t last = mark();
  double flops = 0.0;
  if (p->d_flops != nullptr) cudaMemcpyAsync(&flops, p->d_flops, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  harvest();
  float total = 0.f;
  if (last != nullptr && cudaEventElapsedTime(&total, first, last) != cudaSuccess) cudaGetLastError();
  if (last != nullptr) pool.push_back(last);
  p->solver_stats[0] = ms[0];
  p->solver_stats[1] = ms[1];
  p->solver_stats[2] = total;
  p->solver_stats[3] = flops;
  p->solver_stats[4] = total - ms[0] - ms[1];
}
}  // namespace pwk

using namespace pwk;

extern "C" int pwk_plan_set_solver_timing(pwk_plan* p, int on) {
  if (p == nullptr) {
    set_error("null plan");
    return PWK_ERR_INVALID;
  }
  if (on && p->d_flops == nullptr) {
    if (int rc = plan_alloc(p, (void**)&p->d_flops, sizeof(double))) return rc;
  }
  p->solver_timing = on != 0;
  return PWK_OK;
}

extern "C" int pwk_plan_solver_stats(const pwk_plan* p, double* stats) {
  if (p == nullptr || stats == nullptr) {
    set_error("null pointer");
    return PWK_ERR_INVALID;
  }
  for (int i = 0; i < 5; ++i) stats[i] = p->solver_stats[i];
  return PWK_OK;
}
