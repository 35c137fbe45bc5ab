"""Serving loop on the GPU: every job's result is the same when it runs alone and when it runs
in a mix with other jobs overlapping on the device (within the stated tolerances: H|psi>
1e-12 relative, eigenvalues 1e-8 Ry, Sternheimer solutions 1e-6 relative with residuals
<= 1e-10 in both runs)."""
import numpy as np
import pytest

from paper_2412_01695_gb300 import serve

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _mix():
    jobs = serve.random_mix(14, rate_hz=500.0, seed=11, max_nk=8, max_nb=8, ecut_range=(20.0, 28.0))
    kinds = {j.kind for j in jobs}
    assert {"hpsi", "davidson"} <= kinds
    # make sure a coalescable pair and a Sternheimer job are present
    jobs[1] = serve.Job(1, "hpsi", jobs[0].cell, jobs[0].nb, arrival=jobs[1].arrival) \
        if jobs[0].kind == "hpsi" else jobs[1]
    jobs[-1] = serve.Job(jobs[-1].jid, "sternheimer", jobs[-1].cell, 4, arrival=jobs[-1].arrival)
    return jobs


def _copy(jobs):
    return [serve.Job(j.jid, j.kind, j.cell, j.nb, arrival=j.arrival) for j in jobs]


def test_each_result_alone_equals_result_in_the_mix():
    torch_cuda()
    jobs = _mix()
    # alone: one slot, no coalescing, jobs one after the other
    ex1 = serve.GpuExecutor(slots=1)
    ex1.prepare(jobs)
    alone = serve.Server(ex1, hbm_budget=64 << 30, slots=1, estimate=serve.estimate_for,
                         coalesce=False).run(_copy(jobs), realtime=False)
    # mix: four slots, coalescing, Poisson arrivals in real time
    ex4 = serve.GpuExecutor(slots=4)
    ex4.prepare(jobs)
    srv = serve.Server(ex4, hbm_budget=64 << 30, slots=4, estimate=serve.estimate_for)
    mixed = srv.run(_copy(jobs), realtime=True)
    assert all(j.error is None for j in alone), [j.error for j in alone if j.error]
    assert all(j.error is None for j in mixed), [j.error for j in mixed if j.error]
    for a, m in zip(alone, mixed):
        assert a.jid == m.jid
        if a.kind == "hpsi":
            num = np.linalg.norm(a.result - m.result, axis=-1)
            den = np.maximum(np.linalg.norm(a.result, axis=-1), 1e-300)
            assert np.max(num / den) <= 1e-12
        elif a.kind == "davidson":
            np.testing.assert_allclose(m.result, a.result, atol=1e-8, rtol=0)
        else:
            # the valence states of each run come from its own FP64 Davidson (on plans tuned
            # apart), so within a degenerate level they may differ by a unitary mix, which dpsi
            # follows; sum_n |dpsi_n><psi_n| per k-point is the same either way
            xa, ra, ua = a.result
            xm, rm, um = m.result
            assert ra.max() <= 1e-10 and rm.max() <= 1e-10
            ma = np.einsum("kng,knh->kgh", xa, ua.conj())
            mm = np.einsum("kng,knh->kgh", xm, um.conj())
            assert np.linalg.norm(ma - mm) <= 1e-6 * np.linalg.norm(ma)
    st = serve.latency_stats(mixed)
    assert st["p99_s"] >= st["p50_s"] > 0
