"""Scheduling logic of the serving loop without a GPU (a fake executor that sleeps):
admission never exceeds the HBM budget or the slots, jobs that arrive while others run start
as soon as room frees up, H|psi> requests on the same cell are coalesced, failures are
reported without stopping the server."""
import threading
import time

from paper_2412_01695_gb300 import serve


def _cell(seed=0):
    return serve.CellSpec("fcc", 7.0, 1, 30.0, 16, 2, seed)


class FakeExec:
    def __init__(self, dt=0.02, fail_kind=None):
        self.dt = dt
        self.fail_kind = fail_kind
        self.lock = threading.Lock()
        self.groups = []
        self.active = 0
        self.max_active = 0

    def __call__(self, group, slot):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.groups.append([j.jid for j in group])
        time.sleep(self.dt)
        with self.lock:
            self.active -= 1
        if group[0].kind == self.fail_kind:
            raise RuntimeError("planted failure")
        for j in group:
            j.result = j.jid


def test_budget_and_slots_respected():
    jobs = [serve.Job(i, "davidson", _cell(i % 3), 8, arrival=0.001 * i, footprint=40)
            for i in range(24)]
    ex = FakeExec()
    s = serve.Server(ex, hbm_budget=100, slots=4)
    done = s.run(jobs, realtime=True)
    assert [j.jid for j in done] == list(range(24))
    assert all(j.result == j.jid and j.error is None for j in done)
    assert s.peak_in_use <= 100
    assert ex.max_active <= 2             # 2 x 40 fits in 100, 3 x 40 does not
    assert all(j.start >= j.arrival - 1e-9 and j.finish >= j.start for j in done)


def test_continuous_admission_while_running():
    """A job arriving while a long one runs starts before the long one finishes."""
    long_job = serve.Job(0, "davidson", _cell(), 8, arrival=0.0, footprint=10)
    short = serve.Job(1, "davidson", _cell(1), 8, arrival=0.01, footprint=10)

    class Ex(FakeExec):
        def __call__(self, group, slot):
            time.sleep(0.3 if group[0].jid == 0 else 0.01)
            for j in group:
                j.result = j.jid

    s = serve.Server(Ex(), hbm_budget=100, slots=2)
    done = s.run([long_job, short], realtime=True)
    assert done[1].finish < done[0].finish


def test_hpsi_coalescing():
    """Waiting H|psi> jobs on the same cell and band count run as one group."""
    blocker = serve.Job(0, "davidson", _cell(9), 8, arrival=0.0, footprint=10)
    hp = [serve.Job(1 + i, "hpsi", _cell(), 8, arrival=0.001, footprint=1) for i in range(5)]
    ex = FakeExec(dt=0.05)
    s = serve.Server(ex, hbm_budget=100, slots=1)
    s.run([blocker] + hp, realtime=False)
    assert [1, 2, 3, 4, 5] in ex.groups


def test_oversized_job_runs_alone_and_failures_are_reported():
    big = serve.Job(0, "sternheimer", _cell(), 8, arrival=0.0, footprint=500)
    small = [serve.Job(1 + i, "davidson", _cell(i), 8, arrival=0.0, footprint=10) for i in range(3)]
    ex = FakeExec(fail_kind="sternheimer")
    s = serve.Server(ex, hbm_budget=100, slots=4)
    done = s.run([big] + small, realtime=False)
    assert done[0].error is not None and "planted" in done[0].error
    assert all(j.error is None for j in done[1:])
    st = serve.latency_stats(done)
    assert st["failed"] == 1 and st["jobs"] == 4


def test_random_mix_is_seeded_and_poisson():
    a = serve.random_mix(200, rate_hz=100.0, seed=3)
    b = serve.random_mix(200, rate_hz=100.0, seed=3)
    assert [(j.kind, j.cell) for j in a] == [(j.kind, j.cell) for j in b]
    kinds = [j.kind for j in a]
    assert 0.45 < kinds.count("hpsi") / 200 < 0.75
    gaps = [a[i + 1].arrival - a[i].arrival for i in range(199)]
    assert 0.005 < sum(gaps) / len(gaps) < 0.02     # mean 1/rate
