"""Serving loop: H|psi>, Davidson and Sternheimer jobs on one GPU, admitted as they arrive.

A job names a synthetic cell (lattice, atoms, cut-off, grid), a set of k-points and an
operation.  The server
  * admits a queued job when a slot is free and its estimated device footprint fits in the
    HBM budget next to the jobs already running (the analogue of the paper's memgpu: a block
    of k-points is loaded only when the GPU memory allows it, Sec. 4 / Sec. 7.1);
  * runs every admitted job on its own worker thread and CUDA stream, so the work of different
    jobs overlaps on the device (a job that arrives while others run starts as soon as a slot
    and memory are free: continuous admission, not a queue in front of one job at a time);
  * coalesces H|psi> requests on the same cell and k-set that wait in the queue into one
    batched launch (one work list over all their bands);
  * keeps the plans (k-point tables, projectors, V(r)) of recently used cells resident on the
    device, evicting the least recently used when the budget needs the room;
  * records, per job, the arrival, start and finish times (latency = finish - arrival).
The kernels are the library's (C ABI through the binding); this module is host-side logic.
The executor is pluggable so the scheduling can be tested without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import threading
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass(frozen=True)
class CellSpec:
    lattice: str          # "fcc" or "sc"
    a: float              # bohr
    nat: int
    ecut: float           # Ry
    N: int                # FFT grid
    mp: int               # MP grid q x q x q
    seed: int


@dataclasses.dataclass
class Job:
    jid: int
    kind: str             # "hpsi" | "davidson" | "sternheimer"
    cell: CellSpec
    nb: int
    arrival: float = 0.0
    start: float = math.nan
    finish: float = math.nan
    footprint: int = 0
    result: object = None
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


# ----------------------------------------------------------------------------- job mix
def grid_for(lattice: str, a: float, ecut: float) -> int:
    """Smallest supported N with N >= 4 max|m| (the density sphere of the basis)."""
    from . import pwk, synth
    A = synth.fcc_lattice(a) if lattice == "fcc" else synth.sc_lattice(a)
    mmax = max(int(math.floor(math.sqrt(ecut) * np.linalg.norm(A[i]) / (2 * math.pi))) + 1
               for i in range(3))
    for N in (12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40, 45, 48):
        if N >= 4 * mmax and pwk.supported_grid(N):
            return N
    return 48


def random_mix(n_jobs: int, rate_hz: float, seed: int = 5, max_nk: int = 64, max_nb: int = 16,
               ecut_range=(25.0, 40.0)) -> List[Job]:
    """Poisson arrivals (mean rate rate_hz) of 60% H|psi>, 25% Davidson, 15% Sternheimer jobs
    on fcc / simple-cubic cells with 1, 2 or 4 atoms, cut-offs in 5 Ry steps, seeded."""
    r = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += r.exponential(1.0 / rate_hz)
        u = r.random()
        kind = "hpsi" if u < 0.60 else ("davidson" if u < 0.85 else "sternheimer")
        lattice = "fcc" if r.random() < 0.5 else "sc"
        nat = 1 if lattice == "fcc" else int(r.choice([1, 2, 4]))
        a = float(r.choice([6.5, 7.0, 7.5]))
        lo, hi = ecut_range
        ecut = float(r.choice(np.arange(lo, hi + 1e-9, 5.0)))
        mp = int(r.choice([1, 2, 3, 4]))
        mp = min(mp, int(round(max_nk ** (1 / 3))))
        nb = int(r.integers(4, max_nb + 1))
        if kind == "sternheimer":
            nb = min(nb, 8)
        cell = CellSpec(lattice, a, nat, round(ecut, 1), grid_for(lattice, a, ecut), mp,
                        int(r.integers(0, 2)))
        jobs.append(Job(j, kind, cell, nb, arrival=t))
    return jobs


# ----------------------------------------------------------------------------- footprints
def footprint_bytes(kind: str, nk: int, npw: int, nb: int, nkb: int, N: int) -> int:
    """Device bytes a job holds while it runs (plan tables + vectors + solver workspaces)."""
    c = 16
    plan = nk * npw * (8 + 4 + 4 + 2 * nkb * 12) + 3 * N ** 3 * 8
    if kind == "hpsi":
        work = 2 * nk * nb * npw * c
    elif kind == "davidson":
        mb = min(4 * nb, 160)
        work = nk * npw * c * (2 * mb + 4 * nb) + nk * mb * mb * c * 5
    else:
        work = 2 * plan + nk * nb * npw * c * 9
    return int(plan + work)


# ----------------------------------------------------------------------------- the server
class Server:
    """Admission by slots and HBM budget; one worker thread (and stream) per running job."""

    def __init__(self, execute: Callable[[List[Job], int], None], hbm_budget: int,
                 slots: int = 4, estimate: Optional[Callable[[Job], int]] = None,
                 coalesce: bool = True):
        self.execute = execute          # execute(jobs, slot) runs a group of jobs
        self.budget = int(hbm_budget)
        self.slots = slots
        self.estimate = estimate or (lambda j: j.footprint)
        self.coalesce = coalesce
        self.queue: collections.deque = collections.deque()
        self.lock = threading.Condition()
        self.in_use = 0
        self.free_slots = list(range(slots))
        self.running = 0
        self.peak_in_use = 0
        self.done: List[Job] = []
        self.t0 = 0.0
        self.max_group = 8

    def _group(self) -> Optional[List[Job]]:
        """Head-of-queue job, plus waiting H|psi> jobs on the same cell (coalesced)."""
        head = self.queue[0]
        group = [head]
        if self.coalesce and head.kind == "hpsi":
            for j in list(self.queue)[1:]:
                if len(group) >= self.max_group:
                    break
                if j.kind == "hpsi" and j.cell == head.cell and j.nb == head.nb:
                    group.append(j)
        return group

    def _admit_locked(self):
        started = []
        while self.queue and self.free_slots:
            group = self._group()
            need = sum(self.estimate(j) for j in group)
            if need > self.budget:
                # larger than the whole budget: run it alone when the GPU is idle
                if self.running > 0:
                    break
            elif self.in_use + need > self.budget:
                break
            for j in group:
                self.queue.remove(j)
            slot = self.free_slots.pop()
            self.in_use += need
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            self.running += 1
            started.append((group, slot, need))
        return started

    def _run(self, group: List[Job], slot: int, need: int):
        now = time.perf_counter() - self.t0
        for j in group:
            j.start = now
        try:
            self.execute(group, slot)
        except Exception as exc:   # a failed job is reported, the server goes on
            for j in group:
                j.error = f"{type(exc).__name__}: {exc}"
        end = time.perf_counter() - self.t0
        with self.lock:
            for j in group:
                j.finish = end
                self.done.append(j)
            self.in_use -= need
            self.free_slots.append(slot)
            self.running -= 1
            started = self._admit_locked()
            self.lock.notify_all()
        for g, s, n in started:
            threading.Thread(target=self._run, args=(g, s, n), daemon=True).start()

    def run(self, jobs: List[Job], realtime: bool = True) -> List[Job]:
        """Feed the jobs at their arrival times (or all at once if realtime is False) and wait
        for all of them."""
        self.t0 = time.perf_counter()
        pending = sorted(jobs, key=lambda j: j.arrival)
        for j in pending:
            if realtime:
                delay = j.arrival - (time.perf_counter() - self.t0)
                if delay > 0:
                    time.sleep(delay)
            else:
                j.arrival = time.perf_counter() - self.t0
            with self.lock:
                self.queue.append(j)
                started = self._admit_locked()
            for g, s, n in started:
                threading.Thread(target=self._run, args=(g, s, n), daemon=True).start()
        with self.lock:
            while len(self.done) < len(jobs):
                self.lock.wait(timeout=1.0)
        return sorted(self.done, key=lambda j: j.jid)


def latency_stats(jobs: List[Job]) -> Dict[str, float]:
    lat = np.array([j.latency for j in jobs if j.error is None])
    if len(lat) == 0:
        return {}
    span = max(j.finish for j in jobs) - min(j.arrival for j in jobs)
    return {"jobs": len(jobs), "failed": sum(j.error is not None for j in jobs),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "jobs_per_s": len(jobs) / span, "span_s": span}


# ----------------------------------------------------------------------------- GPU executor
class GpuExecutor:
    """Runs job groups through the library, one CUDA stream per slot, with a cache of device
    plans (LRU, bounded by the server's budget share `plan_cache_bytes`)."""

    def __init__(self, slots: int, plan_cache_bytes: int = 8 << 30, device: str = "cuda"):
        import torch
        self.torch = torch
        self.device = device
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.cache: "collections.OrderedDict" = collections.OrderedDict()
        self.cache_bytes = plan_cache_bytes
        self.cache_lock = threading.Lock()
        self.plan_users: Dict[object, int] = collections.Counter()

    # problems ---------------------------------------------------------------
    def prepare(self, jobs: List[Job]):
        """Build every job's host inputs before the clock starts (a request arrives with its
        inputs): the cell's problem (spheres, projectors, V, D) and the job's trial vectors."""
        self.inputs: Dict[int, tuple] = {}
        self.cells: Dict[tuple, object] = {}
        for j in jobs:
            if j.kind == "sternheimer":
                pk = self._cell_problem(j.cell, j.nb + 4, False)
                pq = self._cell_problem(j.cell, j.nb + 4, True)
                self.inputs[j.jid] = (pk, pq, self.problem_psi(pk, j.jid), self.problem_psi(pq, j.jid))
            else:
                pr = self._cell_problem(j.cell, j.nb, False)
                self.inputs[j.jid] = (pr, self.problem_psi(pr, j.jid))

    def _cell_problem(self, cell, nb, shift_q):
        key = (cell, nb, shift_q)
        if key not in self.cells:
            self.cells[key] = self.problem(cell, nb, shift_q)
        return self.cells[key]

    def problem(self, cell: CellSpec, nb: int, shift_q=False):
        from . import synth
        A = synth.fcc_lattice(cell.a) if cell.lattice == "fcc" else synth.sc_lattice(cell.a)
        base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])[:cell.nat]
        tau = cell.a * base
        B = synth.reciprocal_rows(A)
        k = synth.mp_grid(B, (cell.mp,) * 3)
        if shift_q:
            k = k + 2 * np.pi / cell.a * np.array([0.25, 0.0, 0.0])
        return synth.build_problem(A, tau, (0, 1, 2), cell.N, cell.ecut, k, nb, 900 + cell.seed,
                                   with_psi=False)

    def plan(self, key, prob):
        from . import pwk
        with self.cache_lock:
            if key in self.cache:
                self.cache.move_to_end(key)
                self.plan_users[key] += 1
                return self.cache[key][0]
        p = pwk.plan_from_problem(prob, device=self.device)
        with self.cache_lock:
            if key in self.cache:                      # another worker made it meanwhile
                p.close()
                self.plan_users[key] += 1
                return self.cache[key][0]
            self.cache[key] = (p, p.device_bytes, threading.Lock())
            self.plan_users[key] += 1
            self._evict_locked()
        return p

    def solver_lock(self, key) -> threading.Lock:
        """The Davidson/CG workspaces live in the plan: one solver call per plan at a time."""
        with self.cache_lock:
            return self.cache[key][2]

    def release(self, key):
        with self.cache_lock:
            self.plan_users[key] -= 1
            self._evict_locked()

    def _evict_locked(self):
        total = sum(v[1] for v in self.cache.values())
        for key in list(self.cache.keys()):
            if total <= self.cache_bytes:
                break
            if self.plan_users[key] > 0:
                continue
            p, b, _ = self.cache.pop(key)
            p.close()
            total -= b

    # execution ---------------------------------------------------------------
    def __call__(self, group: List[Job], slot: int):
        torch = self.torch
        from . import pwk
        stream = self.streams[slot]
        job = group[0]
        with torch.cuda.stream(stream):
            if job.kind == "hpsi":
                self._hpsi(group, stream)
            elif job.kind == "davidson":
                self._davidson(job, stream)
            else:
                self._sternheimer(job, stream)
        stream.synchronize()

    def _hpsi(self, group, stream):
        torch = self.torch
        from . import pwk
        cell, nb = group[0].cell, group[0].nb
        prob = self.inputs[group[0].jid][0]
        key = ("k", cell)
        plan = self.plan(key, prob)
        try:
            # one work list over every band of every job of the group
            nj = len(group)
            psi = np.concatenate([self.inputs[j.jid][1] for j in group], axis=1)
            x = torch.from_numpy(psi).to(self.device, non_blocking=True)
            y = torch.empty_like(x)
            items = np.array([[k, v, v] for k in range(prob.nk) for v in range(nj * nb)], np.int32)
            pwk.hpsi_items(plan, pwk.PWK_FP64, x, y, torch.from_numpy(items).to(self.device),
                           nj * nb, stream)
            out = y.cpu().numpy()
            for i, j in enumerate(group):
                j.result = out[:, i * nb:(i + 1) * nb]
        finally:
            self.release(key)

    @staticmethod
    def problem_psi(prob, jid: int):
        """Job-specific trial vectors (seeded by the job id), [nk][nb][npw_max]."""
        from . import synth
        r = np.random.default_rng(424242 + jid)
        return np.stack([synth.random_orthonormal(r, int(prob.npw[k]), prob.npw_max, prob.nb)
                         for k in range(prob.nk)])

    def _davidson(self, job, stream):
        torch = self.torch
        from . import pwk
        prob, psi0 = self.inputs[job.jid]
        key = ("k", job.cell)
        plan = self.plan(key, prob)
        try:
            psi = torch.from_numpy(psi0).to(self.device)
            eig = torch.zeros((prob.nk, job.nb), dtype=torch.float64, device=self.device)
            with self.solver_lock(key):
                rc, iters, notc, napply = pwk.davidson_batched(plan, pwk.PWK_FP32_C128, psi, eig,
                                                               job.nb, 1e-10, 1e-5, 200, 0, stream)
            job.result = eig.cpu().numpy()
        finally:
            self.release(key)

    def _sternheimer(self, job, stream):
        torch = self.torch
        from . import pwk, synth
        nocc = job.nb
        pk, pq, psik0, psiq0 = self.inputs[job.jid]
        kk, kq = ("k", job.cell), ("q", job.cell)
        plan_k = self.plan(kk, pk)
        plan_q = self.plan(kq, pq)
        try:
            def dav(plan, prob, key, psi0):
                psi = torch.from_numpy(psi0).to(self.device)
                eig = torch.zeros((prob.nk, prob.nb), dtype=torch.float64, device=self.device)
                with self.solver_lock(key):
                    pwk.davidson_batched(plan, pwk.PWK_FP64, psi, eig, prob.nb, 1e-10, 1e-6, 300,
                                         0, stream)
                return psi[:, :nocc].contiguous(), eig
            psi_k, ek = dav(plan_k, pk, kk, psik0)
            psi_q, eq = dav(plan_q, pq, kq, psiq0)
            e_occ = torch.cat([ek[:, :nocc], eq[:, :nocc]], 1)
            alpha = torch.clamp(2 * (e_occ.max(1).values - e_occ.min(1).values), min=0.01).contiguous()
            A = synth.fcc_lattice(job.cell.a) if job.cell.lattice == "fcc" else synth.sc_lattice(job.cell.a)
            dv = torch.from_numpy(synth.dv_grid(np.random.default_rng(77 + job.cell.seed),
                                                synth.reciprocal_rows(A), job.cell.N,
                                                job.cell.ecut)).to(self.device)
            dpsi = torch.zeros((pq.nk, nocc, pq.npw_max), dtype=torch.complex128, device=self.device)
            with self.solver_lock(kq):
                rc, iters, resid = pwk.sternheimer_cg_batched(plan_q, plan_k, pwk.PWK_FP32_C128,
                                                              psi_k, ek[:, :nocc].contiguous(),
                                                              psi_q, nocc, alpha, dv, dpsi, 1e-10,
                                                              500, stream)
            # the valence states go with the result: within a degenerate level they are fixed only
            # up to a unitary mix, which carries over to dpsi (sum_n |dpsi_n><psi_n| is unique)
            job.result = (dpsi.cpu().numpy(), resid, psi_k.cpu().numpy())
        finally:
            self.release(kk)
            self.release(kq)


def estimate_for(job: Job) -> int:
    """Footprint of a job from its cell (the npw of the sphere is estimated from the cut-off
    volume)."""
    c = job.cell
    vol = (c.a ** 3) / (4.0 if c.lattice == "fcc" else 1.0)
    npw = int(vol * (c.ecut ** 1.5) / (6 * math.pi ** 2) * 1.15) + 16
    nk = c.mp ** 3
    nkb = 9 * c.nat
    mult = 2 if job.kind == "sternheimer" else 1
    return mult * footprint_bytes(job.kind, nk, npw, job.nb + (4 if job.kind == "sternheimer" else 0),
                                  nkb, c.N)
