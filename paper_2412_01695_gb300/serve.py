"""Serving loop: H|psi>, Davidson and Sternheimer jobs on one GPU, admitted as they arrive.

A job names a synthetic cell (lattice, atoms, cut-off, grid), a set of k-points and an
operation.  The server
  * admits a queued job when a slot is free and its estimated device footprint fits in the
    HBM budget next to the jobs already running (the analogue of the paper's memgpu: a block
    of k-points is loaded only when the GPU memory allows it, Sec. 3 / Sec. 6.1);
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
    precision: str = "fp64"   # H|psi> jobs: "fp64" or "mixed" (FP32 arithmetic, complex128 io)
    start: float = math.nan
    finish: float = math.nan
    footprint: int = 0
    result: object = None
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival

    def fresh(self) -> "Job":
        """The same request, not yet run."""
        return Job(self.jid, self.kind, self.cell, self.nb, arrival=self.arrival, precision=self.precision)


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


# fcc cells take one or two atoms (the second at a(1/4, 1/4, 1/4)); simple-cubic cells take up
# to eight atoms on the sites of the half-lattice {0, 1/2}^3, in this order
SC_SITES = np.array([[0, 0, 0], [.5, .5, .5], [0, .5, .5], [.5, 0, .5], [.5, .5, 0], [.5, 0, 0],
                     [0, .5, 0], [0, 0, .5]])
FCC_SITES = np.array([[0, 0, 0], [.25, .25, .25]])


def config5_cells(n_cells: int, seed: int = 5, ecut_range=(25.0, 60.0), max_nk: int = 1728,
                  max_N: int = 36):
    """A pool of cells over the serving workload's ranges: fcc (1-2 atoms) or simple-cubic (1-8
    atoms) cells, cut-offs 25-60 Ry in 5 Ry steps, Monkhorst-Pack grids q^3 with q log-uniform
    in [1, 12] (1 to 1728 k-points).  The lattice constant is drawn so that the cell's FFT grid
    (N >= 4 max|m|) is at most max_N (36: the largest grid whose FP64 transforms fit in one
    CTA's shared memory, which the FP64 baseline and solvers need); draws outside are
    repeated."""
    from . import pwk
    r = np.random.default_rng(seed)
    qmax = max(1, int(round(max_nk ** (1 / 3))))
    # the largest k-set of the range on a one-atom fcc cell and the largest cell of the range
    # (eight atoms, simple cubic, 25 Ry), then random cells
    cells = [CellSpec("fcc", 7.5, 1, 30.0, grid_for("fcc", 7.5, 30.0), qmax, int(r.integers(0, 1000))),
             CellSpec("sc", 9.6, 8, 25.0, grid_for("sc", 9.6, 25.0), 2, int(r.integers(0, 1000)))]
    while len(cells) < n_cells:
        lattice = "fcc" if r.random() < 0.4 else "sc"
        nat = int(r.integers(1, 3)) if lattice == "fcc" else int(r.integers(1, 9))
        ecut = float(r.choice(np.arange(ecut_range[0], ecut_range[1] + 1e-9, 5.0)))
        # about 100-130 bohr^3 per atom
        vol = nat * float(r.uniform(100.0, 130.0))
        a = (4.0 * vol) ** (1 / 3) if lattice == "fcc" else vol ** (1 / 3)
        N = grid_for(lattice, a, ecut)
        if N > max_N or not pwk.supported_grid(N) or N < 4 * _mmax(lattice, a, ecut):
            continue
        q = int(min(qmax, max(1, round(math.exp(r.uniform(0.0, math.log(qmax + 0.49)))))))
        cells.append(CellSpec(lattice, round(a, 4), nat, ecut, N, q, int(r.integers(0, 1000))))
    return cells


def _mmax(lattice: str, a: float, ecut: float) -> int:
    from . import synth
    A = synth.fcc_lattice(a) if lattice == "fcc" else synth.sc_lattice(a)
    return max(int(math.floor(math.sqrt(ecut) * np.linalg.norm(A[i]) / (2 * math.pi))) + 1 for i in range(3))


def npw_estimate(c: CellSpec) -> int:
    vol = (c.a ** 3) / (4.0 if c.lattice == "fcc" else 1.0)
    return int(vol * (c.ecut ** 1.5) / (6 * math.pi ** 2))


def config5_mix(n_jobs: int, rate_hz: float, seed: int = 7, n_cells: int = 10,
                max_nk: int = 1728, solver_max_nk: int = 512, st_max_bands: int = 16) -> List[Job]:
    """Poisson arrivals (mean rate rate_hz) of 60% H|psi>, 25% Davidson, 15% Sternheimer jobs
    on a pool of n_cells cells (config5_cells): each job picks a cell and 4-60 bands (at most
    a quarter of the cell's plane waves, which the Davidson's 4 nb basis needs).  H|psi> jobs
    run in the mixed path and take any cell (1 to max_nk k-points); the solver jobs take cells
    with at most solver_max_nk k-points, and Sternheimer jobs (which also solve for the valence
    states of k and k+q) at most st_max_bands occupied bands."""
    cells = config5_cells(n_cells, seed=seed + 1, max_nk=max_nk)
    r = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += r.exponential(1.0 / rate_hz)
        u = r.random()
        kind = "hpsi" if u < 0.60 else ("davidson" if u < 0.85 else "sternheimer")
        pool = cells if kind == "hpsi" else [c for c in cells if c.mp ** 3 <= solver_max_nk] or cells[1:2]
        cell = pool[int(r.integers(0, len(pool)))]
        nb = int(r.integers(4, 61))
        nb = max(4, min(nb, npw_estimate(cell) // 4 - 1))
        if kind == "sternheimer":
            nb = min(nb, st_max_bands)
        jobs.append(Job(j, kind, cell, nb, arrival=t, precision="mixed" if kind == "hpsi" else "fp64"))
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
                if j.kind == "hpsi" and j.cell == head.cell and j.precision == head.precision:
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

    def __init__(self, slots: int, plan_cache_bytes: int = 8 << 30, device: str = "cuda",
                 per_k: bool = False):
        import torch
        self.torch = torch
        self.device = device
        # per_k: the plain baseline: H|psi> jobs in FP64 with one launch set per k-point, every
        # solver in FP64
        self.per_k = per_k
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
        base = (FCC_SITES if cell.lattice == "fcc" else SC_SITES)[:cell.nat]
        tau = cell.a * base
        B = synth.reciprocal_rows(A)
        k = synth.mp_grid(B, (cell.mp,) * 3)
        if shift_q:
            k = k + 2 * np.pi / cell.a * np.array([0.25, 0.0, 0.0])
        return synth.build_problem(A, tau, (0, 1, 2), cell.N, cell.ecut, k, nb, 900 + cell.seed,
                                   with_psi=False)

    def warm(self, jobs: List[Job]):
        """Device-resident state before the clock starts (a service loads its cells once): the
        plan of every cell the jobs name (k, and k+q for Sternheimer jobs), with its launch
        shapes tuned, and the solver workspaces at the largest size the jobs need (one
        one-iteration solve per plan), so no job pays for plan creation, autotuning or a
        workspace allocation (which would synchronise the device under the other jobs)."""
        torch = self.torch
        from . import pwk
        dav_nb: Dict[object, int] = {}
        cg_nb: Dict[object, int] = {}
        for j in jobs:
            if j.kind == "sternheimer":
                pk, pq, _, _ = self.inputs[j.jid]
                self.plan(("k", j.cell), pk)
                self.release(("k", j.cell))
                self.plan(("q", j.cell), pq)
                self.release(("q", j.cell))
                for key, pr in ((("k", j.cell), pk), (("q", j.cell), pq)):
                    dav_nb[key] = max(dav_nb.get(key, 0), pr.nb)
                cg_nb[("q", j.cell)] = max(cg_nb.get(("q", j.cell), 0), j.nb)
            else:
                self.plan(("k", j.cell), self.inputs[j.jid][0])
                self.release(("k", j.cell))
                if j.kind == "davidson":
                    dav_nb[("k", j.cell)] = max(dav_nb.get(("k", j.cell), 0), j.nb)
        for key, nocc in cg_nb.items():   # the CG workspace and the k -> k+q maps
            pq_plan = self.cache[key][0]
            pk_plan = self.cache[("k", key[1])][0]
            z = lambda *sh: torch.zeros(sh, dtype=torch.complex128, device=self.device)  # noqa: E731
            pk_ = z(pk_plan.nk, nocc, pk_plan.npw_max)
            pq_ = z(pq_plan.nk, nocc, pq_plan.npw_max)
            pwk.sternheimer_cg_batched(pq_plan, pk_plan, pwk.PWK_FP32_C128, pk_,
                                       torch.zeros((pk_plan.nk, nocc), dtype=torch.float64, device=self.device),
                                       pq_, nocc, torch.ones(pq_plan.nk, dtype=torch.float64, device=self.device),
                                       z(pq_plan.N, pq_plan.N, pq_plan.N), z(pq_plan.nk, nocc, pq_plan.npw_max),
                                       1e-10, 1)
        for key, nb in dav_nb.items():
            p = self.cache[key][0]
            psi = torch.zeros((p.nk, nb, p.npw_max), dtype=torch.complex128, device=self.device)
            psi[:, :, 0] = 1.0
            for b in range(nb):
                psi[:, b, b] = 1.0
            eig = torch.zeros((p.nk, nb), dtype=torch.float64, device=self.device)
            for mode in (pwk.PWK_FP32_C128, pwk.PWK_FP64):
                try:
                    pwk.davidson_batched(p, mode, psi.clone(), eig, nb, 1e-3, 0.0, 1, 0)
                except pwk.PwkError:
                    pass
        torch.cuda.synchronize()

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
        cell = group[0].cell
        prob = self.inputs[group[0].jid][0]
        key = ("k", cell)
        plan = self.plan(key, prob)
        try:
            # one work list over every band of every job of the group
            nbs = [j.nb for j in group]
            nv = sum(nbs)
            psi = np.concatenate([self.inputs[j.jid][1] for j in group], axis=1)
            x = torch.from_numpy(psi).to(self.device, non_blocking=True)
            y = torch.empty_like(x)
            prec = pwk.PWK_FP32_C128 if (group[0].precision == "mixed" and not self.per_k) else pwk.PWK_FP64
            if self.per_k:   # the plain baseline: one launch set per k-point
                for k in range(prob.nk):
                    it = torch.tensor([[k, v, v] for v in range(nv)], dtype=torch.int32, device=self.device)
                    pwk.hpsi_items(plan, prec, x, y, it, nv, stream)
            else:
                items = np.array([[k, v, v] for k in range(prob.nk) for v in range(nv)], np.int32)
                pwk.hpsi_items(plan, prec, x, y, torch.from_numpy(items).to(self.device), nv, stream)
            out = y.cpu().numpy()
            o = 0
            for j, nbj in zip(group, nbs):
                j.result = out[:, o:o + nbj]
                o += nbj
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
            mode = pwk.PWK_FP64 if self.per_k else pwk.PWK_FP32_C128
            with self.solver_lock(key):
                rc, iters, notc, napply = pwk.davidson_batched(plan, mode, psi, eig,
                                                               job.nb, 1e-10, 1e-5, 300, 0, stream)
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
            dmode = pwk.PWK_FP64 if self.per_k else pwk.PWK_FP32_C128

            def dav(plan, prob, key, psi0):
                psi = torch.from_numpy(psi0).to(self.device)
                eig = torch.zeros((prob.nk, prob.nb), dtype=torch.float64, device=self.device)
                with self.solver_lock(key):
                    pwk.davidson_batched(plan, dmode, psi, eig, prob.nb, 1e-10, 1e-6, 300,
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
            cmode = pwk.PWK_FP64 if self.per_k else pwk.PWK_FP32_C128
            with self.solver_lock(kq):
                rc, iters, resid = pwk.sternheimer_cg_batched(plan_q, plan_k, cmode,
                                                              psi_k, ek[:, :nocc].contiguous(),
                                                              psi_q, nocc, alpha, dv, dpsi, 1e-10,
                                                              500, stream)
            # the valence states go with the result: within a degenerate level they are fixed only
            # up to a unitary mix, which carries over to dpsi (sum_n |dpsi_n><psi_n| is unique);
            # eps_k, psi_{k+q}, alpha and dv let a checker rebuild the system
            job.result = (dpsi.cpu().numpy(), resid, psi_k.cpu().numpy(), ek[:, :nocc].cpu().numpy(),
                          psi_q.cpu().numpy(), alpha.cpu().numpy(), dv.cpu().numpy(), eq.cpu().numpy())
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
