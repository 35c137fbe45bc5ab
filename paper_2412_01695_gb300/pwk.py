"""Thin ctypes binding of libpwk.so (include/pwk.h): argument marshalling only.

Every function here forwards to the C ABI with device pointers taken from torch tensors
(torch is used for device memory and streams only).  There is no CPU fallback: if the
library is missing or no CUDA device is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpwk.so")

PWK_FP64, PWK_FP32, PWK_FP32_C128 = 0, 1, 2
PRECISIONS = {"fp64": PWK_FP64, "fp32": PWK_FP32, "fp32_c128": PWK_FP32_C128}
PWK_FLAG_ITEM_SKIPPED, PWK_FLAG_WAIT_TIMEOUT = 1, 2

# every symbol declared in include/pwk.h
EXPORTS = ("pwk_plan_create", "pwk_plan_destroy", "pwk_plan_device_bytes",
           "pwk_plan_launch_shape", "pwk_plan_set_launch_shape", "pwk_plan_set_projector_path",
           "pwk_plan_errors", "pwk_plan_set_wait_limit", "pwk_plan_projector_fused",
           "pwk_plan_projector_choice",
           "pwk_supported_grid",
           "pwk_hpsi_batched", "pwk_hpsi_batched_host", "pwk_hpsi_items", "pwk_hpsi_multi",
           "pwk_plan_set_overlap",
           "pwk_plan_has_overlap",
           "pwk_hspsi_batched", "pwk_hspsi_items", "pwk_drho_batched", "pwk_davidson_batched",
           "pwk_sternheimer_cg_batched", "pwk_eigh_batched", "pwk_eigh_batched_noalloc",
           "pwk_measure_fma_peak", "pwk_launch_count", "pwk_plan_set_solver_timing", "pwk_plan_solver_stats",
           "pwk_strerror", "pwk_last_error_detail", "pwk_version")

_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t


def load(path: str = LIB_PATH):
    """Load libpwk.so and declare its signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2412_01695_gb300.build")
    L = ctypes.CDLL(path)
    sig = {
        "pwk_plan_create": (_I, [ctypes.POINTER(_P), _P, _I, _I, _I, _I, _P, _P, _I, _P, _I, _P, _P,
                                 _P, _SZ]),
        "pwk_plan_destroy": (None, [_P]),
        "pwk_plan_device_bytes": (_SZ, [_P]),
        "pwk_plan_launch_shape": (_I, [_P, _I, _P, _P, _P, _P]),
        "pwk_plan_set_launch_shape": (_I, [_P, _I, _I, _I, _I]),
        "pwk_plan_set_projector_path": (_I, [_P, _I]),
        "pwk_plan_projector_fused": (_I, [_P, _I]),
        "pwk_plan_projector_choice": (_I, [_P, _I]),
        "pwk_plan_errors": (_I, [_P, ctypes.POINTER(_I), _I]),
        "pwk_plan_set_wait_limit": (_I, [_P, ctypes.c_longlong]),
        "pwk_supported_grid": (_I, [_I]),
        "pwk_hpsi_batched": (_I, [_P, _I, _P, _P, _I, _P]),
        "pwk_hpsi_batched_host": (_I, [_P, _I, _P, _P, _P, _P, _I, _I, _P]),
        "pwk_hpsi_items": (_I, [_P, _I, _P, _P, _P, _I, _I, _P]),
        "pwk_hpsi_multi": (_I, [_I, _P, _I, _P, _P, _P, _P, _I, _P]),
        "pwk_plan_set_overlap": (_I, [_P, _P]),
        "pwk_plan_has_overlap": (_I, [_P]),
        "pwk_hspsi_batched": (_I, [_P, _I, _P, _P, _P, _I, _P]),
        "pwk_hspsi_items": (_I, [_P, _I, _P, _P, _P, _P, _I, _I, _P]),
        "pwk_drho_batched": (_I, [_P, _P, _I, _P, _P, _P, _I, _P, _P, _P]),
        "pwk_davidson_batched": (_I, [_P, _I, _P, _P, _I, _D, _D, _I, _I, _P, _P, _P, _P]),
        "pwk_sternheimer_cg_batched": (_I, [_P, _P, _I, _P, _P, _P, _I, _P, _P, _P, _D, _I, _P,
                                            _P, _P]),
        "pwk_eigh_batched": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P]),
        "pwk_eigh_batched_noalloc": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P]),
        "pwk_measure_fma_peak": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(_I), _P]),
        "pwk_launch_count": (ctypes.c_longlong, []),
        "pwk_plan_set_solver_timing": (_I, [_P, _I]),
        "pwk_plan_solver_stats": (_I, [_P, ctypes.POINTER(_D)]),
        "pwk_strerror": (ctypes.c_char_p, [_I]),
        "pwk_last_error_detail": (ctypes.c_char_p, []),
        "pwk_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class PwkError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = load()
        super().__init__(f"{where}: {L.pwk_strerror(code).decode()} ({code}): "
                         f"{L.pwk_last_error_detail().decode()}")
        self.code = code


def _check(code: int, where: str) -> int:
    if code < 0:
        raise PwkError(code, where)
    return code


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Plan:
    """Owns a pwk_plan*; keeps the caller-owned device arrays (beta, V) alive."""

    def __init__(self, handle, keep, geom=(0, 0, 0)):
        self.handle = handle
        self._keep = keep
        self.nk, self.npw_max, self.N = geom

    @property
    def device_bytes(self) -> int:
        return int(load().pwk_plan_device_bytes(self.handle))

    def launch_shape(self, precision: int):
        """(kernel kind, threads per CTA, l3 chunk, shared memory bytes) of a precision."""
        kd, t, l, sm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(load().pwk_plan_launch_shape(self.handle, precision, ctypes.byref(kd), ctypes.byref(t),
                                            ctypes.byref(l), ctypes.byref(sm)),
               "pwk_plan_launch_shape")
        return kd.value, t.value, l.value, sm.value

    def set_launch_shape(self, precision: int, kind: int, threads: int, l3_chunk: int):
        _check(load().pwk_plan_set_launch_shape(self.handle, precision, kind, threads, l3_chunk),
               "pwk_plan_set_launch_shape")

    def set_projector_path(self, path: int) -> None:
        """pwk_plan_set_projector_path: 0 automatic (default), 1 tensor-core projections,
        2 separate CUDA-core kernels, 3 fused into the local kernel."""
        _check(load().pwk_plan_set_projector_path(self.handle, path), "pwk_plan_set_projector_path")

    def projector_fused(self, precision: int) -> bool:
        """pwk_plan_projector_fused: whether H|psi> of this precision runs the projector terms
        inside the local kernel."""
        return load().pwk_plan_projector_fused(self.handle, precision) == 1

    def projector_choice(self, precision: int) -> int:
        """pwk_plan_projector_choice: the projector path whole-k-point H|psi> calls of this
        precision take (3 fused, 1 tensor cores, 2 CUDA cores, 0 no projectors)."""
        return int(load().pwk_plan_projector_choice(self.handle, precision))

    def errors(self, clear: bool = True) -> int:
        """pwk_plan_errors: the device-side flags (PWK_FLAG_*) recorded since the last clear."""
        v = _I()
        _check(load().pwk_plan_errors(self.handle, ctypes.byref(v), 1 if clear else 0), "pwk_plan_errors")
        return v.value

    def set_wait_limit(self, polls: int) -> None:
        """pwk_plan_set_wait_limit: bound on the polls of every device-side wait (diagnostic)."""
        _check(load().pwk_plan_set_wait_limit(self.handle, polls), "pwk_plan_set_wait_limit")

    def set_overlap(self, q) -> None:
        """pwk_plan_set_overlap: q host float64 [nkb][nkb] symmetric, or None (S = 1)."""
        if q is None:
            _check(load().pwk_plan_set_overlap(self.handle, None), "pwk_plan_set_overlap")
            return
        q = np.ascontiguousarray(q, np.float64)
        _check(load().pwk_plan_set_overlap(self.handle, _np_ptr(q)), "pwk_plan_set_overlap")

    def set_solver_timing(self, on: bool) -> None:
        """pwk_plan_set_solver_timing: record the device time of the solvers' phases."""
        _check(load().pwk_plan_set_solver_timing(self.handle, 1 if on else 0), "pwk_plan_set_solver_timing")

    def solver_stats(self) -> dict:
        """pwk_plan_solver_stats of the last solver call on this plan."""
        v = (_D * 5)()
        _check(load().pwk_plan_solver_stats(self.handle, v), "pwk_plan_solver_stats")
        return {"h_ms": v[0], "rr_ms": v[1], "total_ms": v[2], "rr_fp64_flops": v[3], "other_ms": v[4]}

    @property
    def has_overlap(self) -> bool:
        return bool(load().pwk_plan_has_overlap(self.handle))

    def close(self):
        if self.handle:
            load().pwk_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_create(A, N, kcart, npw, miller, beta_dev, D, vloc_dev, hbm_budget: int = 0) -> Plan:
    """pwk_plan_create.  A, kcart, npw, miller, D host numpy; beta_dev (complex128) and
    vloc_dev (float64) torch CUDA tensors."""
    L = load()
    A = np.ascontiguousarray(A, np.float64)
    kcart = np.ascontiguousarray(kcart, np.float64)
    npw = np.ascontiguousarray(npw, np.int32)
    miller = np.ascontiguousarray(miller, np.int32)
    nk, npw_max = miller.shape[0], miller.shape[1]
    nkb = 0 if beta_dev is None else int(beta_dev.shape[1])
    D = np.ascontiguousarray(D if D is not None else np.zeros((0, 0)), np.float64)
    h = ctypes.c_void_p()
    geom = (nk, npw_max, int(N))
    rc = L.pwk_plan_create(ctypes.byref(h), _np_ptr(A), N, N, N, nk, _np_ptr(kcart), _np_ptr(npw),
                           npw_max, _np_ptr(miller), nkb, _ptr(beta_dev) if nkb else None,
                           _np_ptr(D) if nkb else None, _ptr(vloc_dev), hbm_budget)
    _check(rc, "pwk_plan_create")
    return Plan(h, (beta_dev, vloc_dev), geom)


def plan_from_problem(prob, device="cuda", hbm_budget: int = 0) -> Plan:
    """Upload a synth.Problem's beta and V and create its plan."""
    import torch
    beta = torch.from_numpy(np.ascontiguousarray(prob.beta)).to(device) if prob.nkb else None
    v = torch.from_numpy(np.ascontiguousarray(prob.V_r)).to(device)
    return plan_create(prob.A, prob.N, prob.kpts, prob.npw, prob.miller, beta, prob.D, v,
                       hbm_budget)


def _need(t, shape, dtype, name):
    """Shape/dtype check of a tensor handed to the library (plain pointers cannot be checked
    on the C side, so a wrong size here would read or write outside the tensor)."""
    if tuple(t.shape) != tuple(shape) or t.dtype != dtype:
        raise ValueError(f"{name}: expected shape {tuple(shape)} {dtype}, got {tuple(t.shape)} {t.dtype}")


def hpsi_batched(plan: Plan, precision: int, psi, hpsi, nb: int, stream=None) -> None:
    import torch
    dt = torch.complex64 if precision == PWK_FP32 else torch.complex128
    shape = (plan.nk, nb, plan.npw_max)
    _need(psi, shape, dt, "psi")
    _need(hpsi, shape, dt, "hpsi")
    _check(load().pwk_hpsi_batched(plan.handle, precision, _ptr(psi), _ptr(hpsi), nb,
                                   _stream(stream)), "pwk_hpsi_batched")


def hpsi_batched_host(plan: Plan, precision: int, h_psi, h_hpsi, d_psi, d_hpsi, nb: int,
                      nchunk: int, stream=None) -> None:
    """H|psi> with the vectors in (page-locked) host tensors; d_psi, d_hpsi are device work
    buffers of the same shape.  Copies in, applications and copies out of nchunk groups of
    k-points overlap; the result is in h_hpsi once `stream` has completed."""
    import torch
    dt = torch.complex64 if precision == PWK_FP32 else torch.complex128
    shape = (plan.nk, nb, plan.npw_max)
    for t, name in ((h_psi, "h_psi"), (h_hpsi, "h_hpsi")):
        if t.is_cuda or tuple(t.shape) != shape or t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous host tensor {shape} of {dt}")
    _need(d_psi, shape, dt, "d_psi")
    _need(d_hpsi, shape, dt, "d_hpsi")
    _check(load().pwk_hpsi_batched_host(plan.handle, precision, ctypes.c_void_p(h_psi.data_ptr()),
                                        ctypes.c_void_p(h_hpsi.data_ptr()), _ptr(d_psi), _ptr(d_hpsi),
                                        nb, nchunk, _stream(stream)), "pwk_hpsi_batched_host")


def hpsi_items(plan: Plan, precision: int, psi, hpsi, items, nvec_per_k: int, stream=None):
    import torch
    dt = torch.complex64 if precision == PWK_FP32 else torch.complex128
    shape = (plan.nk, nvec_per_k, plan.npw_max)
    _need(psi, shape, dt, "psi")
    _need(hpsi, shape, dt, "hpsi")
    n = 0 if items is None else int(items.shape[0])
    if n:
        _need(items, (n, 3), torch.int32, "items")
    _check(load().pwk_hpsi_items(plan.handle, precision, _ptr(psi), _ptr(hpsi),
                                 _ptr(items) if n else None, n, nvec_per_k, _stream(stream)),
           "pwk_hpsi_items")


def hpsi_multi(plans, precision: int, psis, hpsis, items, stream=None):
    """pwk_hpsi_multi: one work list over several plans of one grid.  plans, psis, hpsis are
    lists (one entry per plan; psis[i] [nk_i][nvec_i][npw_max_i]); items a device int32 tensor
    [n][4] of (plan, k, in_slot, out_slot)."""
    import torch
    npl = len(plans)
    if not (len(psis) == len(hpsis) == npl) or npl < 1:
        raise ValueError("one psi and one hpsi per plan")
    dt = torch.complex64 if precision == PWK_FP32 else torch.complex128
    nvec = []
    for p, x, y in zip(plans, psis, hpsis):
        if x.dim() != 3:
            raise ValueError("psi must be [nk][nvec][npw_max]")
        shape = (p.nk, int(x.shape[1]), p.npw_max)
        _need(x, shape, dt, "psi")
        _need(y, shape, dt, "hpsi")
        nvec.append(int(x.shape[1]))
    n = 0 if items is None else int(items.shape[0])
    if n:
        _need(items, (n, 4), torch.int32, "items")
    ph = (ctypes.c_void_p * npl)(*[p.handle for p in plans])
    xs = (ctypes.c_void_p * npl)(*[_ptr(x) for x in psis])
    ys = (ctypes.c_void_p * npl)(*[_ptr(y) for y in hpsis])
    nv = (ctypes.c_int * npl)(*nvec)
    _check(load().pwk_hpsi_multi(npl, ph, precision, xs, ys, nv, _ptr(items) if n else None, n,
                                 _stream(stream)), "pwk_hpsi_multi")


def hspsi_batched(plan: Plan, precision: int, psi, hpsi, spsi, nb: int, stream=None) -> None:
    import torch
    dt = torch.complex64 if precision == PWK_FP32 else torch.complex128
    shape = (plan.nk, nb, plan.npw_max)
    for t, name in ((psi, "psi"), (hpsi, "hpsi"), (spsi, "spsi")):
        _need(t, shape, dt, name)
    _check(load().pwk_hspsi_batched(plan.handle, precision, _ptr(psi), _ptr(hpsi), _ptr(spsi), nb,
                                    _stream(stream)), "pwk_hspsi_batched")


def hspsi_items(plan: Plan, precision: int, psi, hpsi, spsi, items, nvec_per_k: int, stream=None):
    import torch
    dt = torch.complex64 if precision == PWK_FP32 else torch.complex128
    shape = (plan.nk, nvec_per_k, plan.npw_max)
    for t, name in ((psi, "psi"), (hpsi, "hpsi"), (spsi, "spsi")):
        _need(t, shape, dt, name)
    n = 0 if items is None else int(items.shape[0])
    if n:
        _need(items, (n, 3), torch.int32, "items")
    _check(load().pwk_hspsi_items(plan.handle, precision, _ptr(psi), _ptr(hpsi), _ptr(spsi),
                                  _ptr(items) if n else None, n, nvec_per_k, _stream(stream)),
           "pwk_hspsi_items")


def drho_batched(plan_kq: Plan, plan_k: Plan, precision: int, psi_k, psi_kq, dpsi, nocc: int,
                 weights, drho, stream=None) -> None:
    """pwk_drho_batched: drho (complex128 [N, N, N]) from u_k, the k+q valence states and du."""
    import torch
    nk = plan_kq.nk
    _need(psi_k, (nk, nocc, plan_k.npw_max), torch.complex128, "psi_k")
    _need(psi_kq, (nk, nocc, plan_kq.npw_max), torch.complex128, "psi_kq")
    _need(dpsi, (nk, nocc, plan_kq.npw_max), torch.complex128, "dpsi")
    _need(weights, (nk,), torch.float64, "weights")
    _need(drho, (plan_kq.N,) * 3, torch.complex128, "drho")
    _check(load().pwk_drho_batched(plan_kq.handle, plan_k.handle, precision, _ptr(psi_k), _ptr(psi_kq),
                                   _ptr(dpsi), nocc, _ptr(weights), _ptr(drho), _stream(stream)),
           "pwk_drho_batched")


def davidson_batched(plan: Plan, mode: int, psi, eig, nb: int, eth: float, res_tol: float = 0.0,
                     max_iter: int = 100, max_basis: int = 0, stream=None):
    """Returns (unconverged count, iters[nk], notconv[nk], napply[2])."""
    import torch
    L = load()
    nk = plan.nk
    _need(psi, (nk, nb, plan.npw_max), torch.complex128, "psi")
    _need(eig, (nk, nb), torch.float64, "eig")
    iters = np.zeros(nk, np.int32)
    notc = np.zeros(nk, np.int32)
    napply = np.zeros(2, np.int64)
    rc = L.pwk_davidson_batched(plan.handle, mode, _ptr(psi), _ptr(eig), nb, eth, res_tol,
                                max_iter, max_basis, _np_ptr(iters), _np_ptr(notc),
                                _np_ptr(napply), _stream(stream))
    _check(rc, "pwk_davidson_batched")
    return rc, iters, notc, napply


def sternheimer_cg_batched(plan_kq: Plan, plan_k: Plan, mode: int, psi_k, eps_k, psi_kq,
                           nocc: int, alpha, dv, dpsi, tol: float, max_iter: int = 500,
                           stream=None):
    """Returns (count above tol, iters[nk*nocc], resid[nk*nocc])."""
    import torch
    L = load()
    nk = plan_kq.nk
    _need(psi_k, (nk, nocc, plan_k.npw_max), torch.complex128, "psi_k")
    _need(psi_kq, (nk, nocc, plan_kq.npw_max), torch.complex128, "psi_kq")
    _need(dpsi, (nk, nocc, plan_kq.npw_max), torch.complex128, "dpsi")
    _need(eps_k, (nk, nocc), torch.float64, "eps_k")
    _need(alpha, (nk,), torch.float64, "alpha")
    _need(dv, (plan_kq.N,) * 3, torch.complex128, "dv")
    iters = np.zeros(nk * nocc, np.int32)
    resid = np.zeros(nk * nocc, np.float64)
    rc = L.pwk_sternheimer_cg_batched(plan_kq.handle, plan_k.handle, mode, _ptr(psi_k),
                                      _ptr(eps_k), _ptr(psi_kq), nocc, _ptr(alpha), _ptr(dv),
                                      _ptr(dpsi), tol, max_iter, _np_ptr(iters), _np_ptr(resid),
                                      _stream(stream))
    _check(rc, "pwk_sternheimer_cg_batched")
    return rc, iters, resid


def _check_eigh_args(H, S, nev: int, eig=None, vec=None, status=None):
    """Shapes, dtypes and device of the reduced-eigensolver arguments, checked before any
    pointer reaches the library (the kernel trusts them): H, S complex128 [nprob][n][n],
    1 <= nev <= n, eig float64 [nprob][nev], vec complex128 [nprob][n][nev], status int32
    [nprob], all contiguous on one CUDA device.  Raises ValueError."""
    import torch
    if H.dim() != 3 or H.shape[1] != H.shape[2]:
        raise ValueError("H must have shape (nprob, n, n)")
    nprob, n = int(H.shape[0]), int(H.shape[1])
    if not 1 <= int(nev) <= n:
        raise ValueError("need 1 <= nev <= n")
    want = [("H", H, torch.complex128, (nprob, n, n)), ("S", S, torch.complex128, (nprob, n, n)),
            ("eig", eig, torch.float64, (nprob, nev)), ("vec", vec, torch.complex128, (nprob, n, nev)),
            ("status", status, torch.int32, (nprob,))]
    dev = None
    for name, t, dt, shape in want:
        if t is None:
            continue
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    for name, t, dt, shape in want:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError(f"{name} is on {t.device}, H on {dev}: all arguments on one device")
    return nprob, n, dev


def eigh_batched(H, S, nev: int, status=None, stream=None):
    """pwk_eigh_batched on complex128 CUDA tensors H, S [nprob][n][n]; returns (eig, vec)."""
    import torch
    nprob, n, dev = _check_eigh_args(H, S, nev, status=status)
    eig = torch.empty((nprob, nev), dtype=torch.float64, device=dev)
    vec = torch.empty((nprob, n, nev), dtype=torch.complex128, device=dev)
    with torch.cuda.device(dev):
        _check(load().pwk_eigh_batched(nprob, n, nev, _ptr(H), _ptr(S), _ptr(eig), _ptr(vec),
                                       _ptr(status) if status is not None else None,
                                       _stream(stream)), "pwk_eigh_batched")
    return eig, vec


def eigh_batched_noalloc(H, S, nev: int, eig, vec, status=None, stream=None):
    """pwk_eigh_batched_noalloc: the same solve with the library's built-in workspace; the
    caller provides the outputs eig [nprob][nev] float64 and vec [nprob][n][nev] complex128
    (and optionally status [nprob] int32), all on H's device, where the call runs.
    Asynchronous: synchronise the stream before reading the results."""
    import torch
    nprob, n, dev = _check_eigh_args(H, S, nev, eig, vec, status)
    with torch.cuda.device(dev):
        _check(load().pwk_eigh_batched_noalloc(nprob, n, nev, _ptr(H), _ptr(S), _ptr(eig), _ptr(vec),
                                               _ptr(status) if status is not None else None,
                                               _stream(stream)), "pwk_eigh_batched_noalloc")


def measure_fma_peak(precision: int, stream=None):
    """pwk_measure_fma_peak on the current device: (FLOP/s, SM count)."""
    f = _D(0.0)
    n = _I(0)
    _check(load().pwk_measure_fma_peak(precision, ctypes.byref(f), ctypes.byref(n), _stream(stream)),
           "pwk_measure_fma_peak")
    return f.value, n.value


def launch_count() -> int:
    """pwk_launch_count: kernels the library has launched in this process so far."""
    return int(load().pwk_launch_count())


def supported_grid(N: int) -> bool:
    return bool(load().pwk_supported_grid(N))


def version() -> str:
    return load().pwk_version().decode()
