"""Planted mistakes in the oracle (CPU only): each one must fail at least one pin.

Every case below replaces one oracle function, in this process only, by a copy carrying a
plausible slip (a dropped term or factor, a wrong sign, a missing or misplaced conjugate, a
transposed operand or index, swapped grid axes) and runs the pins of tests/test_oracle_*.py
until one fails.  A case that no pin catches is a hole in the pins, and this test names it.
Nothing here touches the GPU path: the mistakes are planted in the oracle only.
"""
import inspect

import numpy as np
import pytest

from oracle import davidson as dav
from oracle import drho as dr
from oracle import hamiltonian as ham
from oracle import overlap as ov
from oracle import sternheimer as st

import test_oracle_drho
import test_oracle_hamiltonian
import test_oracle_overlap
import test_oracle_sternheimer

_PIN_MODULES = {"hamiltonian": test_oracle_hamiltonian, "davidson": test_oracle_hamiltonian,
                "sternheimer": test_oracle_sternheimer, "overlap": test_oracle_overlap,
                "drho": test_oracle_drho}

# originals, taken before any case patches them
_kinetic = ham.kinetic
_grid = ham.grid_coefficients
_local = ham.local_matrix
_phase = ham.phase_matrix
_reduced_eig_keep = dav._reduced_eig_keep
_lowest = dav.lowest_eigenpairs
_st_rhs = st.rhs
_drho = dr.drho


def _dense_h_without_kinetic(kc, miller, B, V_r, beta_k, D, vt=None):
    if vt is None:
        vt = ham.grid_coefficients(V_r)
    return ham.local_matrix(miller, miller, vt) + ham.nonlocal_matrix(beta_k, D)


def _reduced_without_conjugate(basis, hbasis, sbasis):
    Hr = basis @ hbasis.T
    Sr = basis @ sbasis.T
    return 0.5 * (Hr + Hr.conj().T), 0.5 * (Sr + Sr.conj().T)


def _reduced_eig_without_overlap(Hr, Sr, nb, drop_tol=1e-6):
    _, _, keep = _reduced_eig_keep(Hr, Sr, nb, drop_tol)
    w, v = np.linalg.eigh(Hr[np.ix_(keep, keep)])
    full = np.zeros((len(Sr), nb), np.complex128)
    full[keep] = v[:, :nb]
    return w[:nb], full, keep


def _pcg_wrong_step_sign(apply_a, b, m_diag, x0=None, thr=1e-20, max_iter=1000):
    x = np.zeros_like(b)
    r = apply_a(x) - b
    d_old = rho_old = None
    it = 0
    for it in range(1, max_iter + 1):
        d = r / m_diag
        rho = np.real(np.vdot(d, r))
        if abs(rho) < thr:
            return x, it - 1
        if d_old is not None:
            d = d + (rho / rho_old) * d_old
        t = apply_a(d)
        lam = np.real(np.vdot(d, r)) / np.real(np.vdot(d, t))      # slip: sign of the step
        x = x + lam * d
        r = r + lam * t
        d_old, rho_old = d, rho
    return x, it


def _pcg_inverted_gamma(apply_a, b, m_diag, x0=None, thr=1e-20, max_iter=1000):
    x = np.zeros_like(b)
    r = apply_a(x) - b
    d_old = rho_old = None
    it = 0
    for it in range(1, max_iter + 1):
        d = r / m_diag
        rho = np.real(np.vdot(d, r))
        if abs(rho) < thr:
            return x, it - 1
        if d_old is not None:
            d = d + (rho_old / rho) * d_old                           # slip: gamma inverted
        t = apply_a(d)
        lam = -np.real(np.vdot(d, r)) / np.real(np.vdot(d, t))
        x = x + lam * d
        r = r + lam * t
        d_old, rho_old = d, rho
    return x, it


# (case name, oracle module, attribute, replacement, module whose pins run first)
CASES = [
    ("kinetic: k dropped", ham, "kinetic", lambda kc, m, B: _kinetic(np.zeros(3), m, B), "hamiltonian"),
    ("kinetic: |k-G|^2", ham, "kinetic", lambda kc, m, B: _kinetic(kc, -m, B), "hamiltonian"),
    ("kinetic: Ha instead of Ry", ham, "kinetic", lambda kc, m, B: 0.5 * _kinetic(kc, m, B), "hamiltonian"),
    ("forward transform exponent e^{+i}", ham, "grid_coefficients",
     lambda f: np.conj(_grid(np.conj(f))), "hamiltonian"),
    ("forward transform without 1/N_r", ham, "grid_coefficients",
     lambda f: _grid(f) * f.size, "hamiltonian"),
    ("local matrix indexed m' - m", ham, "local_matrix",
     lambda mo, mi, ft: _local(mi, mo, ft).T, "hamiltonian"),
    ("nonlocal matrix conjugate on the wrong side", ham, "nonlocal_matrix",
     lambda b, D: b.conj().T @ D @ b, "hamiltonian"),
    ("nonlocal term dropped", ham, "nonlocal_matrix",
     lambda b, D: np.zeros((b.shape[1], b.shape[1]), np.complex128), "hamiltonian"),
    ("kinetic term dropped from H", ham, "dense_h", _dense_h_without_kinetic, "hamiltonian"),
    ("inverse transform exponent e^{-i}", ham, "to_real_space",
     lambda c, E: c @ E.conj().T, "hamiltonian"),
    ("forward route without 1/N_r", ham, "to_reciprocal", lambda f, E: f @ E.conj(), "hamiltonian"),
    ("forward route without conjugate", ham, "to_reciprocal",
     lambda f, E: f @ E / E.shape[0], "hamiltonian"),
    ("grid axes 2 and 3 swapped", ham, "phase_matrix",
     lambda m, N: _phase(m[:, [0, 2, 1]], N), "hamiltonian"),
    ("projections without conjugate", ham, "projections", lambda b, psi: psi @ b.T, "hamiltonian"),
    ("reduced matrices without conjugate", dav, "_reduced", _reduced_without_conjugate, "davidson"),
    ("reduced problem without the overlap", dav, "_reduced_eig_keep", _reduced_eig_without_overlap,
     "davidson"),
    ("exact reference takes the highest pairs", dav, "lowest_eigenpairs",
     lambda H, nb: (np.linalg.eigh(H)[0][-nb:], np.linalg.eigh(H)[1][:, -nb:].T), "davidson"),
    ("P_c without conjugate", st, "project_conduction",
     lambda p, x: x - (x @ p.T) @ p, "sternheimer"),
    ("alpha P_v with the wrong sign", st, "operator",
     lambda H, p, e, a: H - a * (p.T @ p.conj()) - e * np.eye(len(H)), "sternheimer"),
    ("P_v un-conjugated", st, "operator",
     lambda H, p, e, a: H + a * (p.T @ p) - e * np.eye(len(H)), "sternheimer"),
    ("eps added instead of subtracted", st, "operator",
     lambda H, p, e, a: H + a * (p.T @ p.conj()) + e * np.eye(len(H)), "sternheimer"),
    ("right-hand side with + sign", st, "rhs", lambda d, p: -_st_rhs(d, p), "sternheimer"),
    ("right-hand side without P_c", st, "rhs", lambda d, p: -d, "sternheimer"),
    ("CG step with the wrong sign", st, "pcg", _pcg_wrong_step_sign, "sternheimer"),
    ("CG gamma inverted", st, "pcg", _pcg_inverted_gamma, "sternheimer"),
    ("S without the identity", ov, "overlap_matrix", lambda b, q: b.T @ q @ b.conj(), "overlap"),
    ("S conjugate on the wrong side", ov, "overlap_matrix",
     lambda b, q: np.eye(b.shape[1]) + b.conj().T @ q @ b, "overlap"),
    ("S steps without conjugate", ov, "spsi_steps", lambda b, q, psi: psi + (psi @ b.T) @ q.T @ b,
     "overlap"),
    ("alpha Q without S", ov, "operator",
     lambda H, S, u, e, a: H + a * (u.T @ u.conj()) - e * S, "overlap"),
    ("eps I in place of eps S", ov, "operator",
     lambda H, S, u, e, a: H + a * ((S @ u.T) @ (S @ u.T).conj().T) - e * np.eye(len(H)), "overlap"),
    ("right-hand side (1 - P_v S)", ov, "rhs",
     lambda d, S, u: -(d - ((d @ S.T) @ u.conj().T) @ u), "overlap"),
    ("generalized reference without S", ov, "lowest_generalized",
     lambda H, S, nb: (np.linalg.eigh(H)[0][:nb], np.linalg.eigh(H)[1][:, :nb].T), "overlap"),
    ("drho without the conjugate of u", dr, "drho_k",
     lambda mk, mq, N, u, du: np.sum(ham.to_real_space(u, ham.phase_matrix(mk, N))
                                     * ham.to_real_space(du, ham.phase_matrix(mq, N)), axis=0),
     "drho"),
    ("drho without the factor 4", dr, "drho", lambda *a, **k: _drho(*a, **k) / 4, "drho"),
    ("drho weights ignored", dr, "drho",
     lambda pk, pq, u, uq, du, weights=None, S_list=None: _drho(pk, pq, u, uq, du, None, S_list),
     "drho"),
    ("P_c in drho without S", dr, "project_conduction",
     lambda u, du, S=None: du - (du @ u.conj().T) @ u, "drho"),
]


def _pins(first: str):
    order = [_PIN_MODULES[first]] + [m for m in dict.fromkeys(_PIN_MODULES.values())
                                     if m is not _PIN_MODULES[first]]
    for mod in order:
        for name, fn in sorted(vars(mod).items()):
            if name.startswith("test_") and callable(fn):
                yield f"{mod.__name__}::{name}", fn


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(case, cfg1, monkeypatch):
    label, module, attr, replacement, first = case
    assert hasattr(module, attr), attr
    monkeypatch.setattr(module, attr, replacement)
    crashes = []
    for pin, fn in _pins(first):
        args = [cfg1 for p in inspect.signature(fn).parameters if p == "cfg1"]
        try:
            with np.errstate(all="ignore"):
                fn(*args)
        except AssertionError:               # a pin's check failed: the slip is caught
            return
        except Exception as exc:             # a crash is not a catch: the next pin must assert
            crashes.append(f"{pin}: {type(exc).__name__}")
    pytest.fail(f"no pin asserts against the planted mistake '{label}' in {module.__name__}.{attr}"
                + (f" (pins that crashed instead: {crashes})" if crashes else ""))


def test_cases_cover_every_oracle_module():
    touched = {c[1].__name__ for c in CASES}
    assert touched == {m.__name__ for m in (ham, dav, st, ov, dr)}
