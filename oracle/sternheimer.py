"""Oracle: the DFPT linear system and its preconditioned CG (TEST INFRASTRUCTURE ONLY).

Follows paper Sec. 2.3-2.4 with S = I and dS = 0 (norm-conserving), in FP64, one (k, n)
at a time:

  [H_{k+q} + alpha P_v - eps_{k,n}] dpsi = -P_c dV psi_{k,n}           (Eq. linear_system)

with P_v = sum_v |psi_{k+q,v}><psi_{k+q,v}| (Eq. projector with S = I), P_c = 1 - P_v and
dV = e^{iq.r} dv(r), so the lattice-periodic part of dV psi_{k,n} is dv(r) u_{k,n}(r),
expanded on the k+q sphere.  ``solve_dense`` is the exact answer (LAPACK LU);
``pcg`` follows Eqs. ax1 to updatedold literally.

Readings: d^T r is taken as Re<d|r> (Hermitian product); the preconditioner is
M_GG = max(1, |k+q+G|^2 / <psi_{k+q,nu}|T|psi_{k+q,nu}>) in Ry (Sec. 2.4, same ratio as the
Ha form); alpha = max(2 (eps_max - eps_min), 0.01 Ry) over the occupied eigenvalues at k and k+q.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as ham


def dv_psi_dense(miller_kq, miller_k, dvt, psi_k):
    """Periodic part of dV psi_{k,n} on the k+q sphere by the circular convolution with
    dv~(m) (the composition of inverse transform, product, forward transform, Sec. 2.2.2)."""
    M = ham.local_matrix(miller_kq, miller_k, dvt)
    return psi_k @ M.T


def dv_psi_direct(miller_kq, miller_k, dv_r, psi_k, N):
    """Same quantity by the paper's route with direct Fourier sums: u_k(r) = sum_G psi e^{iG.r},
    multiply by dv(r), C(G) = (1/N_r) sum_r (.) e^{-iG.r} for G on the k+q sphere."""
    Ek = ham.phase_matrix(miller_k, N)
    Ekq = ham.phase_matrix(miller_kq, N)
    u = ham.to_real_space(psi_k, Ek)
    return ham.to_reciprocal(u * dv_r.ravel()[None, :], Ekq)


def project_conduction(psi_kq_occ: np.ndarray, x: np.ndarray) -> np.ndarray:
    """P_c x = x - sum_v psi_v <psi_v|x> (rows of x are vectors; Eq. linear_system)."""
    return x - (x @ psi_kq_occ.conj().T) @ psi_kq_occ


def alpha_pv(eps_k_occ: np.ndarray, eps_kq_occ: np.ndarray) -> float:
    e = np.concatenate([np.ravel(eps_k_occ), np.ravel(eps_kq_occ)])
    return max(2.0 * (e.max() - e.min()), 0.01)


def operator(H_kq: np.ndarray, psi_kq_occ: np.ndarray, eps: float, alpha: float) -> np.ndarray:
    """A = H_{k+q} - eps_{k,n} + alpha sum_v |psi_v><psi_v| (Eq. linear_system, Eq. projector)."""
    P = psi_kq_occ.T @ psi_kq_occ.conj()          # columns psi_v
    A = H_kq + alpha * P
    A[np.diag_indices_from(A)] -= eps
    return A


def rhs(dvpsi: np.ndarray, psi_kq_occ: np.ndarray) -> np.ndarray:
    """b = -P_c dV psi_{k,n} (right-hand side of Eq. linear_system with dS = 0)."""
    return -project_conduction(psi_kq_occ, dvpsi)


def solve_dense(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    return np.linalg.solve(A, b)


def preconditioner(g2_kq: np.ndarray, psi_kq_nu: np.ndarray) -> np.ndarray:
    """M_GG = max(1, |k+q+G|^2 / <psi|T|psi>) (Sec. 2.4; Ry form of the Ha ratio)."""
    tkin = float(np.real(np.vdot(psi_kq_nu, g2_kq * psi_kq_nu)) / np.real(np.vdot(psi_kq_nu, psi_kq_nu)))
    return np.maximum(1.0, g2_kq / tkin)


def pcg(apply_a, b: np.ndarray, m_diag: np.ndarray, x0: np.ndarray = None, thr: float = 1e-20,
        max_iter: int = 1000):
    """Preconditioned CG of Sec. 2.4, Eqs. ax1 .. updatedold, for one right-hand side.

    Iterates from Eq. row2 until |rho| < thr.  Returns (x, iterations)."""
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128).copy()
    r = apply_a(x) - b                        # Eq. ax1
    d_old = None
    rho_old = None
    it = 0
    for it in range(1, max_iter + 1):
        d = r / m_diag                        # Eq. row2
        rho = np.real(np.vdot(d, r))          # Eq. row3
        if abs(rho) < thr:
            return x, it - 1
        if d_old is not None:
            gamma = rho / rho_old             # Eq. row4
            d = d + gamma * d_old             # Eq. updated
        t = apply_a(d)                        # Eq. ax2
        lam = -np.real(np.vdot(d, r)) / np.real(np.vdot(d, t))   # Eq. lambda
        x = x + lam * d                       # Eq. updatex
        r = r + lam * t                       # Eq. updater
        d_old = d                             # Eq. updatedold
        rho_old = rho
    return x, it
