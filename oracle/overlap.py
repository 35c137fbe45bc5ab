"""Oracle: the ultrasoft/PAW overlap operator S and the generalized problems built on it
(TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the bench baseline).

FP64, one k at a time, Rydberg units.

  S|psi> = |psi> + sum_{I,mn} q^I_mn |beta^I_m><beta^I_n|psi>          (Sec. 2.2, overlap)

reached by the steps of Sec. 2.2.3: lambda = <beta|psi> (Eq. lambdah), delta = q lambda
(Eq. delta_eq), S psi = psi + sum_m delta_m beta_m (Eq. finals).  ``overlap_matrix`` is the
dense definition, ``spsi_steps`` the three steps; the pins check one against the other and
both against closed forms.

Generalized problems:
  * H x = eps S x (Eq. ks with S): ``lowest_generalized`` (LAPACK through scipy, as the
    paper's ZHEGV step of Sec. 5);
  * the DFPT system of Eq. linear_system with S (dS = 0, the perturbation being a local
    potential dv):  [H_{k+q} + alpha Q - eps S] dpsi = -P_c^dagger dV psi, with
    alpha Q = alpha sum_v S|u_v><u_v|S (Eq. projector) and P_c^dagger = 1 - S P_v,
    P_v = sum_v |u_v><u_v| over S-orthonormal valence states of k+q.

Reading (the paper writes P_c on the right-hand side and does not spell out its adjoint
form): the right-hand side is taken as -(1 - S P_v) dV psi, the form for which the
right-hand side has no component along any valence state (<u_v|b> = 0 for S-orthonormal
u_v); with S = I it is the norm-conserving -P_c dV psi.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def overlap_matrix(beta_k: np.ndarray, q: np.ndarray) -> np.ndarray:
    """S[G, G'] = delta_GG' + sum_mn beta_m(k+G) q_mn conj(beta_n(k+G')) (Sec. 2.2).

    beta_k (nkb, npw) complex, q (nkb, nkb) real symmetric, block diagonal per atom."""
    npw = beta_k.shape[1]
    return np.eye(npw, dtype=np.complex128) + beta_k.T @ q @ beta_k.conj()


def spsi_steps(beta_k: np.ndarray, q: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """S psi for rows psi (nv, npw), by Eqs. lambdah, delta_eq and finals in that order."""
    lam = psi @ beta_k.conj().T          # lambda[v, n] = sum_G conj(beta_n(G)) psi_v(G)
    delta = lam @ q.T                    # delta[v, m] = sum_n q_mn lambda[v, n]
    return psi + delta @ beta_k          # psi_v(G) + sum_m delta[v, m] beta_m(G)


def lowest_generalized(H: np.ndarray, S: np.ndarray, nb: int):
    """Exact lowest nb eigenpairs of H x = eps S x; eigenvectors as S-orthonormal rows."""
    w, v = scipy.linalg.eigh(H, S)
    return w[:nb], v[:, :nb].T


def s_orthonormal(S: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Rows of X made S-orthonormal (Cholesky of the Gram matrix X S X^H), for inputs."""
    G = X.conj() @ S @ X.T
    L = np.linalg.cholesky(0.5 * (G + G.conj().T))
    return np.linalg.solve(L.conj(), X)


def operator(H_kq: np.ndarray, S_kq: np.ndarray, u_occ: np.ndarray, eps: float,
             alpha: float) -> np.ndarray:
    """A = H_{k+q} + alpha sum_v S|u_v><u_v|S - eps S (Eq. linear_system, Eq. projector)."""
    SU = S_kq @ u_occ.T                    # columns S u_v
    return H_kq + alpha * (SU @ SU.conj().T) - eps * S_kq


def rhs(dvpsi: np.ndarray, S_kq: np.ndarray, u_occ: np.ndarray) -> np.ndarray:
    """b = -(1 - S P_v) dV psi for rows dvpsi (reading in the module docstring)."""
    coef = dvpsi @ u_occ.conj().T          # <u_v|dV psi>
    return -(dvpsi - (coef @ u_occ) @ S_kq.T)
