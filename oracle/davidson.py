"""Oracle: block Davidson diagonalisation of one k (TEST INFRASTRUCTURE ONLY).

Follows the steps of paper Sec. 2.1 in order, in FP64, for one k at a time, with S = I
(norm-conserving projectors) unless an overlap operator S is passed (ultrasoft/PAW q_mn,
Sec. 2.2; oracle/overlap.py builds it).  The reduced generalized problem (H~ - eps S~) v = 0
is solved with LAPACK (scipy.linalg.eigh), which the paper also uses for this step
(Sec. 5, ZHEGV/ZHEGVX).  ``lowest_eigenpairs`` is the exact result the iteration reaches.

Readings of points the paper leaves open (listed with the design notes):
  * the preconditioner denominator x = H_GG - eps_i S_GG is clamped to sign(x) max(|x|, 1e-2 Ry);
  * a band is converged when |eps_i^(n+1) - eps_i^(n)| < eps_th; an optional residual
    bound ||H phi - eps S phi|| < res_tol may be required as well;
  * a restart keeps the current Ritz vectors and eigenvalues as the new basis (the restart
    step of Sec. 2.1);
  * when the preconditioned residual is numerically parallel to its Ritz vector
    (|cos| > 1 - 1e-6, which happens when H is diagonal in the plane-wave basis and the
    diagonal preconditioner is exact), or when the band's previous correction was left out
    of the reduced problem as dependent on the basis, the unpreconditioned residual is used
    instead (Galerkin-orthogonal to the basis), so the correction brings a new direction;
  * basis vectors that are numerically dependent on the earlier ones (the Cholesky pivot of
    S~ below 1e-6 of its diagonal, a new direction below 1e-3 of the vector's norm) are
    left out of the reduced problem.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def lowest_eigenpairs(H: np.ndarray, nb: int):
    """Exact lowest nb eigenpairs of the dense Hermitian H(k) (Eq. ks with S = I)."""
    w, v = np.linalg.eigh(H)
    return w[:nb], v[:, :nb].T


def _reduced_eig(Hr, Sr, nb, drop_tol=1e-6):
    """Lowest nb eigenpairs of (H~ - eps S~) v = 0 on the basis vectors that are independent:
    a vector whose Cholesky pivot falls below drop_tol of its S~ diagonal is left out (its
    coefficients are zero)."""
    w, full, _ = _reduced_eig_keep(Hr, Sr, nb, drop_tol)
    return w, full


def _reduced_eig_keep(Hr, Sr, nb, drop_tol=1e-6):
    """_reduced_eig, also returning the indices of the basis vectors kept."""
    n = len(Sr)
    keep = []
    for j in range(n):
        idx = keep + [j]
        S = Sr[np.ix_(idx, idx)]
        try:
            L = np.linalg.cholesky(S)
        except np.linalg.LinAlgError:
            continue
        if L[-1, -1].real ** 2 > drop_tol * Sr[j, j].real:
            keep.append(j)
    w, v = scipy.linalg.eigh(Hr[np.ix_(keep, keep)], Sr[np.ix_(keep, keep)])
    full = np.zeros((n, nb), np.complex128)
    full[keep] = v[:, :nb]
    return w[:nb], full, keep


def _reduced(basis, hbasis, sbasis):
    # H~_ij = <phi_i|H|phi_j>, S~_ij = <phi_i|S|phi_j> (Sec. 2.1)
    Hr = basis.conj() @ hbasis.T
    Sr = basis.conj() @ sbasis.T
    return 0.5 * (Hr + Hr.conj().T), 0.5 * (Sr + Sr.conj().T)


def _precondition_denominator(x: np.ndarray, floor: float = 1e-2) -> np.ndarray:
    s = np.where(x >= 0, 1.0, -1.0)
    return s * np.maximum(np.abs(x), floor)


def davidson(apply_h, h_diag: np.ndarray, psi0: np.ndarray, eth: float = 1e-10,
             max_iter: int = 100, max_basis: int = None, res_tol: float = None,
             apply_s=None, s_diag: np.ndarray = None):
    """Block Davidson (Sec. 2.1) for one k.

    apply_h(X) -> H X for rows X (n, npw); h_diag (npw,) the diagonal of H in the plane-wave
    basis; psi0 (nb, npw) trial vectors; apply_s / s_diag the overlap S and its diagonal
    (None: S = I).  Returns (eps (nb,), psi (nb, npw) S-orthonormal, iterations, number of
    H applications, converged flags)."""
    nb = psi0.shape[0]
    if max_basis is None:
        max_basis = 4 * nb
    if apply_s is None:
        apply_s = lambda X: X  # noqa: E731
        s_diag = np.ones_like(h_diag)
    basis = psi0.astype(np.complex128).copy()
    hbasis = apply_h(basis)
    sbasis = apply_s(basis)
    napply = nb
    # 1. reduced problem on the trial vectors, eigenpairs {phi^(n), eps^(n)}
    Hr, Sr = _reduced(basis, hbasis, sbasis)
    eps, vecs, keep = _reduced_eig_keep(Hr, Sr, nb)
    last = np.full(nb, -1)                  # basis row of each band's latest correction
    todo = np.arange(nb)                    # the first step corrects every band
    conv = np.zeros(nb, bool)
    it = 0
    for it in range(1, max_iter + 1):
        # 2. correction vectors (H_diag - eps_i S_diag)^-1 (H - eps_i S)|phi_i>
        ritz = vecs[:, todo].T @ basis
        hritz = vecs[:, todo].T @ hbasis
        sritz = vecs[:, todo].T @ sbasis
        resid = hritz - eps[todo, None] * sritz
        corr = resid / _precondition_denominator(h_diag[None, :] - eps[todo, None] * s_diag[None, :])
        cos = np.abs(np.sum(ritz.conj() * corr, axis=1)) / (
            np.linalg.norm(ritz, axis=1) * np.linalg.norm(corr, axis=1))
        dropped = np.array([last[i] >= 0 and last[i] not in keep for i in todo], bool)
        parallel = (cos > 1.0 - 1e-6) | dropped
        corr[parallel] = resid[parallel]
        # 3. normalisation
        corr /= np.linalg.norm(corr, axis=1, keepdims=True)
        # restart with the current Ritz vectors when the basis would grow too large
        if basis.shape[0] + len(todo) > max_basis:
            basis = vecs.T @ basis
            hbasis = vecs.T @ hbasis
            sbasis = vecs.T @ sbasis
            last[:] = -1
        # 4. extended reduced Hamiltonian and overlap
        last[todo] = basis.shape[0] + np.arange(len(todo))
        basis = np.vstack([basis, corr])
        hbasis = np.vstack([hbasis, apply_h(corr)])
        sbasis = np.vstack([sbasis, apply_s(corr)])
        napply += len(todo)
        Hr, Sr = _reduced(basis, hbasis, sbasis)
        # 5. diagonalise the N_base x N_base reduced problem
        eps_new, vecs, keep = _reduced_eig_keep(Hr, Sr, nb)
        # 6. bands whose eigenvalue moved by more than eps_th still need a correction
        moved = np.abs(eps_new - eps) > eth
        if res_tol is not None:
            sritz = vecs.T @ sbasis
            rn = np.linalg.norm(vecs.T @ hbasis - eps_new[:, None] * sritz, axis=1)
            moved |= rn > res_tol
        eps = eps_new
        todo = np.nonzero(moved)[0]
        conv = ~moved
        if len(todo) == 0:
            break
    psi = vecs.T @ basis
    return eps, psi, it, napply, conv
