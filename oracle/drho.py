"""Oracle: the charge density induced by a perturbation, Eq. drho (TEST INFRASTRUCTURE ONLY:
imported by tests/, the smoke check and the bench baseline).

FP64, direct Fourier sums (no FFT library), Rydberg units.

  drho(r) = 4 sum_{k,nu} w_k conj(u_{k,nu}(r)) [P_c du_{k,nu}](r)        (Eq. drho)

without the augmentation term (the paper did not accelerate it).  u_{k,nu}(r) and du(r) are
the lattice-periodic parts on the real-space grid by the paper's inverse transform without
normalisation (Sec. 2.2.2): u(r_l) = sum_G C(G) e^{i G.r_l}, G on the k sphere for u and on
the k+q sphere for du; the product is the lattice-periodic part of psi* dpsi (the e^{iq.r}
factor of dpsi and e^{-ik.r} of psi* combine to e^{iq.r}, left out like the 1/sqrt(V) of
the Bloch functions).

Readings (the paper leaves them implicit):
  * w_k = 1 / N_k, the weights of the unreduced Monkhorst-Pack grid (they sum to 1); the
    factor 4 is the paper's (spin and the two terms psi* dpsi + dpsi* psi of a real
    perturbation);
  * P_c du = du - sum_v u_{k+q,v} <u_{k+q,v}| S |du> with S-orthonormal u_{k+q,v} (S = 1
    without q), the projector of Eq. linear_system on the k+q conduction space;
  * drho is returned on the N1 x N2 x N3 grid (l3 fastest), per grid point, without the
    1/Omega of a density per volume.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as ham


def project_conduction(u_kq_occ: np.ndarray, du: np.ndarray, S_kq: np.ndarray = None) -> np.ndarray:
    """P_c du = du - sum_v u_v <u_v|S|du> for rows du; S_kq None means S = 1."""
    sdu = du if S_kq is None else du @ S_kq.T
    return du - (sdu @ u_kq_occ.conj().T) @ u_kq_occ


def drho_k(miller_k, miller_kq, N, u_k: np.ndarray, du_c: np.ndarray) -> np.ndarray:
    """sum_nu conj(u_nu(r)) du_nu(r) on the grid for one k (rows u_k, du_c already projected)."""
    Ek = ham.phase_matrix(miller_k, N)
    Ekq = ham.phase_matrix(miller_kq, N)
    ur = ham.to_real_space(u_k, Ek)          # (nocc, N_r)
    dr = ham.to_real_space(du_c, Ekq)
    return np.sum(ur.conj() * dr, axis=0)


def drho(pk, pq, u_k: np.ndarray, u_kq: np.ndarray, du: np.ndarray, weights=None,
         S_list=None) -> np.ndarray:
    """Eq. drho over every k of the problems pk (k points) and pq (k+q points).

    u_k (nk, nocc, npw_max_k), u_kq (nk, nocc, npw_max_kq), du (nk, nocc, npw_max_kq);
    weights (nk,) the w_k (default 1/nk); S_list: per-k overlap matrices of the k+q spheres
    or None.  Returns (N, N, N) complex."""
    N = pk.N
    nk = pk.nk
    w = np.full(nk, 1.0 / nk) if weights is None else np.asarray(weights, float)
    acc = np.zeros(N ** 3, np.complex128)
    for i in range(nk):
        nkk, nq = int(pk.npw[i]), int(pq.npw[i])
        S = None if S_list is None else S_list[i]
        duc = project_conduction(u_kq[i, :, :nq], du[i, :, :nq], S)
        acc += 4.0 * w[i] * drho_k(pk.miller[i, :nkk], pq.miller[i, :nq], N, u_k[i, :, :nkk], duc)
    return acc.reshape(N, N, N)
