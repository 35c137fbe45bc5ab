"""Oracle: the Kohn-Sham Hamiltonian applied to Bloch wave-functions (TEST INFRASTRUCTURE ONLY).

Units: Rydberg (kinetic energy |k+G|^2), the Ry form of paper Sec. 2.2.1 (1/2|k+G|^2 in Ha).
Everything is FP64.  Two independent routes are provided for the local term:

  * ``local_matrix``: the exact G-space definition reached by the FFT method, a circular
    convolution with the grid coefficients V~(m) = (1/N_r) sum_r V(r) e^{-2 pi i m.l/N};
  * ``hpsi_direct``: the paper's own route written as direct Fourier sums (Sec. 2.2.2,
    u = sum_G C e^{iG.r}, u' = V u, C' = (1/N_r) sum_r u' e^{-iG.r}; Sec. 4, Eq. fwFFT),
    O(npw * N_r) per band, no FFT.

Parity pins live in tests/test_oracle_*.py (free electrons, constant shift, single
sine wave, translation invariance, Hermiticity, secular equation, dense == direct).
"""
from __future__ import annotations

import numpy as np


def reciprocal(A: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij (Sec. 4, the mesh G_{m1,m2,m3})."""
    return 2.0 * np.pi * np.linalg.inv(A).T


def kinetic(kc: np.ndarray, miller: np.ndarray, B: np.ndarray) -> np.ndarray:
    """|k+G|^2 in Ry for G = m1 b1 + m2 b2 + m3 b3 (Sec. 2.2.1, C' = 1/2|k+G|^2 C in Ha)."""
    q = kc[None, :] + miller @ B
    return np.einsum("gi,gi->g", q, q)


def _dft_matrix(N: int, sign: int) -> np.ndarray:
    l = np.arange(N)
    return np.exp(sign * 2j * np.pi * np.outer(l, l) / N)


def grid_coefficients(f_r: np.ndarray) -> np.ndarray:
    """f~(m) = (1/N_r) sum_l f(l) e^{-2 pi i m.l/N} for all m mod N (Sec. 4, Eq. fwFFT).

    Written as three separable direct sums over l3, l2, l1 (no FFT library)."""
    N1, N2, N3 = f_r.shape
    E1, E2, E3 = _dft_matrix(N1, -1), _dft_matrix(N2, -1), _dft_matrix(N3, -1)
    t = np.einsum("kc,abc->abk", E3, f_r.astype(np.complex128))
    t = np.einsum("jb,abk->ajk", E2, t)
    t = np.einsum("ia,ajk->ijk", E1, t)
    return t / (N1 * N2 * N3)


def local_matrix(miller_out: np.ndarray, miller_in: np.ndarray, ft: np.ndarray) -> np.ndarray:
    """M[G, G'] = f~((m - m') mod N): the local operator in the plane-wave basis.

    The inverse transform, pointwise product and forward transform of Sec. 2.2.2 compose
    to this circular convolution exactly (Eqs. zfft, yfft, xfft, fwFFT)."""
    N = np.array(ft.shape)
    d = (miller_out[:, None, :] - miller_in[None, :, :]) % N
    return ft[d[..., 0], d[..., 1], d[..., 2]]


def nonlocal_matrix(beta_k: np.ndarray, D: np.ndarray) -> np.ndarray:
    """V_NL[G, G'] = sum_{mn} beta_m(k+G) D_mn conj(beta_n(k+G')) (Sec. 2.2, Eqs. lambdah,
    gamma, finalnl composed).  beta_k is (nkb, npw); D (nkb, nkb), block diagonal per atom."""
    return beta_k.T @ D @ beta_k.conj()


def dense_h(kc, miller, B, V_r, beta_k, D, vt=None) -> np.ndarray:
    """Dense H(k) = |k+G|^2 delta + V~(m-m') + V_NL (Sec. 2.2, H_KS = kinetic + local + nonlocal)."""
    if vt is None:
        vt = grid_coefficients(V_r)
    H = local_matrix(miller, miller, vt)
    H = H + nonlocal_matrix(beta_k, D)
    H[np.diag_indices_from(H)] += kinetic(kc, miller, B)
    return H


def problem_h(prob, ik: int, vt=None) -> np.ndarray:
    n = int(prob.npw[ik])
    return dense_h(prob.kpts[ik], prob.miller[ik, :n], prob.B, prob.V_r, prob.beta[ik, :, :n],
                   prob.D, vt)


def hpsi_dense(prob, ik: int, psi_k: np.ndarray, vt=None) -> np.ndarray:
    """H|psi> for all bands of one k by the dense matrix; psi_k (nb, npw_max), zero padded."""
    n = int(prob.npw[ik])
    H = problem_h(prob, ik, vt)
    out = np.zeros_like(psi_k, dtype=np.complex128)
    out[:, :n] = psi_k[:, :n] @ H.T
    return out


def phase_matrix(miller: np.ndarray, N) -> np.ndarray:
    """E[l, G] = e^{2 pi i m.l / N} for every grid point l (l3 fastest) and basis G."""
    N1, N2, N3 = (N, N, N) if np.isscalar(N) else N
    l1, l2, l3 = np.meshgrid(np.arange(N1), np.arange(N2), np.arange(N3), indexing="ij")
    arg = (np.outer(l1.ravel(), miller[:, 0]) / N1 + np.outer(l2.ravel(), miller[:, 1]) / N2
           + np.outer(l3.ravel(), miller[:, 2]) / N3)
    return np.exp(2j * np.pi * arg)


def to_real_space(coef: np.ndarray, E: np.ndarray) -> np.ndarray:
    """u(r) = sum_G C(G) e^{iG.r} (Sec. 2.2.2, inverse transform, no normalisation)."""
    return coef @ E.T


def to_reciprocal(f_r: np.ndarray, E: np.ndarray) -> np.ndarray:
    """C'(G) = (1/N_r) sum_r f(r) e^{-iG.r} (Sec. 2.2.2 and Eq. fwFFT, factor 1/N_r)."""
    return f_r @ E.conj() / E.shape[0]


def projections(beta_k: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """lambda_n(nu) = sum_G conj(beta_n(k+G)) C_nu(G)  (Eq. lambdah).  Returns (nb, nkb)."""
    return psi @ beta_k.conj().T


def hpsi_direct(prob, ik: int, psi_k: np.ndarray, E=None) -> np.ndarray:
    """H|psi> by the paper's route with direct sums in place of FFTs.

    kinetic (Sec. 2.2.1) + [inverse transform -> V(r) u(r) -> forward transform] (Sec. 2.2.2)
    + nonlocal by lambda (Eq. lambdah), gamma = D lambda (Eq. gamma), add-back (Eq. finalnl)."""
    n = int(prob.npw[ik])
    m = prob.miller[ik, :n]
    C = psi_k[:, :n].astype(np.complex128)
    if E is None:
        E = phase_matrix(m, prob.N)
    out = kinetic(prob.kpts[ik], m, prob.B)[None, :] * C
    u = to_real_space(C, E)
    out = out + to_reciprocal(u * prob.V_r.ravel()[None, :], E)
    beta_k = prob.beta[ik, :, :n]
    lam = projections(beta_k, C)            # (nb, nkb)
    gam = lam @ prob.D.T                    # gamma_m = sum_n D_mn lambda_n
    out = out + gam @ beta_k                # sum_m gamma_m beta_m(k+G)
    res = np.zeros_like(psi_k, dtype=np.complex128)
    res[:, :n] = out
    return res


def relative_error(a: np.ndarray, b: np.ndarray, axis=-1) -> np.ndarray:
    """||a - b||_2 / ||b||_2 along the coefficient axis (per band-k)."""
    return np.linalg.norm(a - b, axis=axis) / np.maximum(np.linalg.norm(b, axis=axis), 1e-300)
