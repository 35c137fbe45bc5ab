"""Seeded synthetic inputs for the many-k H|psi> path.

This module builds problem *inputs* only: lattices, Monkhorst-Pack k-grids,
the plane-wave sphere of every k (Miller indices), the local potential on the
real-space grid, the projector table beta_i(k+G), the D coefficients, trial
wave-functions and the DFPT potential change.  It holds none of the arithmetic
of the method itself (no kinetic term, no Fourier transform of a wave-function,
no projection, no eigensolver, no CG).  Both the CPU oracle and the CUDA path
are fed from here; neither is imported by this module.

Conventions (Rydberg atomic units, lengths in bohr, energies in Ry):
  * lattice vectors a_i are the rows of A; reciprocal vectors b_i are the rows
    of B with a_i . b_j = 2 pi delta_ij (paper Sec. 4, Miller mesh G_{m1,m2,m3});
  * the basis of k is every G = m1 b1 + m2 b2 + m3 b3 with |k+G|^2 < ecut (Ry),
    the Rydberg form of the paper's cut-off (Sec. 2.2.1, 1/2|k+G|^2 < E_cut in Ha);
  * the real-space grid is r_l = sum_i (l_i/N_i) a_i (Sec. 4), arrays indexed
    [l1][l2][l3] with l3 fastest;
  * V(r) = sum_G V(G) e^{iG.r} is real; projectors follow
      beta_{I,lm}(q) = Omega^{-1/2} (-i)^l P_lm(q) exp(-|q|^2/4) exp(-i q.tau_I),
    q = k+G, P_lm the real solid harmonic (|q|^l Y_lm(q^)), order
    l=0; l=1 (x, y, z); l=2 (xy, yz, 3z^2-r^2, xz, x^2-y^2).
Seeds: seed = 2412016950 + 100*cfg + stream, stream V=0, beta=1 (unused: the
table is deterministic), D=2, psi=3, dv=4, tau=5; numpy PCG64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

SEED_BASE = 2412016950
STREAMS = {"V": 0, "beta": 1, "D": 2, "psi": 3, "dv": 4, "tau": 5, "q": 6}


def rng_for(cfg_id: int, stream: str) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 100 * cfg_id + STREAMS[stream]))


# ----------------------------------------------------------------------------- geometry
def fcc_lattice(a: float) -> np.ndarray:
    return 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])


def sc_lattice(a: float) -> np.ndarray:
    return a * np.eye(3)


def reciprocal_rows(A: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(A).T


def mp_grid(B: np.ndarray, q: Sequence[int]) -> np.ndarray:
    """Unreduced Monkhorst-Pack grid, u_r = (2r - q - 1)/(2q), r = 1..q (cartesian, bohr^-1).

    Ordered with the first reduced coordinate slowest."""
    us = [np.array([(2 * r - qi - 1) / (2.0 * qi) for r in range(1, qi + 1)]) for qi in q]
    u = np.array(np.meshgrid(*us, indexing="ij")).reshape(3, -1).T
    return u @ B


def gsphere(kc: np.ndarray, B: np.ndarray, ecut: float, A: np.ndarray):
    """Miller indices of every G with |k+G|^2 < ecut, sorted by (|k+G|^2, m1, m2, m3).

    Returns (miller[n,3] int32, margin) where margin is the smallest distance of
    |k+G|^2 to ecut over all candidate G (basis membership is never a tie)."""
    kmax = math.sqrt(ecut) + np.linalg.norm(kc)
    nmax = [int(math.floor(kmax * np.linalg.norm(A[i]) / (2 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-n, n + 1) for n in nmax]
    m = np.array(np.meshgrid(*r, indexing="ij")).reshape(3, -1).T
    g2 = np.sum((kc[None, :] + m @ B) ** 2, axis=1)
    margin = float(np.min(np.abs(g2 - ecut)))
    sel = g2 < ecut
    m, g2 = m[sel], g2[sel]
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], g2))
    return m[order].astype(np.int32), margin


# ----------------------------------------------------------------------------- projectors
def solid_harmonics(q: np.ndarray, lmax: int) -> list:
    """Real solid harmonics |q|^l Y_lm(q^) for l <= lmax, list over l of (2l+1, n) arrays."""
    x, y, z = q[:, 0], q[:, 1], q[:, 2]
    out = [np.full((1, len(q)), 1.0 / math.sqrt(4 * math.pi))]
    if lmax >= 1:
        c1 = math.sqrt(3.0 / (4 * math.pi))
        out.append(c1 * np.stack([x, y, z]))
    if lmax >= 2:
        c2 = math.sqrt(15.0 / (4 * math.pi))
        c20 = math.sqrt(5.0 / (16 * math.pi))
        c22 = math.sqrt(15.0 / (16 * math.pi))
        r2 = x * x + y * y + z * z
        out.append(np.stack([c2 * x * y, c2 * y * z, c20 * (3 * z * z - r2), c2 * x * z,
                             c22 * (x * x - y * y)]))
    return out


def projector_layout(nat: int, lset: Sequence[int]):
    """(atom, l) of every projector; atoms slowest, then l, then m."""
    atom, ls = [], []
    for ia in range(nat):
        for l in lset:
            for _ in range(2 * l + 1):
                atom.append(ia)
                ls.append(l)
    return np.array(atom, np.int32), np.array(ls, np.int32)


def beta_table(kc, miller, B, tau, lset, omega) -> np.ndarray:
    """beta_i(k+G) for every projector i and basis G of one k: complex (nkb, npw)."""
    q = kc[None, :] + miller @ B
    q2 = np.sum(q * q, axis=1)
    radial = np.exp(-q2 / 4.0)
    sh = solid_harmonics(q, max(lset))
    rows = []
    for t in tau:
        phase = np.exp(-1j * (q @ t))
        for l in lset:
            for p in sh[l]:
                rows.append(((-1j) ** l) * p * radial * phase / math.sqrt(omega))
    return np.array(rows, np.complex128)


def random_D(rng: np.random.Generator, nat: int, lset: Sequence[int]) -> np.ndarray:
    """Block-diagonal real symmetric D (Ry): one U(-1,1) symmetric block per atom."""
    npa = sum(2 * l + 1 for l in lset)
    D = np.zeros((nat * npa, nat * npa))
    for ia in range(nat):
        blk = rng.uniform(-1.0, 1.0, size=(npa, npa))
        blk = np.triu(blk) + np.triu(blk, 1).T
        D[ia * npa:(ia + 1) * npa, ia * npa:(ia + 1) * npa] = blk
    return D


def random_q(rng: np.random.Generator, nat: int, lset: Sequence[int], scale: float = 20.0) -> np.ndarray:
    """Block-diagonal real symmetric positive semi-definite q (ultrasoft/PAW augmentation
    coefficients): one block scale * R R^T / n per atom, R with U(-1,1) entries.  With the
    Gaussian projectors of this generator S = 1 + sum beta q beta^* then has eigenvalues in
    about [1, 3]; positive semi-definite q keeps S positive definite for any projector set."""
    npa = sum(2 * l + 1 for l in lset)
    q = np.zeros((nat * npa, nat * npa))
    for ia in range(nat):
        R = rng.uniform(-1.0, 1.0, size=(npa, npa))
        q[ia * npa:(ia + 1) * npa, ia * npa:(ia + 1) * npa] = scale * (R @ R.T) / npa
    return q


def q_for(cfg: int) -> np.ndarray:
    """The augmentation coefficients q of a synthetic cell (ultrasoft/PAW variant)."""
    c = CONFIGS[cfg]
    _, tau = cell_for(cfg)
    return random_q(rng_for(cfg, "q"), len(tau), c["lset"])


# ----------------------------------------------------------------------------- fields on the grid
def _fourier_candidates(B, N, ecut_rho):
    h = (N - 1) // 2  # strictly |m_i| < N/2: no Nyquist plane
    r = np.arange(-h, h + 1)
    m = np.array(np.meshgrid(r, r, r, indexing="ij")).reshape(3, -1).T
    g2 = np.sum((m @ B) ** 2, axis=1)
    return m, g2


def _synthesise(coef_m: np.ndarray, coef: np.ndarray, N: int) -> np.ndarray:
    """f(l) = sum_m c(m) e^{2 pi i m.l/N} on the N^3 grid (separable direct sums)."""
    grid = np.zeros((N, N, N), np.complex128)
    mm = np.mod(coef_m, N)
    np.add.at(grid, (mm[:, 0], mm[:, 1], mm[:, 2]), coef)
    l = np.arange(N)
    E = np.exp(2j * np.pi * np.outer(l, l) / N)
    return np.einsum("ai,bj,ck,ijk->abc", E, E, E, grid, optimize=True)


def vloc_grid(rng, B, N, ecut, amp=1.0, v0=0.0):
    """Real V(r) on the grid from V(G) = amp (x+iy)/sqrt2 exp(-|G|^2/8), 0<|G|^2<4 ecut,
    V(-G) = conj V(G), V(0) = v0.  Returns (V_r float64 [N,N,N], miller, V(G))."""
    m, g2 = _fourier_candidates(B, N, 4 * ecut)
    half = (m[:, 0] > 0) | ((m[:, 0] == 0) & (m[:, 1] > 0)) | \
           ((m[:, 0] == 0) & (m[:, 1] == 0) & (m[:, 2] > 0))
    sel = half & (g2 < 4 * ecut) & (g2 > 0)
    mh, g2h = m[sel], g2[sel]
    xy = rng.standard_normal((len(mh), 2))
    c = amp * (xy[:, 0] + 1j * xy[:, 1]) / math.sqrt(2.0) * np.exp(-g2h / 8.0)
    ms = np.concatenate([mh, -mh, np.zeros((1, 3), np.int64)])
    cs = np.concatenate([c, np.conj(c), np.array([v0], np.complex128)])
    f = _synthesise(ms, cs, N)
    assert np.max(np.abs(f.imag)) < 1e-12 * max(1.0, np.max(np.abs(f.real)))
    return np.ascontiguousarray(f.real), ms, cs


def dv_grid(rng, B, N, ecut, amp=1.0):
    """Complex lattice-periodic part of the DFPT potential change, dv(r) = sum_G dv(G) e^{iG.r},
    dv(G) = amp (x+iy)/sqrt2 exp(-|G|^2/8) for |G|^2 < 4 ecut (G = 0 included)."""
    m, g2 = _fourier_candidates(B, N, 4 * ecut)
    sel = g2 < 4 * ecut
    m, g2 = m[sel], g2[sel]
    xy = rng.standard_normal((len(m), 2))
    c = amp * (xy[:, 0] + 1j * xy[:, 1]) / math.sqrt(2.0) * np.exp(-g2 / 8.0)
    return _synthesise(m, c, N)


def single_wave_grid(N, m0, coef):
    """f(r) = coef e^{i G0.r} + conj(coef) e^{-i G0.r} for a single Miller index m0 (real field)."""
    ms = np.array([m0, [-x for x in m0]])
    cs = np.array([coef, np.conj(coef)], np.complex128)
    f = _synthesise(ms, cs, N)
    return np.ascontiguousarray(f.real)


# ----------------------------------------------------------------------------- wave-functions
def random_orthonormal(rng, npw: int, npw_max: int, nb: int) -> np.ndarray:
    """nb complex-normal vectors on the first npw coefficients, orthonormalised (modified
    Gram-Schmidt, FP64), zero padding beyond npw.  Returns (nb, npw_max) complex128."""
    X = (rng.standard_normal((nb, npw)) + 1j * rng.standard_normal((nb, npw))) / math.sqrt(2.0)
    for i in range(nb):
        for j in range(i):
            X[i] -= np.vdot(X[j], X[i]) * X[j]
        X[i] /= np.linalg.norm(X[i])
    out = np.zeros((nb, npw_max), np.complex128)
    out[:, :npw] = X
    return out


# ----------------------------------------------------------------------------- problems
@dataclasses.dataclass
class Problem:
    cfg: int
    A: np.ndarray            # (3,3) rows a_i, bohr
    B: np.ndarray            # (3,3) rows b_i, bohr^-1
    omega: float
    tau: np.ndarray          # (nat,3) cartesian bohr
    lset: tuple              # angular momenta of the projectors of one atom
    N: int                   # FFT grid N1 = N2 = N3
    ecut: float              # Ry
    kpts: np.ndarray         # (nk,3) cartesian bohr^-1
    npw: np.ndarray          # (nk,) int32
    npw_max: int
    miller: np.ndarray       # (nk, npw_max, 3) int32, zero padded
    beta: np.ndarray         # (nk, nkb, npw_max) complex128, zero padded
    D: np.ndarray            # (nkb, nkb) float64, block diagonal per atom
    proj_atom: np.ndarray
    proj_l: np.ndarray
    V_r: np.ndarray          # (N,N,N) float64, l3 fastest
    nb: int
    psi: Optional[np.ndarray] = None   # (nk, nb, npw_max) complex128
    margin: float = 0.0

    @property
    def nk(self):
        return len(self.kpts)

    @property
    def nkb(self):
        return self.beta.shape[1]


CONFIGS = {
    1: dict(lattice="fcc", a=7.5, nat=1, ecut=20.0, N=16, nb=8, mp=(2, 2, 2), lset=(0, 1)),
    2: dict(lattice="fcc", a=7.5, nat=1, ecut=45.0, N=24, nb=20, mp=(8, 8, 8), lset=(0, 1, 2)),
    3: dict(lattice="sc4", a=7.5, nat=4, ecut=40.0, N=36, nb=40, mp=(10, 10, 10), lset=(0, 1, 2)),
    4: dict(lattice="fcc", a=7.5, nat=1, ecut=35.0, N=20, nb=12, mp=(16, 16, 16), lset=(0, 1, 2),
            q_frac=(0.25, 0.0, 0.0)),
}


def cell_for(cfg: int):
    c = CONFIGS[cfg]
    a = c["a"]
    if c["lattice"] == "fcc":
        A = fcc_lattice(a)
        tau = np.zeros((1, 3))
    else:
        A = sc_lattice(a)
        tau = a * np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0.0]])
    return A, tau


def qvector(cfg: int) -> np.ndarray:
    c = CONFIGS[cfg]
    return 2 * np.pi / c["a"] * np.array(c.get("q_frac", (0.0, 0.0, 0.0)))


def build_problem(A, tau, lset, N, ecut, kpts, nb, cfg_id, *, V_r=None, D=None,
                  with_psi=True, npw_max=None, vamp=1.0, v0=0.0) -> Problem:
    B = reciprocal_rows(A)
    omega = abs(np.linalg.det(A))
    spheres, margin = [], np.inf
    for kc in kpts:
        m, mg = gsphere(kc, B, ecut, A)
        spheres.append(m)
        margin = min(margin, mg)
    npw = np.array([len(m) for m in spheres], np.int32)
    if npw_max is None:
        npw_max = int(npw.max())
    nk = len(kpts)
    miller = np.zeros((nk, npw_max, 3), np.int32)
    nat = len(tau)
    proj_atom, proj_l = projector_layout(nat, lset)
    nkb = len(proj_atom)
    beta = np.zeros((nk, nkb, npw_max), np.complex128)
    omega_f = float(omega)
    for ik, m in enumerate(spheres):
        miller[ik, :len(m)] = m
        beta[ik, :, :len(m)] = beta_table(kpts[ik], m, B, tau, lset, omega_f)
    if V_r is None:
        V_r = vloc_grid(rng_for(cfg_id, "V"), B, N, ecut, amp=vamp, v0=v0)[0]
    if D is None:
        D = random_D(rng_for(cfg_id, "D"), nat, lset)
    prob = Problem(cfg=cfg_id, A=A, B=B, omega=omega_f, tau=tau, lset=tuple(lset), N=N, ecut=ecut,
                   kpts=np.asarray(kpts, float), npw=npw, npw_max=npw_max, miller=miller, beta=beta,
                   D=D, proj_atom=proj_atom, proj_l=proj_l, V_r=V_r, nb=nb, margin=float(margin))
    if with_psi:
        r = rng_for(cfg_id, "psi")
        prob.psi = np.stack([random_orthonormal(r, int(npw[ik]), npw_max, nb) for ik in range(nk)])
    return prob


def make_config(cfg: int, k_subset=None, with_psi=True, shift_q=False, nb=None, V_r=None,
                D=None) -> Problem:
    """Problem for one of the four synthetic cells.  k_subset picks k indices of the full
    MP grid (the V, D and beta of the full problem are unchanged by sub-setting); shift_q
    gives the k+q set of the DFPT cell.  psi is drawn for the selected k only, in order."""
    c = CONFIGS[cfg]
    A, tau = cell_for(cfg)
    B = reciprocal_rows(A)
    kpts = mp_grid(B, c["mp"])
    if shift_q:
        kpts = kpts + qvector(cfg)[None, :]
    if k_subset is not None:
        kpts = kpts[np.asarray(k_subset)]
    return build_problem(A, tau, c["lset"], c["N"], c["ecut"], kpts, nb or c["nb"], cfg,
                         V_r=V_r, D=D, with_psi=with_psi)


def dv_for(cfg: int, N: int = None) -> np.ndarray:
    c = CONFIGS[cfg]
    A, _ = cell_for(cfg)
    return dv_grid(rng_for(cfg, "dv"), reciprocal_rows(A), N or c["N"], c["ecut"])


def sample_k(nk_total: int, n: int, seed: int = 7) -> np.ndarray:
    """Seeded sorted sample of k indices (includes 0 and the last index)."""
    if n >= nk_total:
        return np.arange(nk_total)
    r = np.random.Generator(np.random.PCG64(SEED_BASE + seed))
    mid = r.choice(np.arange(1, nk_total - 1), size=n - 2, replace=False)
    return np.sort(np.concatenate([[0, nk_total - 1], mid]))
