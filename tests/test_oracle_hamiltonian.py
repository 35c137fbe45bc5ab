"""Pins of the H|psi> oracle against facts fixed by the paper and by mathematics (no GPU).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign
in an exponent, a transposed or un-conjugated operand, a missing 1/N_r) fails it.
"""
import math
import os

import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import davidson as dav
from paper_2412_01695_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _free(prob):
    prob.V_r = np.zeros_like(prob.V_r)
    prob.D = np.zeros_like(prob.D)
    return prob


def test_free_electron_eigenvalues_closed_form():
    """V = 0, D = 0: eps = (2pi/a)^2 n/16 from the hand-derived golden table (Sec. 2.2.1)."""
    prob = _free(synth.make_config(1, with_psi=False))
    H = ham.problem_h(prob, 0)
    w = np.linalg.eigvalsh(H)
    rows = np.loadtxt(os.path.join(GOLDEN, "free_electron_fcc_k0.txt"))
    expect = (2 * math.pi / 7.5) ** 2 * rows[:, 1] / 16.0
    np.testing.assert_allclose(w[:len(expect)], expect, rtol=0, atol=1e-12)
    # H is exactly diagonal: kinetic only
    assert np.count_nonzero(H - np.diag(np.diag(H))) == 0


def test_kinetic_energy_of_named_plane_waves():
    """|k+G|^2 for named Miller indices at the first MP point against the hand-derived table
    (Sec. 2.2.1).  G and -G differ there, so |k-G|^2 fails it while the free-electron
    spectrum above (the sphere mapped onto its inversion) would not."""
    prob = synth.make_config(1, with_psi=False)
    unit = 2 * math.pi / 7.5
    np.testing.assert_allclose(prob.kpts[0], -unit / 4 * np.ones(3), rtol=0, atol=1e-14)
    rows = np.loadtxt(os.path.join(GOLDEN, "kinetic_fcc_k0_named_g.txt"))
    g2 = ham.kinetic(prob.kpts[0], rows[:, :3].astype(np.int64), prob.B)
    np.testing.assert_allclose(g2, unit ** 2 * rows[:, 3] / 16.0, rtol=0, atol=1e-12)


def test_free_electron_hpsi_exact(cfg1):
    prob = _free(synth.make_config(1))
    for ik in range(prob.nk):
        n = prob.npw[ik]
        out = ham.hpsi_direct(prob, ik, prob.psi[ik])
        g2 = ham.kinetic(prob.kpts[ik], prob.miller[ik, :n], prob.B)
        ref = prob.psi[ik][:, :n] * g2[None, :]
        assert np.max(np.abs(out[:, :n] - ref)) < 1e-13 * np.max(np.abs(ref))


def test_constant_potential_rigid_shift():
    """V(r) = c shifts H by c exactly and every eigenvalue by c (Sec. 2.2.2 with V_eff = c)."""
    prob = synth.make_config(1, with_psi=False)
    H0 = ham.problem_h(prob, 3)
    c = 0.731
    prob.V_r = prob.V_r + c
    H1 = ham.problem_h(prob, 3)
    np.testing.assert_allclose(H1 - H0, c * np.eye(len(H0)), atol=1e-13)
    w0, w1 = np.linalg.eigvalsh(H0), np.linalg.eigvalsh(H1)
    np.testing.assert_allclose(w1 - w0, c, atol=1e-12)


def test_single_wave_couplings():
    """V(r) = v e^{iG0.r} + c.c. couples G and G' only when m - m' = +-m0, with V~ = v for
    m - m' = m0 and conj(v) for m - m' = -m0 (Sec. 2.2.2 and Eq. fwFFT, 1/N_r included)."""
    prob = synth.make_config(1, with_psi=False)
    N = prob.N
    m0 = np.array([1, -2, 1])
    v = 0.3 - 0.7j
    l = np.indices((N, N, N)).reshape(3, -1).T
    V_r = 2 * np.real(v * np.exp(2j * np.pi * (l @ m0) / N)).reshape(N, N, N)
    vt = ham.grid_coefficients(V_r)
    n = prob.npw[0]
    m = prob.miller[0, :n]
    M = ham.local_matrix(m, m, vt)
    d = m[:, None, :] - m[None, :, :]
    plus = np.all(d == m0, axis=-1)
    minus = np.all(d == -m0, axis=-1)
    assert plus.sum() > 10 and minus.sum() > 10
    np.testing.assert_allclose(M[plus], v, atol=1e-13)
    np.testing.assert_allclose(M[minus], np.conj(v), atol=1e-13)
    assert np.max(np.abs(M[~(plus | minus)])) < 1e-13


def test_roundtrip_normalisation():
    """Forward(inverse(C)) = C: the 1/N_r of Eq. fwFFT against the unnormalised inverse."""
    prob = synth.make_config(1)
    n = prob.npw[2]
    E = ham.phase_matrix(prob.miller[2, :n], prob.N)
    C = prob.psi[2][:, :n]
    back = ham.to_reciprocal(ham.to_real_space(C, E), E)
    np.testing.assert_allclose(back, C, atol=1e-13)


def test_dense_equals_direct_sums(cfg1):
    """The dense convolution route and the paper's transform route agree (<= 1e-13 rel.)."""
    vt = ham.grid_coefficients(cfg1.V_r)
    for ik in range(cfg1.nk):
        a = ham.hpsi_dense(cfg1, ik, cfg1.psi[ik], vt)
        b = ham.hpsi_direct(cfg1, ik, cfg1.psi[ik])
        assert np.max(ham.relative_error(a, b)) < 1e-13


def test_hermiticity(cfg1):
    """<phi|H psi> = conj <psi|H phi> through the direct-sum route; dense H is Hermitian."""
    H = ham.problem_h(cfg1, 5)
    assert np.max(np.abs(H - H.conj().T)) < 1e-13 * np.max(np.abs(H))
    psi = cfg1.psi[5]
    hp = ham.hpsi_direct(cfg1, 5, psi)
    G = psi.conj() @ hp.T            # G_ij = <psi_i|H psi_j>
    np.testing.assert_allclose(G, G.conj().T, atol=1e-12)


def test_translation_invariance():
    """Moving the atom and V(r) together by a grid vector leaves the spectrum unchanged.
    Catches a sign or conjugation slip between the local and nonlocal terms
    (structure factor e^{-i(k+G).tau} of beta against e^{-iG.r} of Eq. fwFFT)."""
    p0 = synth.make_config(1, with_psi=False)
    N = p0.N
    j = np.array([3, 5, 1])
    t = (j / N) @ p0.A
    V_shift = np.roll(p0.V_r, shift=tuple(j), axis=(0, 1, 2))   # V'(r) = V(r - t)
    p1 = synth.build_problem(p0.A, p0.tau + t, p0.lset, N, p0.ecut, p0.kpts, p0.nb, 1,
                             V_r=V_shift, D=p0.D, with_psi=False)
    for ik in (0, 6):
        w0 = np.linalg.eigvalsh(ham.problem_h(p0, ik))
        w1 = np.linalg.eigvalsh(ham.problem_h(p1, ik))
        np.testing.assert_allclose(w1, w0, atol=1e-11)
    # and a non-grid-consistent move must change it (the check has teeth)
    p2 = synth.build_problem(p0.A, p0.tau - t, p0.lset, N, p0.ecut, p0.kpts, p0.nb, 1,
                             V_r=V_shift, D=p0.D, with_psi=False)
    w2 = np.linalg.eigvalsh(ham.problem_h(p2, 0))
    assert np.max(np.abs(w2 - np.linalg.eigvalsh(ham.problem_h(p0, 0)))) > 1e-4


def test_time_reversal(cfg1):
    """Real V and beta(-q) = conj beta(q): eps(-k) = eps(k) over the symmetric MP grid."""
    k = cfg1.kpts
    vt = ham.grid_coefficients(cfg1.V_r)
    for ik in range(cfg1.nk):
        jk = int(np.argmin(np.linalg.norm(k + k[ik], axis=1)))
        assert np.linalg.norm(k[jk] + k[ik]) < 1e-12
        w0 = np.linalg.eigvalsh(ham.problem_h(cfg1, ik, vt))
        w1 = np.linalg.eigvalsh(ham.problem_h(cfg1, jk, vt))
        np.testing.assert_allclose(w0, w1, atol=1e-11)


def _secular_roots(poles, weights, d, count):
    """Roots of 1 = d sum_j w_j/(eps - p_j) by bisection, plus the poles that keep
    multiplicity (a projector couples one combination per degenerate level)."""
    p = np.array(poles)
    w = np.array(weights)

    def f(e):
        return 1.0 - d * np.sum(w / (e - p))

    roots = []
    order = np.argsort(p)
    p, w = p[order], w[order]
    brackets = []
    if d < 0:
        lo = p[0] - 1.0
        while f(lo) < 0:
            lo -= 2 * (p[0] - lo)
        brackets.append((lo, p[0]))
    for i in range(len(p) - 1):
        brackets.append((p[i], p[i + 1]))
    for a, b in brackets:
        eps_a, eps_b = a + 1e-14 * max(1, abs(a)), b - 1e-14 * max(1, abs(b))
        fa, fb = f(eps_a), f(eps_b)
        if fa * fb > 0:
            continue
        for _ in range(200):
            mid = 0.5 * (eps_a + eps_b)
            if f(mid) * fa > 0:
                eps_a, fa = mid, f(mid)
            else:
                eps_b = mid
        roots.append(0.5 * (eps_a + eps_b))
    return np.sort(np.array(roots))[:count]


def test_secular_equation_single_projector():
    """Free electrons plus one s projector with D = d: eigenvalues solve
    1 = d sum_G |beta(k+G)|^2/(eps - |k+G|^2) (closed form of Eqs. lambdah-finalnl)."""
    A, tau = synth.cell_for(1)
    B = synth.reciprocal_rows(A)
    k = synth.mp_grid(B, (2, 2, 2))[[1]]
    d = -400.0   # |beta|^2 carries 1/Omega: a strong coupling gives a clear bound state
    p = synth.build_problem(A, tau, (0,), 16, 20.0, k, 8, 1, V_r=np.zeros((16, 16, 16)),
                            D=np.array([[d]]), with_psi=False)
    n = p.npw[0]
    H = ham.problem_h(p, 0)
    w = np.linalg.eigvalsh(H)
    g2 = ham.kinetic(p.kpts[0], p.miller[0, :n], p.B)
    b2 = np.abs(p.beta[0, 0, :n]) ** 2
    # group degenerate kinetic levels
    key = np.round(g2, 9)
    levels, inv, mult = np.unique(key, return_inverse=True, return_counts=True)
    poles = np.array([g2[inv == j].mean() for j in range(len(levels))])
    weights = np.array([b2[inv == j].sum() for j in range(len(levels))])
    roots = _secular_roots(poles, weights, d, 6)
    kept = np.concatenate([np.full(mult[j] - (1 if weights[j] > 0 else 0), poles[j])
                           for j in range(len(levels))])
    expect = np.sort(np.concatenate([roots, kept]))[:6]
    np.testing.assert_allclose(w[:6], expect, atol=1e-10)
    assert w[0] < poles.min() - 1e-3   # a bound state below the free-electron bottom


def test_davidson_matches_dense(cfg1):
    """The Davidson iteration of Sec. 2.1 reaches the lowest eigenpairs of the dense H(k)."""
    vt = ham.grid_coefficients(cfg1.V_r)
    for ik in (0, 4):
        n = cfg1.npw[ik]
        H = ham.problem_h(cfg1, ik, vt)
        w_ref, v_ref = dav.lowest_eigenpairs(H, cfg1.nb)
        eps, psi, it, napply, conv = dav.davidson(lambda X: X @ H.T, np.real(np.diag(H)),
                                                  cfg1.psi[ik][:, :n], eth=1e-11, max_iter=200,
                                                  res_tol=1e-7)
        assert conv.all()
        np.testing.assert_allclose(eps, w_ref, atol=1e-9)
        P1 = psi.T @ psi.conj()
        P0 = v_ref.T @ v_ref.conj()
        assert np.linalg.norm(P1 - P0) < 1e-6
        assert napply > cfg1.nb


def test_davidson_restart_path(cfg1):
    """A basis cap of nb + 2 forces restarts every step; the result is unchanged."""
    vt = ham.grid_coefficients(cfg1.V_r)
    n = cfg1.npw[1]
    H = ham.problem_h(cfg1, 1, vt)
    w_ref, _ = dav.lowest_eigenpairs(H, 4)
    eps, psi, it, napply, conv = dav.davidson(lambda X: X @ H.T, np.real(np.diag(H)),
                                              cfg1.psi[1][:4, :n], eth=1e-11, max_iter=500,
                                              max_basis=8, res_tol=1e-7)
    assert conv.all()
    np.testing.assert_allclose(eps, w_ref, atol=1e-9)


def test_davidson_free_electron_degenerate():
    """V = D = 0: H is diagonal and the diagonal preconditioner is exact, so the preconditioned
    residual is parallel to the Ritz vector; the iteration still reaches the degenerate
    free-electron levels (closed form of the golden table)."""
    prob = _free(synth.make_config(1))
    H = ham.problem_h(prob, 0)
    n = prob.npw[0]
    eps, psi, it, napply, conv = dav.davidson(lambda X: X @ H.T, np.real(np.diag(H)),
                                              prob.psi[0][:, :n], eth=1e-11, max_iter=300,
                                              res_tol=1e-7)
    rows = np.loadtxt(os.path.join(GOLDEN, "free_electron_fcc_k0.txt"))
    expect = (2 * math.pi / 7.5) ** 2 * rows[:prob.nb, 1] / 16.0
    assert conv.all()
    np.testing.assert_allclose(eps, expect, atol=1e-9)


def test_rayleigh_ritz_on_rotated_eigenvectors(cfg1):
    """The reduced problem of Sec. 2.1 on a basis that spans an exact invariant subspace: six
    eigenvectors of the dense H(k) mixed by a random complex unitary.  Its reduced overlap
    <phi_i|phi_j> is the identity (the basis is orthonormal in the Hermitian product), and
    its Ritz values are the six exact eigenvalues."""
    vt = ham.grid_coefficients(cfg1.V_r)
    H = ham.problem_h(cfg1, 2, vt)
    w, V = np.linalg.eigh(H)
    rng = np.random.default_rng(8)
    U = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))[0]
    phi = U @ V[:, :6].T                     # rows: an orthonormal complex basis
    Hr, Sr = dav._reduced(phi, phi @ H.T, phi)
    np.testing.assert_allclose(Sr, np.eye(6), atol=1e-12)
    np.testing.assert_allclose(np.linalg.eigvalsh(Hr), w[:6], atol=1e-10)
    eps, vecs = dav._reduced_eig(Hr, Sr, 4)
    np.testing.assert_allclose(eps, w[:4], atol=1e-10)
