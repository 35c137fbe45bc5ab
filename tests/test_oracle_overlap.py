"""Pins of the overlap (ultrasoft/PAW S) oracle against closed forms and invariants (no GPU).

Each test is chosen so that a plausible slip (q transposed or dropped, beta un-conjugated,
the identity term missing, the S P_v S projector written without S, the residual of the
generalized Davidson taken without S) fails at least one of them.
"""
import numpy as np

from oracle import davidson as dav
from oracle import hamiltonian as ham
from oracle import overlap as ov
from oracle import sternheimer as st
from paper_2412_01695_gb300 import synth


def _cell1(k_index=0, q=None, D=None, lset=(0, 1), V=True):
    prob = synth.make_config(1, k_subset=[k_index], with_psi=False)
    if not V:
        prob.V_r = np.zeros_like(prob.V_r)
    if D is not None:
        prob.D = D
    q = synth.q_for(1) if q is None else q
    return prob, q


def test_q_zero_is_identity():
    prob, _ = _cell1()
    n = prob.npw[0]
    S = ov.overlap_matrix(prob.beta[0][:, :n], np.zeros((prob.nkb, prob.nkb)))
    assert np.array_equal(S, np.eye(n))


def test_steps_equal_dense_and_hermitian_positive():
    """Eqs. lambdah, delta_eq, finals composed equal the dense S; S is Hermitian and >= 1
    for positive semi-definite q."""
    prob, q = _cell1(3)
    n = prob.npw[0]
    b = prob.beta[0][:, :n]
    S = ov.overlap_matrix(b, q)
    rng = np.random.default_rng(5)
    X = rng.normal(size=(4, n)) + 1j * rng.normal(size=(4, n))
    np.testing.assert_allclose(ov.spsi_steps(b, q, X), X @ S.T, atol=1e-13)
    assert np.max(np.abs(S - S.conj().T)) < 1e-15
    w = np.linalg.eigvalsh(S)
    assert w.min() > 1 - 1e-12 and w.max() > 1.1   # the q term is not negligible


def test_single_projector_rank_one():
    """One projector, scalar q: S beta = (1 + q |beta|^2) beta and S x = x for x orthogonal
    to beta (the only eigenvalues are 1 and 1 + q |beta|^2)."""
    prob, _ = _cell1()
    n = prob.npw[0]
    b = prob.beta[0][:1, :n]
    qs = 37.0
    S = ov.overlap_matrix(b, np.array([[qs]]))
    v = b[0].copy()                                   # the vector beta(k+G) itself
    nb2 = np.vdot(v, v).real
    np.testing.assert_allclose(S @ v, (1 + qs * nb2) * v, rtol=1e-13)
    rng = np.random.default_rng(1)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    x -= v * np.vdot(v, x) / nb2
    np.testing.assert_allclose(S @ x, x, atol=1e-13)
    w = np.linalg.eigvalsh(S)
    np.testing.assert_allclose(w[-1], 1 + qs * nb2, rtol=1e-12)
    np.testing.assert_allclose(w[:-1], 1.0, atol=1e-12)


def _pencil_roots(poles, weights, d, qs, count):
    """Roots of 1 = (eps q - d) sum_j w_j / (p_j - eps) below the count-th pole, by
    sign changes on a fine grid and bisection."""
    order = np.argsort(poles)
    p, w = np.asarray(poles)[order], np.asarray(weights)[order]

    def f(e):
        return 1.0 - (e * qs - d) * np.sum(w / (p - e))

    edges = [p[0] - 50.0] + list(p[:count + 1])
    roots = []
    for a, b in zip(edges[:-1], edges[1:]):
        xs = np.linspace(a + 1e-9, b - 1e-9, 4001)
        fs = np.array([f(x) for x in xs])
        for i in np.nonzero(np.sign(fs[:-1]) * np.sign(fs[1:]) < 0)[0]:
            lo, hi = xs[i], xs[i + 1]
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if np.sign(f(mid)) == np.sign(f(lo)):
                    lo = mid
                else:
                    hi = mid
            roots.append(0.5 * (lo + hi))
    return np.array(roots)


def test_generalized_secular_equation_single_projector():
    """Free electrons, one s projector with D = d and q: the eigenvalues of H x = eps S x
    off the kinetic levels solve 1 = (eps q - d) sum_G |beta(k+G)|^2 / (|k+G|^2 - eps)."""
    A, tau = synth.cell_for(1)
    B = synth.reciprocal_rows(A)
    k = synth.mp_grid(B, (2, 2, 2))[[1]]
    d, qs = -400.0, 60.0
    p = synth.build_problem(A, tau, (0,), 16, 20.0, k, 8, 1, V_r=np.zeros((16, 16, 16)),
                            D=np.array([[d]]), with_psi=False)
    n = p.npw[0]
    H = ham.problem_h(p, 0)
    S = ov.overlap_matrix(p.beta[0][:, :n], np.array([[qs]]))
    w, _ = ov.lowest_generalized(H, S, 8)
    g2 = ham.kinetic(p.kpts[0], p.miller[0, :n], p.B)
    b2 = np.abs(p.beta[0, 0, :n]) ** 2
    key = np.round(g2, 9)
    levels, inv, mult = np.unique(key, return_inverse=True, return_counts=True)
    poles = np.array([g2[inv == j].mean() for j in range(len(levels))])
    weights = np.array([b2[inv == j].sum() for j in range(len(levels))])
    roots = _pencil_roots(poles, weights, d, qs, 4)
    kept = np.concatenate([np.full(mult[j] - (1 if weights[j] > 0 else 0), poles[j])
                           for j in range(len(levels))])
    expect = np.sort(np.concatenate([roots, kept]))[:6]
    np.testing.assert_allclose(w[:6], expect, atol=1e-9)
    # the same H with S = 1 has a different spectrum: the q term matters
    assert abs(np.linalg.eigvalsh(H)[0] - w[0]) > 1e-3


def test_generalized_davidson_reaches_dense():
    """The Davidson of Sec. 2.1 with S (S~, (H - eps S) phi, H_diag - eps S_diag) reaches the
    lowest eigenpairs of H x = eps S x; its vectors are S-orthonormal."""
    prob, q = _cell1(2)
    prob.psi = None
    n = prob.npw[0]
    H = ham.problem_h(prob, 0)
    S = ov.overlap_matrix(prob.beta[0][:, :n], q)
    nb = 6
    w_ref, v_ref = ov.lowest_generalized(H, S, nb)
    rng = np.random.default_rng(3)
    psi0 = np.linalg.qr(rng.normal(size=(n, nb)) + 1j * rng.normal(size=(n, nb)))[0].T
    eps, psi, it, napply, conv = dav.davidson(lambda X: X @ H.T, np.real(np.diag(H)), psi0,
                                              eth=1e-11, max_iter=300, res_tol=1e-7,
                                              apply_s=lambda X: X @ S.T, s_diag=np.real(np.diag(S)))
    assert conv.all()
    np.testing.assert_allclose(eps, w_ref, atol=1e-9)
    np.testing.assert_allclose(psi.conj() @ S @ psi.T, np.eye(nb), atol=1e-9)
    # the plain (S = 1) eigenvalues differ: the iteration really solved the pencil
    assert np.max(np.abs(np.linalg.eigvalsh(H)[:nb] - w_ref)) > 1e-3


def test_sternheimer_operator_closed_forms():
    """With exact S-orthonormal eigenvectors u_v of (H, S): A u_v = (eps_v + alpha - eps) S u_v,
    <u_v|b> = 0, the solution is S-orthogonal to every u_v, and q = 0 gives the
    norm-conserving operator and right-hand side."""
    prob, q = _cell1(1)
    n = prob.npw[0]
    H = ham.problem_h(prob, 0)
    S = ov.overlap_matrix(prob.beta[0][:, :n], q)
    nocc = 4
    e_occ, u = ov.lowest_generalized(H, S, nocc)
    eps, alpha = e_occ[1], 0.7
    A = ov.operator(H, S, u, eps, alpha)
    for v in range(nocc):
        np.testing.assert_allclose(A @ u[v], (e_occ[v] + alpha - eps) * (S @ u[v]), atol=1e-11)
    rng = np.random.default_rng(9)
    dvpsi = rng.normal(size=(1, n)) + 1j * rng.normal(size=(1, n))
    b = ov.rhs(dvpsi, S, u)
    assert np.max(np.abs(u.conj() @ b[0])) < 1e-12
    x = np.linalg.solve(A, b[0])
    assert np.max(np.abs(u.conj() @ S @ x)) < 1e-10 * np.linalg.norm(x)
    # S = 1 reduces to the norm-conserving forms
    I = np.eye(n)
    w0, u0 = np.linalg.eigh(H)
    u0 = u0[:, :nocc].T
    np.testing.assert_allclose(ov.operator(H, I, u0, eps, alpha), st.operator(H, u0, eps, alpha), atol=1e-13)
    np.testing.assert_allclose(ov.rhs(dvpsi, I, u0), st.rhs(dvpsi, u0), atol=1e-13)


def test_s_orthonormal_inputs():
    prob, q = _cell1(5)
    n = prob.npw[0]
    S = ov.overlap_matrix(prob.beta[0][:, :n], q)
    rng = np.random.default_rng(2)
    X = ov.s_orthonormal(S, rng.normal(size=(5, n)) + 1j * rng.normal(size=(5, n)))
    np.testing.assert_allclose(X.conj() @ S @ X.T, np.eye(5), atol=1e-12)


def test_solution_is_the_first_order_eigenvector_change():
    """First-order perturbation theory for the pencil (H + delta dV, S) with dS = 0 and q = 0:
    the S-conduction part (1 - P_v S) of d u_n / d delta (central difference of the dense
    generalized eigenvectors, gauge <u_n(0)|S|u_n(delta)> real) is the solution of the
    generalized Eq. linear_system.  Fixes the right-hand side's sign and its (1 - S P_v) form."""
    import scipy.linalg
    prob, q = _cell1(3)
    n = prob.npw[0]
    m = prob.miller[0, :n]
    H = ham.problem_h(prob, 0)
    S = ov.overlap_matrix(prob.beta[0][:, :n], q)
    rng = np.random.default_rng(11)
    dv_r = rng.normal(size=(prob.N,) * 3)               # any real periodic potential change
    dvt = ham.grid_coefficients(dv_r)
    M = ham.local_matrix(m, m, dvt)
    w, V = scipy.linalg.eigh(H, S)
    nocc = 4
    u = V[:, :nocc].T
    alpha = 0.9
    dvpsi = st.dv_psi_dense(m, m, dvt, u)
    gaps = np.minimum(np.diff(w, prepend=-np.inf)[:nocc], np.diff(w)[:nocc])
    picked = [j for j in range(nocc) if gaps[j] > 1e-3]
    assert len(picked) >= 2
    h = 1e-5

    def vec(sign, j):
        v = scipy.linalg.eigh(H + sign * h * M, S)[1][:, j]
        ph = np.vdot(u[j], S @ v)
        return v * (abs(ph) / ph)

    for j in picked:
        d = (vec(1, j) - vec(-1, j)) / (2 * h)
        fd = d - u.T @ (u.conj() @ (S @ d))
        x = np.linalg.solve(ov.operator(H, S, u, w[j], alpha), ov.rhs(dvpsi[j][None, :], S, u)[0])
        assert np.linalg.norm(fd - x) < 1e-6 * np.linalg.norm(x)
