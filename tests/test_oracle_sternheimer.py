"""Pins of the Sternheimer / PCG oracle (no GPU): dense LU, closed forms, PCG convergence."""
import numpy as np
import scipy.linalg

from oracle import hamiltonian as ham
from oracle import sternheimer as st
from paper_2412_01695_gb300 import synth


def _kq_pair(ks=(0, 1)):
    pk = synth.make_config(4, k_subset=list(ks), with_psi=False)
    pq = synth.make_config(4, k_subset=list(ks), with_psi=False, shift_q=True)
    return pk, pq


def test_dv_dense_equals_direct():
    """dV psi by the circular convolution equals the paper's transform route (direct sums)."""
    pk, pq = _kq_pair((3,))
    dv = synth.dv_for(4)
    dvt = ham.grid_coefficients(dv)
    nk, nq = pk.npw[0], pq.npw[0]
    rng = np.random.default_rng(0)
    psi = rng.standard_normal((3, nk)) + 1j * rng.standard_normal((3, nk))
    a = st.dv_psi_dense(pq.miller[0, :nq], pk.miller[0, :nk], dvt, psi)
    b = st.dv_psi_direct(pq.miller[0, :nq], pk.miller[0, :nk], dv, psi, pk.N)
    assert np.max(ham.relative_error(a, b)) < 1e-13


def test_free_electron_closed_form():
    """V = D = 0: H diagonal, psi_{k+q,v} unit vectors on the lowest G.  Then
    x(G) = b(G) / (|k+q+G|^2 - eps + alpha [G occupied]) exactly (Eq. linear_system)."""
    pk, pq = _kq_pair((5,))
    pq.V_r[:] = 0
    pq.D[:] = 0
    nq = pq.npw[0]
    Hq = ham.problem_h(pq, 0)
    g2 = np.real(np.diag(Hq))
    nocc = 4
    occ = np.argsort(g2)[:nocc]
    psi_kq = np.zeros((nocc, nq), complex)
    psi_kq[np.arange(nocc), occ] = 1.0
    eps, alpha = 0.05, 3.0
    rng = np.random.default_rng(1)
    b = st.rhs(rng.standard_normal(nq) + 1j * rng.standard_normal(nq), psi_kq)
    A = st.operator(Hq, psi_kq, eps, alpha)
    x = st.solve_dense(A, b)
    denom = g2 - eps
    denom[occ] += alpha
    np.testing.assert_allclose(x, b / denom, atol=1e-13)
    assert np.max(np.abs(b[occ])) < 1e-14     # P_c removes the valence components
    # on the valence space the operator is |k+q+G|^2 - eps + alpha (sign of alpha P_v)
    full = rng.standard_normal(nq) + 1j * rng.standard_normal(nq)
    np.testing.assert_allclose(st.solve_dense(A, full), full / denom, atol=1e-13)


def _setup_pair(ik=2, nocc=12):
    pk, pq = _kq_pair((ik,))
    vt = ham.grid_coefficients(pk.V_r)
    Hk = ham.problem_h(pk, 0, vt)
    Hq = ham.problem_h(pq, 0, vt)
    ek, vk = np.linalg.eigh(Hk)
    eq, vq = np.linalg.eigh(Hq)
    return pk, pq, Hk, Hq, ek[:nocc], vk[:, :nocc].T, eq, vq


def test_solution_conduction_space_and_lu_residual():
    """With exact eigenvectors at k+q the solution lies in the conduction space (P_v x = 0)
    and the dense solve has a tiny true residual."""
    pk, pq, Hk, Hq, ek, psik, eq, vq = _setup_pair()
    nocc = 12
    psikq = vq[:, :nocc].T
    dv = synth.dv_for(4)
    dvt = ham.grid_coefficients(dv)
    nk, nq = pk.npw[0], pq.npw[0]
    alpha = st.alpha_pv(ek, eq[:nocc])
    dvpsi = st.dv_psi_dense(pq.miller[0, :nq], pk.miller[0, :nk], dvt, psik)
    for n in (0, 7, 11):
        b = st.rhs(dvpsi[n], psikq)
        A = st.operator(Hq, psikq, ek[n], alpha)
        x = st.solve_dense(A, b)
        assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-12
        assert np.linalg.norm(psikq.conj() @ x) < 1e-10 * np.linalg.norm(x)


def test_pcg_reaches_dense_solution():
    """The PCG of Eqs. ax1-updatedold converges to the LU answer (1e-10 relative residual)."""
    pk, pq, Hk, Hq, ek, psik, eq, vq = _setup_pair(ik=9)
    nocc = 12
    psikq = vq[:, :nocc].T
    dv = synth.dv_for(4)
    dvt = ham.grid_coefficients(dv)
    nk, nq = pk.npw[0], pq.npw[0]
    alpha = st.alpha_pv(ek, eq[:nocc])
    gap = eq[nocc] - ek.max()
    assert gap > 0, "this pair is positive definite on the conduction space"
    g2q = ham.kinetic(pq.kpts[0], pq.miller[0, :nq], pq.B)
    dvpsi = st.dv_psi_dense(pq.miller[0, :nq], pk.miller[0, :nk], dvt, psik)
    for n in (0, 11):
        b = st.rhs(dvpsi[n], psikq)
        A = st.operator(Hq, psikq, ek[n], alpha)
        M = st.preconditioner(g2q, psikq[n])
        x, it = st.pcg(lambda v: A @ v, b, M, thr=1e-24 * np.vdot(b, b).real, max_iter=2000)
        xr = st.solve_dense(A, b)
        assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-10
        assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-8
        assert 2 < it < 2000


def _continued_vector(Hd, j, ref, Sd=None):
    """Eigenvector j of Hd (or of the pencil Hd, Sd), phase fixed so <ref|S|v> is real positive."""
    _, V = np.linalg.eigh(Hd) if Sd is None else scipy.linalg.eigh(Hd, Sd)
    v = V[:, j]
    ph = np.vdot(ref, v if Sd is None else Sd @ v)
    return v * (abs(ph) / ph)


def test_solution_is_the_first_order_eigenvector_change():
    """First-order perturbation theory: for q = 0 and a real dv, the conduction part of
    d psi_n / d delta for H + delta dV (central difference of the dense eigenvectors, gauge
    <psi_n(0)|psi_n(delta)> real) is the solution of Eq. linear_system.  Fixes the sign of its
    right-hand side and that dV enters as <c|dV|n> and not its conjugate."""
    pk = synth.make_config(4, k_subset=[2], with_psi=False)
    n = pk.npw[0]
    m = pk.miller[0, :n]
    H = ham.problem_h(pk, 0)
    dvt = ham.grid_coefficients(np.real(synth.dv_for(4)))
    M = ham.local_matrix(m, m, dvt)
    assert np.max(np.abs(M - M.conj().T)) < 1e-14
    w, V = np.linalg.eigh(H)
    nocc = 12
    psi = V[:, :nocc].T
    alpha = st.alpha_pv(w[:nocc], w[:nocc])
    dvpsi = st.dv_psi_dense(m, m, dvt, psi)
    gaps = np.minimum(np.diff(w, prepend=-np.inf)[:nocc], np.diff(w)[:nocc])
    picked = [j for j in range(nocc) if gaps[j] > 1e-3]
    assert len(picked) >= 6
    h = 1e-5
    for j in picked:
        vp = _continued_vector(H + h * M, j, psi[j])
        vm = _continued_vector(H - h * M, j, psi[j])
        fd = st.project_conduction(psi, ((vp - vm) / (2 * h))[None, :])[0]
        x = st.solve_dense(st.operator(H, psi, w[j], alpha), st.rhs(dvpsi[j], psi))
        assert np.linalg.norm(fd - x) < 1e-6 * np.linalg.norm(x)
