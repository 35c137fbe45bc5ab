"""Pins of the induced-density oracle (Eq. drho) against closed forms and invariants (no GPU).

Each pin is chosen so a plausible slip fails it: a conjugate on the wrong factor, the k and
k+q spheres swapped, a sign in the transform exponent, the projector P_c left out or taken
without S, the factor 4 w_k, the grid order.
"""
import numpy as np

from oracle import drho as dr
from oracle import overlap as ov
from paper_2412_01695_gb300 import synth


def _pair(ks, nb=3):
    pk = synth.make_config(4, k_subset=ks, with_psi=False)
    pq = synth.make_config(4, k_subset=ks, with_psi=False, shift_q=True)
    return pk, pq


def _unit(npw_max, idx):
    v = np.zeros(npw_max, complex)
    v[idx] = 1.0
    return v


def test_plane_waves_closed_form():
    """u = e^{i G1.r} on the k sphere, du = e^{i G2.r} on the k+q sphere, orthogonal to the
    valence states: drho(r_l) = 4 w e^{2 pi i (m2 - m1).l / N}."""
    pk, pq = _pair([5])
    N = pk.N
    i1, i2 = 3, 17
    u_k = _unit(pk.npw_max, i1)[None, None, :]
    du = _unit(pq.npw_max, i2)[None, None, :]
    u_kq = _unit(pq.npw_max, 0)[None, None, :]             # a valence state orthogonal to du
    out = dr.drho(pk, pq, u_k, u_kq, du, weights=[0.25])
    m1, m2 = pk.miller[0, i1], pq.miller[0, i2]
    l = np.stack(np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij"), -1)
    expect = 4 * 0.25 * np.exp(2j * np.pi * (l @ (m2 - m1)) / N)
    np.testing.assert_allclose(out, expect, atol=1e-12)


def test_valence_direction_is_projected_out():
    """du along a valence state of k+q gives zero (P_c u_v = 0), with and without S."""
    pk, pq = _pair([0, 9])
    rng = np.random.default_rng(1)
    nq = pq.npw_max
    q = synth.q_for(4)
    for with_s in (False, True):
        S_list, u_kq = [], np.zeros((2, 2, nq), complex)
        for i in range(2):
            n = pq.npw[i]
            S = ov.overlap_matrix(pq.beta[i][:, :n], q) if with_s else np.eye(n)
            X = rng.normal(size=(2, n)) + 1j * rng.normal(size=(2, n))
            u_kq[i, :, :n] = ov.s_orthonormal(S, X)
            S_list.append(S)
        u_k = rng.normal(size=(2, 2, pk.npw_max)) + 0j
        for i in range(2):
            u_k[i, :, pk.npw[i]:] = 0
        du = u_kq[:, ::-1].copy() * (0.3 - 0.2j)
        out = dr.drho(pk, pq, u_k, u_kq, du, S_list=S_list if with_s else None)
        assert np.max(np.abs(out)) < 1e-12


def test_sum_over_grid_is_the_overlap():
    """sum_l drho(r_l) = 4 sum_k w_k N_r sum_nu sum_m conj(C(m)) [P_c dC](m) over the Miller
    indices the k and k+q spheres share (Parseval for the discrete transform)."""
    pk, pq = _pair([1, 77, 400], nb=3)
    rng = np.random.default_rng(4)
    nk, nocc = 3, 2
    u_k = rng.normal(size=(nk, nocc, pk.npw_max)) + 1j * rng.normal(size=(nk, nocc, pk.npw_max))
    du = rng.normal(size=(nk, nocc, pq.npw_max)) + 1j * rng.normal(size=(nk, nocc, pq.npw_max))
    u_kq = np.zeros((nk, 1, pq.npw_max), complex)
    for i in range(nk):
        u_k[i, :, pk.npw[i]:] = 0
        du[i, :, pq.npw[i]:] = 0
        v = rng.normal(size=pq.npw[i]) + 1j * rng.normal(size=pq.npw[i])
        u_kq[i, 0, :pq.npw[i]] = v / np.linalg.norm(v)
    w = np.array([0.5, 0.3, 0.2])
    out = dr.drho(pk, pq, u_k, u_kq, du, weights=w)
    Nr = pk.N ** 3
    ref = 0.0
    for i in range(nk):
        nkk, nq = pk.npw[i], pq.npw[i]
        duc = dr.project_conduction(u_kq[i, :, :nq], du[i, :, :nq])
        mk = {tuple(m): g for g, m in enumerate(pk.miller[i, :nkk])}
        for g2, m in enumerate(pq.miller[i, :nq]):
            g1 = mk.get(tuple(m))
            if g1 is not None:
                ref += 4 * w[i] * Nr * np.sum(u_k[i, :, g1].conj() * duc[:, g2])
    np.testing.assert_allclose(out.sum(), ref, rtol=1e-11)


def test_linear_in_du_and_antilinear_in_u():
    pk, pq = _pair([3])
    rng = np.random.default_rng(6)
    u_k = rng.normal(size=(1, 2, pk.npw_max)) + 1j * rng.normal(size=(1, 2, pk.npw_max))
    du = rng.normal(size=(1, 2, pq.npw_max)) + 1j * rng.normal(size=(1, 2, pq.npw_max))
    u_k[0, :, pk.npw[0]:] = 0
    du[0, :, pq.npw[0]:] = 0
    u_kq = np.zeros((1, 1, pq.npw_max), complex)
    u_kq[0, 0, 0] = 1.0
    a = 0.7 - 1.3j
    base = dr.drho(pk, pq, u_k, u_kq, du)
    np.testing.assert_allclose(dr.drho(pk, pq, u_k, u_kq, a * du), a * base, atol=1e-12)
    np.testing.assert_allclose(dr.drho(pk, pq, a * u_k, u_kq, du), np.conj(a) * base, atol=1e-12)


def test_first_order_density_change():
    """At q = 0 with a real dv, the real part of Eq. drho for one k (w = 1) built from the
    Sternheimer solutions equals d/d delta of the density 2 sum_n |u_n(r)|^2 of the lowest
    states of H + delta dV (central difference of dense eigenvectors, gauge-free).  The
    valence-valence and phase terms of d u_n cancel in the sum, which is why P_c du is enough."""
    from oracle import hamiltonian as ham
    from oracle import sternheimer as st
    pk = synth.make_config(4, k_subset=[6], with_psi=False)
    n = pk.npw[0]
    m = pk.miller[0, :n]
    H = ham.problem_h(pk, 0)
    dvt = ham.grid_coefficients(np.real(synth.dv_for(4)))
    M = ham.local_matrix(m, m, dvt)
    w, V = np.linalg.eigh(H)
    nocc = 6
    assert w[nocc] - w[nocc - 1] > 1e-2          # the occupied manifold is separated
    u = V[:, :nocc].T
    alpha = st.alpha_pv(w[:nocc], w[:nocc])
    dvpsi = st.dv_psi_dense(m, m, dvt, u)
    du = np.array([st.solve_dense(st.operator(H, u, w[j], alpha), st.rhs(dvpsi[j], u))
                   for j in range(nocc)])
    out = dr.drho(pk, pk, u[None], u[None], du[None], weights=[1.0])
    E = ham.phase_matrix(m, pk.N)
    h = 1e-5

    def density(sign):
        X = np.linalg.eigh(H + sign * h * M)[1][:, :nocc].T
        return 2.0 * np.sum(np.abs(ham.to_real_space(X, E)) ** 2, axis=0)

    fd = ((density(1) - density(-1)) / (2 * h)).reshape(out.shape)
    scale = np.max(np.abs(fd))
    assert scale > 1e-3
    np.testing.assert_allclose(out.real, fd, rtol=0, atol=1e-6 * scale)
