"""GPU parity of the solvers with the ultrasoft/PAW overlap S (plans with q_mn) against the
oracle, through the C ABI.

Davidson: H x = eps S x; eigenvalues within 1e-8 Ry of the dense generalized problem
(LAPACK through the oracle), eigenvectors S-orthonormal, the occupied subspace equal to the
dense one (S-metric projector difference, Davis-Kahan bound).
Sternheimer: [H + alpha Q - eps S] x = -(1 - S P_v) dV psi (oracle/overlap.py), true residual
<= 1e-10 with the oracle's dense operator for every positive-definite pair, x within 1e-7 of
the dense LU solution.
"""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import overlap as ov
from oracle import sternheimer as st
from paper_2412_01695_gb300 import synth

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

TOL = 1e-10


def run_dav_s(prob, q, mode, max_iter=300):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    plan = pwk.plan_from_problem(prob)
    plan.set_overlap(q)
    psi = torch.from_numpy(np.ascontiguousarray(prob.psi)).cuda()
    eig = torch.zeros((prob.nk, prob.nb), dtype=torch.float64, device="cuda")
    m = pwk.PWK_FP64 if mode == "fp64" else pwk.PWK_FP32_C128
    rc, iters, notc, napply = pwk.davidson_batched(plan, m, psi, eig, prob.nb, 1e-10, 1e-5, max_iter, 0)
    out = eig.cpu().numpy(), psi.cpu().numpy()
    plan.close()
    return rc, out[0], out[1], iters


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("cfg,ks", [(1, None), (2, [0, 77, 300])])
def test_davidson_generalized(mode, cfg, ks):
    prob = synth.make_config(cfg, k_subset=ks)
    q = synth.q_for(cfg)
    rc, eig, psi, iters = run_dav_s(prob, q, mode)
    assert rc == 0
    vt = ham.grid_coefficients(prob.V_r)
    for ik in range(prob.nk):
        n = prob.npw[ik]
        H = ham.problem_h(prob, ik, vt)
        S = ov.overlap_matrix(prob.beta[ik][:, :n], q)
        w, v = ov.lowest_generalized(H, S, prob.nb + 1)
        np.testing.assert_allclose(eig[ik], w[:prob.nb], atol=1e-8)
        X = psi[ik][:, :n]
        np.testing.assert_allclose(X.conj() @ S @ X.T, np.eye(prob.nb), atol=1e-8)
        # same subspace: ||P_gpu - P_ref|| in the S metric, P = X^T X^* S
        gap = w[prob.nb] - w[prob.nb - 1]
        Pg = X.T @ X.conj() @ S
        Pr = v[:prob.nb].T @ v[:prob.nb].conj() @ S
        assert np.linalg.norm(Pg - Pr, 2) <= 10 * 1e-5 / gap + 1e-8
    # S really matters: the S = 1 eigenvalues differ
    H0 = ham.problem_h(prob, 0, vt)
    assert np.max(np.abs(np.linalg.eigvalsh(H0)[:prob.nb] - eig[0])) > 1e-3


def make_inputs_s(ks, q, nocc=12):
    pk = synth.make_config(4, k_subset=ks, with_psi=False)
    pq = synth.make_config(4, k_subset=ks, with_psi=False, shift_q=True)
    vt = ham.grid_coefficients(pk.V_r)
    nk = len(ks)
    psi_k = np.zeros((nk, nocc, pk.npw_max), complex)
    psi_q = np.zeros((nk, nocc, pq.npw_max), complex)
    eps_k = np.zeros((nk, nocc))
    eq_all, Hq_all, Sq_all = [], [], []
    for i in range(nk):
        Hk, Hq = ham.problem_h(pk, i, vt), ham.problem_h(pq, i, vt)
        Sk = ov.overlap_matrix(pk.beta[i][:, :pk.npw[i]], q)
        Sq = ov.overlap_matrix(pq.beta[i][:, :pq.npw[i]], q)
        wk, vk = ov.lowest_generalized(Hk, Sk, nocc)
        wq, vq = ov.lowest_generalized(Hq, Sq, nocc + 1)
        psi_k[i, :, :pk.npw[i]] = vk
        psi_q[i, :, :pq.npw[i]] = vq[:nocc]
        eps_k[i] = wk
        eq_all.append(wq)
        Hq_all.append(Hq)
        Sq_all.append(Sq)
    alpha = np.array([st.alpha_pv(eps_k[i], eq_all[i][:nocc]) for i in range(nk)])
    return pk, pq, psi_k, psi_q, eps_k, eq_all, Hq_all, Sq_all, alpha, synth.dv_for(4)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_sternheimer_with_overlap(mode):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    q = synth.q_for(4)
    ks = [0, 1, 1234, 4095]
    pk, pq, psi_k, psi_q, eps_k, eq_all, Hq_all, Sq_all, alpha, dv = make_inputs_s(ks, q)
    plan_k, plan_q = pwk.plan_from_problem(pk), pwk.plan_from_problem(pq)
    plan_q.set_overlap(q)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    nocc = psi_k.shape[1]
    dpsi = torch.zeros((pq.nk, nocc, pq.npw_max), dtype=torch.complex128, device="cuda")
    m = pwk.PWK_FP64 if mode == "fp64" else pwk.PWK_FP32_C128
    rc, iters, resid = pwk.sternheimer_cg_batched(plan_q, plan_k, m, t(psi_k), t(eps_k), t(psi_q), nocc,
                                                  t(alpha), t(dv), dpsi, TOL, 400)
    x = dpsi.cpu().numpy()
    plan_k.close()
    plan_q.close()
    dvt = ham.grid_coefficients(dv)
    worst_res, worst_x, n_pd = 0.0, 0.0, 0
    for i in range(len(ks)):
        nkk, nq = pk.npw[i], pq.npw[i]
        U = psi_q[i, :, :nq]
        dvpsi = st.dv_psi_dense(pq.miller[i, :nq], pk.miller[i, :nkk], dvt, psi_k[i, :, :nkk])
        b_all = ov.rhs(dvpsi, Sq_all[i], U)
        for n in range(nocc):
            A = ov.operator(Hq_all[i], Sq_all[i], U, eps_k[i, n], alpha[i])
            b = b_all[n]
            xg = x[i, n, :nq]
            assert np.all(x[i, n, nq:] == 0)
            if eq_all[i][nocc] - eps_k[i, n] > 0:
                n_pd += 1
                rel = np.linalg.norm(A @ xg - b) / np.linalg.norm(b)
                xr = np.linalg.solve(A, b)
                worst_res = max(worst_res, rel)
                worst_x = max(worst_x, np.linalg.norm(xg - xr) / np.linalg.norm(xr))
                assert abs(resid[i * nocc + n] - rel) < 1e-11 + 0.05 * rel
                # the solution has no component along the valence states in the S metric
                assert np.max(np.abs(U.conj() @ Sq_all[i] @ xg)) < 1e-8 * np.linalg.norm(xg)
    assert n_pd > 0
    assert worst_res <= TOL, worst_res
    assert worst_x <= 1e-7, worst_x
