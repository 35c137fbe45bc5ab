"""GPU parity of pwk_drho_batched (Eq. drho) against the oracle, through the C ABI.

Bar: FP64 ||drho_gpu - drho_ref||_2 / ||drho_ref||_2 <= 1e-12 (the FP64 path's bound);
FP32 transforms with FP64 products and sums <= 5e-6 (the FP32 bound of H|psi>: the same
transform pair, here the inverse only).  Inputs are seeded: random coefficients on the spheres,
k+q valence states orthonormalised (S-orthonormalised with q) by the oracle.
"""
import numpy as np
import pytest

from oracle import drho as dr
from oracle import overlap as ov
from paper_2412_01695_gb300 import synth

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def make(ks, nocc, q=None, seed=0):
    pk = synth.make_config(4, k_subset=ks, with_psi=False)
    pq = synth.make_config(4, k_subset=ks, with_psi=False, shift_q=True)
    rng = np.random.default_rng(seed)
    nk = len(ks)
    u_k = np.zeros((nk, nocc, pk.npw_max), complex)
    u_q = np.zeros((nk, nocc, pq.npw_max), complex)
    du = np.zeros((nk, nocc, pq.npw_max), complex)
    S_list = []
    for i in range(nk):
        a, b = pk.npw[i], pq.npw[i]
        u_k[i, :, :a] = np.linalg.qr(rng.normal(size=(a, nocc)) + 1j * rng.normal(size=(a, nocc)))[0].T
        S = np.eye(b) if q is None else ov.overlap_matrix(pq.beta[i][:, :b], q)
        u_q[i, :, :b] = ov.s_orthonormal(S, rng.normal(size=(nocc, b)) + 1j * rng.normal(size=(nocc, b)))
        du[i, :, :b] = rng.normal(size=(nocc, b)) + 1j * rng.normal(size=(nocc, b))
        S_list.append(S)
    w = rng.uniform(0.5, 1.5, nk) / nk
    return pk, pq, u_k, u_q, du, w, (None if q is None else S_list)


def run_gpu(pk, pq, u_k, u_q, du, w, precision, q=None):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    plan_k, plan_q = pwk.plan_from_problem(pk), pwk.plan_from_problem(pq)
    if q is not None:
        plan_q.set_overlap(q)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = torch.full((pk.N,) * 3, complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    pwk.drho_batched(plan_q, plan_k, pwk.PRECISIONS[precision], t(u_k), t(u_q), t(du), u_k.shape[1],
                     t(w), out)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    plan_k.close()
    plan_q.close()
    return res


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_c128", 5e-6)])
def test_drho_matches_oracle(precision, tol):
    pk, pq, u_k, u_q, du, w, _ = make([0, 1, 999, 4095], nocc=5)
    ref = dr.drho(pk, pq, u_k, u_q, du, weights=w)
    out = run_gpu(pk, pq, u_k, u_q, du, w, precision)
    assert rel(out, ref) <= tol, rel(out, ref)


def test_drho_with_overlap():
    q = synth.q_for(4)
    pk, pq, u_k, u_q, du, w, S_list = make([3, 2048], nocc=4, q=q, seed=1)
    ref = dr.drho(pk, pq, u_k, u_q, du, weights=w, S_list=S_list)
    out = run_gpu(pk, pq, u_k, u_q, du, w, "fp64", q=q)
    assert rel(out, ref) <= 1e-12
    # S really enters: the S = 1 projector gives a different density
    ref1 = dr.drho(pk, pq, u_k, u_q, du, weights=w)
    assert rel(ref1, ref) > 1e-3


def test_valence_input_gives_zero_and_runs_are_identical():
    """du along the valence states: P_c removes it (zero to rounding); two calls agree bit for bit."""
    pk, pq, u_k, u_q, du, w, _ = make([10, 11, 12], nocc=3, seed=2)
    zero = run_gpu(pk, pq, u_k, u_q, u_q * (0.5 + 0.25j), w, "fp64")
    assert np.max(np.abs(zero)) < 1e-12
    a = run_gpu(pk, pq, u_k, u_q, du, w, "fp64")
    b = run_gpu(pk, pq, u_k, u_q, du, w, "fp64")
    assert np.array_equal(a, b)


def test_many_pairs_more_than_partial_grids():
    """64 k-points x 6 bands = 384 pairs > 256 partial grids (CTAs take several pairs)."""
    ks = list(range(0, 4096, 64))
    pk, pq, u_k, u_q, du, w, _ = make(ks, nocc=6, seed=3)
    ref = dr.drho(pk, pq, u_k, u_q, du, weights=w)
    out = run_gpu(pk, pq, u_k, u_q, du, w, "fp64")
    assert rel(out, ref) <= 1e-12


def test_full_grid_with_weights_on_three_k_points():
    """All 4096 k-points x 6 bands of the DFPT cell in one call (every pair transformed), with
    the weights zero except on three k-points: the result must equal the oracle's induced
    density of those three alone (FP64 bound)."""
    ks = list(range(4096))
    nocc = 6
    pk = synth.make_config(4, k_subset=ks)
    pq = synth.make_config(4, k_subset=ks, shift_q=True)
    u_k = np.ascontiguousarray(pk.psi[:, :nocc])
    u_q = np.ascontiguousarray(pq.psi[:, :nocc])
    rng = np.random.default_rng(17)
    du = np.zeros((pq.nk, nocc, pq.npw_max), complex)
    for i in range(pq.nk):
        b = pq.npw[i]
        du[i, :, :b] = rng.normal(size=(nocc, b)) + 1j * rng.normal(size=(nocc, b))
    sel = [5, 2222, 4090]
    w = np.zeros(pk.nk)
    w[sel] = 1.0 / 3.0
    out = run_gpu(pk, pq, u_k, u_q, du, w, "fp64")
    sk = synth.make_config(4, k_subset=sel, with_psi=False)
    sq = synth.make_config(4, k_subset=sel, with_psi=False, shift_q=True)
    ref = dr.drho(sk, sq, u_k[sel][:, :, :sk.npw_max], u_q[sel][:, :, :sq.npw_max],
                  du[sel][:, :, :sq.npw_max], weights=w[sel])
    assert rel(out, ref) <= 1e-12, rel(out, ref)
