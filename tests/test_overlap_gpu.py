"""GPU parity of the overlap operator S (ultrasoft/PAW q_mn) and of H and S applied together
(pwk_hspsi_batched / pwk_hspsi_items) against the FP64 oracle, through the C ABI.

Tolerances as for H alone: FP64 <= 1e-12 relative per band-k, FP32 <= 5e-6 (S - 1 is a
projector sum of norm <= 1.5 on these cells, so it adds nothing to the FP32 bound).
"""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import overlap as ov
from paper_2412_01695_gb300 import synth

from gpu_util import max_rel_err, oracle_hpsi, torch_cuda

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 5e-6


def run_hs(prob, q, precision="fp64", items=None, nvec=None, path=0):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    plan = pwk.plan_from_problem(prob)
    plan.set_projector_path(path)
    plan.set_overlap(q)
    assert plan.has_overlap == (q is not None and prob.nkb > 0)
    prec = pwk.PRECISIONS[precision]
    dt = torch.complex64 if precision == "fp32" else torch.complex128
    x = torch.from_numpy(np.ascontiguousarray(prob.psi)).to("cuda", dt)
    h = torch.full_like(x, complex(np.nan, np.nan))
    s = torch.full_like(x, complex(np.nan, np.nan))
    if items is None:
        pwk.hspsi_batched(plan, prec, x, h, s, prob.nb)
    else:
        it = torch.tensor(items, dtype=torch.int32, device="cuda")
        pwk.hspsi_items(plan, prec, x, h, s, it, prob.nb)
    torch.cuda.synchronize()
    out = h.cpu().numpy().astype(np.complex128), s.cpu().numpy().astype(np.complex128)
    plan.close()
    return out


def oracle_spsi(prob, q, psi=None):
    psi = prob.psi if psi is None else psi
    out = {}
    for ik in range(prob.nk):
        n = prob.npw[ik]
        r = np.zeros_like(psi[ik])
        r[:, :n] = ov.spsi_steps(prob.beta[ik][:, :n], q, psi[ik][:, :n])
        out[ik] = r
    return out


@pytest.mark.parametrize("cfg,nks", [(1, 8), (2, 4), (3, 2)])
def test_hs_fp64(cfg, nks):
    nkfull = int(np.prod(synth.CONFIGS[cfg]["mp"]))
    prob = synth.make_config(cfg, k_subset=synth.sample_k(nkfull, nks), nb=min(6, synth.CONFIGS[cfg]["nb"]))
    q = synth.q_for(cfg)
    h, s = run_hs(prob, q)
    assert max_rel_err(h, oracle_hpsi(prob), prob) <= TOL64
    assert max_rel_err(s, oracle_spsi(prob, q), prob) <= TOL64
    # the q term is really there: S psi differs from psi by more than rounding
    ik = 0
    n = prob.npw[ik]
    assert np.max(np.abs(s[ik][:, :n] - prob.psi[ik][:, :n])) > 1e-3


@pytest.mark.parametrize("precision", ["fp32", "fp32_c128"])
def test_hs_fp32(precision):
    prob = synth.make_config(2, k_subset=synth.sample_k(512, 4), nb=6)
    q = synth.q_for(2)
    psi = prob.psi.astype(np.complex64).astype(np.complex128) if precision == "fp32" else prob.psi
    prob.psi = psi
    h, s = run_hs(prob, q, precision)
    assert max_rel_err(h, oracle_hpsi(prob), prob) <= TOL32
    assert max_rel_err(s, oracle_spsi(prob, q), prob) <= TOL32


def test_without_q_s_is_identity():
    """No q: S psi = psi bit for bit (the add-back adds nothing)."""
    prob = synth.make_config(1)
    h, s = run_hs(prob, None)
    np.testing.assert_array_equal(s, prob.psi)
    assert max_rel_err(h, oracle_hpsi(prob), prob) <= TOL64


def test_items_subset_and_order():
    """A work list with empty slots, two k-points interleaved and out-of-order outputs."""
    prob = synth.make_config(2, k_subset=[0, 100, 511], nb=5)
    q = synth.q_for(2)
    items = [(0, 0, 4), (2, 3, 1), (-1, 0, 0), (1, 2, 2), (0, 1, 0), (2, 4, 4)]
    h, s = run_hs(prob, q, items=items)
    ref_h, ref_s = oracle_hpsi(prob), oracle_spsi(prob, q)
    for k, vi, vo in items:
        if k < 0:
            continue
        n = prob.npw[k]
        assert ham.relative_error(h[k][vo, :n], ref_h[k][vi, :n]) <= TOL64
        assert ham.relative_error(s[k][vo, :n], ref_s[k][vi, :n]) <= TOL64
        assert np.all(s[k][vo, n:] == 0)
    # untouched outputs keep their (NaN) fill
    assert np.isnan(h[1][0]).all() and np.isnan(s[2][0]).all()


def test_aliasing_rejected():
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(1, nb=2)
    plan = pwk.plan_from_problem(prob)
    x = torch.from_numpy(np.ascontiguousarray(prob.psi)).cuda()
    y = torch.empty_like(x)
    with pytest.raises(pwk.PwkError):
        pwk.hspsi_batched(plan, pwk.PWK_FP64, x, x, y, prob.nb)
    with pytest.raises(pwk.PwkError):
        pwk.hspsi_batched(plan, pwk.PWK_FP64, x, y, x, prob.nb)
    plan.close()


@pytest.mark.parametrize("path", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32_c128"])
@pytest.mark.parametrize("cfg,nks", [(1, 8), (2, 4), (4, 3)])
def test_hs_each_projector_path(path, precision, cfg, nks):
    """H and S together with the projector terms in separate kernels (path 2) and inside the
    local kernel (path 3), batched and on a work list, against the oracle; without q, S psi is
    psi bit for bit on both paths."""
    nkfull = int(np.prod(synth.CONFIGS[cfg]["mp"]))
    prob = synth.make_config(cfg, k_subset=synth.sample_k(nkfull, nks), nb=4)
    q = synth.q_for(cfg)
    tol = TOL64 if precision == "fp64" else TOL32
    h, s = run_hs(prob, q, precision, path=path)
    assert max_rel_err(h, oracle_hpsi(prob), prob) <= tol
    assert max_rel_err(s, oracle_spsi(prob, q), prob) <= tol
    items = [(0, 0, 3), (prob.nk - 1, 2, 1), (-1, 0, 0), (0, 1, 0)]
    h, s = run_hs(prob, q, precision, items=items, path=path)
    ref_h, ref_s = oracle_hpsi(prob), oracle_spsi(prob, q)
    for k, vi, vo in items:
        if k < 0:
            continue
        n = prob.npw[k]
        assert ham.relative_error(h[k][vo, :n], ref_h[k][vi, :n]) <= tol
        assert ham.relative_error(s[k][vo, :n], ref_s[k][vi, :n]) <= tol
        assert np.all(s[k][vo, n:] == 0) and np.all(h[k][vo, n:] == 0)
    h, s = run_hs(prob, None, precision, path=path)
    np.testing.assert_array_equal(s, prob.psi)
