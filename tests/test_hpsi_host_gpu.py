"""GPU parity of pwk_hpsi_batched_host (H|psi> with the vectors in host memory, copies in,
applications and copies out of groups of k-points overlapped) through the C ABI.

Bar: the same kernels run per band-k as in pwk_hpsi_batched, so the result must equal it bit
for bit for every group count; against the FP64 oracle the FP64 bound 1e-12 (relative, per
band-k) of the H|psi> tests holds.
"""
import numpy as np
import pytest

from paper_2412_01695_gb300 import synth

from gpu_util import max_rel_err, oracle_hpsi, torch_cuda

pytestmark = pytest.mark.gpu


def host_apply(plan, prec, psi_np, nb, nchunk, dt, in_place=False):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    h_in = torch.from_numpy(np.ascontiguousarray(psi_np)).to(dt).pin_memory()
    h_out = torch.full_like(h_in, complex(np.nan, np.nan)).pin_memory()
    d_in = torch.full(h_in.shape, complex(np.nan, np.nan), dtype=dt, device="cuda")
    d_out = d_in if in_place else torch.full_like(d_in, complex(np.nan, np.nan))
    pwk.hpsi_batched_host(plan, prec, h_in, h_out, d_in, d_out, nb, nchunk)
    torch.cuda.current_stream().synchronize()
    return h_out.numpy().copy()


def device_apply(plan, prec, psi_np, nb, dt):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    x = torch.from_numpy(np.ascontiguousarray(psi_np)).to("cuda", dt)
    y = torch.full_like(x, complex(np.nan, np.nan))
    pwk.hpsi_batched(plan, prec, x, y, nb)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("nchunk", [1, 2, 3, 7, 1000])
def test_host_fp64_cfg1_equals_device_path_and_oracle(nchunk):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(1)
    plan = pwk.plan_from_problem(prob)
    ref_dev = device_apply(plan, pwk.PWK_FP64, prob.psi, prob.nb, torch.complex128)
    out = host_apply(plan, pwk.PWK_FP64, prob.psi, prob.nb, nchunk, torch.complex128)
    assert np.array_equal(out, ref_dev)
    assert max_rel_err(out, oracle_hpsi(prob), prob) <= 1e-12
    plan.close()


def test_host_in_place_work_buffer():
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(2, k_subset=synth.sample_k(512, 9), nb=4)
    plan = pwk.plan_from_problem(prob)
    ref_dev = device_apply(plan, pwk.PWK_FP64, prob.psi, prob.nb, torch.complex128)
    out = host_apply(plan, pwk.PWK_FP64, prob.psi, prob.nb, 4, torch.complex128, in_place=True)
    assert np.array_equal(out, ref_dev)
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp32_c128"])
def test_host_full_size_cfg2_equals_device_path(precision):
    """The 512 k x 20 bands batch in eight groups (the benchmark's end-to-end call); a seeded
    sample of k-points against the oracle."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(2)
    prec = pwk.PRECISIONS[precision]
    dt = torch.complex64 if precision == "fp32" else torch.complex128
    psi = prob.psi.astype(np.complex64).astype(np.complex128) if precision == "fp32" else prob.psi
    plan = pwk.plan_from_problem(prob)
    ref_dev = device_apply(plan, prec, psi, prob.nb, dt)
    out = host_apply(plan, prec, psi, prob.nb, 8, dt)
    assert np.array_equal(out, ref_dev)
    ks = synth.sample_k(prob.nk, 4, seed=5)
    assert max_rel_err(out.astype(np.complex128), oracle_hpsi(prob, psi=psi, ks=ks), prob, ks=ks) <= 5e-6
    plan.close()


def test_host_bad_arguments_are_refused():
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(1)
    plan = pwk.plan_from_problem(prob)
    h = torch.from_numpy(prob.psi.copy()).pin_memory()
    d = torch.from_numpy(prob.psi).cuda()
    with pytest.raises(pwk.PwkError) as ei:
        pwk.hpsi_batched_host(plan, pwk.PWK_FP64, h, h.clone(), d, d.clone(), prob.nb, 0)
    assert ei.value.code == -1
    with pytest.raises(ValueError):   # device tensor where a host one belongs
        pwk.hpsi_batched_host(plan, pwk.PWK_FP64, d, h, d, d.clone(), prob.nb, 2)
    plan.close()
