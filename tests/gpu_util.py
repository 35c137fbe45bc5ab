"""Helpers shared by the GPU parity tests: run the CUDA path through the C-ABI binding and
the oracle on the same seeded inputs."""
import numpy as np

from oracle import hamiltonian as ham


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test without a CUDA device"
    return torch


def run_hpsi(prob, precision="fp64", psi=None, nb=None):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    plan = pwk.plan_from_problem(prob)
    psi = prob.psi if psi is None else psi
    nb = psi.shape[1] if nb is None else nb
    prec = pwk.PRECISIONS[precision]
    dt = torch.complex64 if precision == "fp32" else torch.complex128
    x = torch.from_numpy(np.ascontiguousarray(psi)).to("cuda", dt)
    y = torch.full_like(x, complex(np.nan, np.nan))
    pwk.hpsi_batched(plan, prec, x, y, nb)
    torch.cuda.synchronize()
    out = y.cpu().numpy().astype(np.complex128)
    plan.close()
    return out


def oracle_hpsi(prob, psi=None, ks=None):
    psi = prob.psi if psi is None else psi
    vt = ham.grid_coefficients(prob.V_r)
    ks = range(prob.nk) if ks is None else ks
    return {ik: ham.hpsi_dense(prob, ik, psi[ik], vt) for ik in ks}


def max_rel_err(gpu, ref, prob, ks=None):
    """max over band-k of ||gpu - ref||_2 / ||ref||_2 on the valid coefficients; also checks
    that the padding is exactly zero."""
    worst = 0.0
    for ik in (ref.keys() if ks is None else ks):
        n = prob.npw[ik]
        assert np.all(gpu[ik][:, n:] == 0), "padding must be written as zero"
        e = ham.relative_error(gpu[ik][:, :n], ref[ik][:, :n])
        worst = max(worst, float(np.max(e)))
    return worst
