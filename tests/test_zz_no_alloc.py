"""pwk_eigh_batched_noalloc against pwk_eigh_batched (through the C ABI).

The allocation-free entry point serves callers that cannot call cudaMalloc where they solve:
a latency-bound serving loop (cudaMalloc and cudaFree synchronise the whole device) or a
process whose device memory is entirely reserved by another allocator.  It runs the same
batched eigensolver on a fixed workspace held in the library's device memory.  Here two calls
in a row, with different inputs (the second at the workspace limit), must each match the
allocating entry point within the tolerance of the eigensolver tests, and a call above the
limit must be refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _pair(rng, nprob, n):
    H = rng.standard_normal((nprob, n, n)) + 1j * rng.standard_normal((nprob, n, n))
    H = 0.5 * (H + np.conj(np.transpose(H, (0, 2, 1))))
    S = np.zeros_like(H)
    for p in range(nprob):
        Q = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
        S[p] = (Q * np.logspace(0, -3, n)) @ Q.conj().T
        S[p] = 0.5 * (S[p] + S[p].conj().T)
    return np.ascontiguousarray(H), np.ascontiguousarray(S)


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    """First a call at the workspace limit whose H is all NaN (its results and status are not
    looked at): it leaves NaN in the workspace regions that hold L^-1 H and the reduced matrix.
    A later call that read any workspace element before writing it would carry NaN into its
    results; the two valid calls that follow must be finite and match the allocating entry
    point."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    rng = np.random.default_rng(2412)
    Hn, Sn = _pair(rng, 16, 160)
    Hn[:] = np.nan
    eig = torch.empty((16, 40), dtype=torch.float64, device="cuda")
    vec = torch.empty((16, 160, 40), dtype=torch.complex128, device="cuda")
    pwk.eigh_batched_noalloc(torch.from_numpy(Hn).cuda(), torch.from_numpy(Sn).cuda(), 40, eig, vec)
    torch.cuda.synchronize()
    for nprob, n, nev in ((6, 48, 12), (16, 160, 40)):
        H, S = _pair(rng, nprob, n)
        Hd, Sd = torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda()
        e_ref, v_ref = pwk.eigh_batched(Hd, Sd, nev)
        eig = torch.full((nprob, nev), np.nan, dtype=torch.float64, device="cuda")
        vec = torch.full((nprob, n, nev), np.nan, dtype=torch.complex128, device="cuda")
        st = torch.full((nprob,), 99, dtype=torch.int32, device="cuda")
        pwk.eigh_batched_noalloc(Hd, Sd, nev, eig, vec, status=st)
        torch.cuda.synchronize()
        assert np.all(st.cpu().numpy() == 0)
        e_ref, v_ref = e_ref.cpu().numpy(), v_ref.cpu().numpy()
        e, v = eig.cpu().numpy(), vec.cpu().numpy()
        assert np.all(np.isfinite(e)) and np.all(np.isfinite(v))
        scale = max(1.0, float(np.max(np.abs(e_ref))))
        np.testing.assert_allclose(e, e_ref, rtol=0, atol=1e-11 * scale)
        np.testing.assert_allclose(v, v_ref, rtol=0, atol=1e-9)


def test_noalloc_refuses_calls_above_its_workspace():
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    n, nprob = 160, 17            # 17 * 160^2 > 409600
    H = torch.zeros((nprob, n, n), dtype=torch.complex128, device="cuda")
    eig = torch.zeros((nprob, 4), dtype=torch.float64, device="cuda")
    vec = torch.zeros((nprob, n, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(pwk.PwkError) as ei:
        pwk.eigh_batched_noalloc(H, H, 4, eig, vec)
    assert ei.value.code == -2
