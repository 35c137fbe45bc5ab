"""GPU parity of pwk_eigh_batched (batched FP64 generalized Hermitian eigensolver of the
Davidson reduced problem) against LAPACK through the oracle's reduced-problem routine."""
import numpy as np
import pytest

from oracle import davidson as dav

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def random_pair(rng, nprob, n, cond=1e3):
    H = rng.standard_normal((nprob, n, n)) + 1j * rng.standard_normal((nprob, n, n))
    H = 0.5 * (H + np.conj(np.transpose(H, (0, 2, 1))))
    S = np.zeros_like(H)
    for p in range(nprob):
        Q = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
        S[p] = (Q * np.logspace(0, -np.log10(cond), n)) @ Q.conj().T
        S[p] = 0.5 * (S[p] + S[p].conj().T)
    return np.ascontiguousarray(H), np.ascontiguousarray(S)


def check(H, S, eig, vec, nev, tol):
    for p in range(H.shape[0]):
        w, v = dav._reduced_eig(H[p], S[p], nev)
        scale = max(1.0, np.max(np.abs(w)))
        np.testing.assert_allclose(eig[p], w, rtol=0, atol=tol * scale)
        X = vec[p]
        np.testing.assert_allclose(X.conj().T @ S[p] @ X, np.eye(nev), atol=1e-9)
        R = H[p] @ X - S[p] @ X * eig[p][None, :]
        assert np.max(np.linalg.norm(R, axis=0)) < 1e-9 * scale


@pytest.mark.parametrize("n,nev", [(1, 1), (2, 1), (8, 8), (48, 12), (160, 40), (97, 31)])
def test_random_pairs(n, nev):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    rng = np.random.default_rng(n)
    H, S = random_pair(rng, 5, n)
    st = torch.full((5,), 99, dtype=torch.int32, device="cuda")
    eig, vec = pwk.eigh_batched(torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda(), nev, status=st)
    assert np.all(st.cpu().numpy() == 0)
    check(H, S, eig.cpu().numpy(), vec.cpu().numpy(), nev, 1e-11)


def test_dependent_row_is_left_out():
    """A row of S beyond nev that is a copy of another is dependent: it is left out, exactly as
    the oracle's reduced-problem routine does."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    rng = np.random.default_rng(5)
    n, nev = 30, 6
    B = rng.standard_normal((n, 60)) + 1j * rng.standard_normal((n, 60))
    B[20] = B[3]                                  # basis vector 20 duplicates vector 3
    A = rng.standard_normal((60, 60)) + 1j * rng.standard_normal((60, 60))
    A = A + A.conj().T
    S = np.ascontiguousarray((B.conj() @ B.T)[None])
    H = np.ascontiguousarray((B.conj() @ A @ B.T)[None])
    eig, vec = pwk.eigh_batched(torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda(), nev)
    w, v = dav._reduced_eig(H[0], S[0], nev)
    np.testing.assert_allclose(eig.cpu().numpy()[0], w, atol=1e-9 * np.max(np.abs(w)))
    assert np.max(np.abs(vec.cpu().numpy()[0][20])) < 1e-12


def test_nearly_dependent_chain_matches_oracle():
    """Vectors that add less than 1e-3 of a new direction (pivot below 1e-6 of the diagonal),
    one of them built on another such vector, and an exact linear combination: all are left
    out, the Ritz values equal the oracle's and no spurious value appears below the spectrum."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    rng = np.random.default_rng(11)
    n, nev, m = 32, 8, 80
    B = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    B /= np.linalg.norm(B, axis=1, keepdims=True)
    noise = lambda: 1e-4 * (rng.standard_normal(m) + 1j * rng.standard_normal(m)) / np.sqrt(2 * m)  # noqa: E731
    B[20] = B[3] + noise()
    B[21] = B[20] + noise()
    B[25] = 3.0 * B[7] - 2.0 * B[11]
    B[28] = B[25] + noise()
    A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    A = A + A.conj().T
    S = np.ascontiguousarray((B.conj() @ B.T)[None])
    H = np.ascontiguousarray((B.conj() @ A @ B.T)[None])
    eig, vec = pwk.eigh_batched(torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda(), nev)
    w, v = dav._reduced_eig(H[0], S[0], nev)
    np.testing.assert_allclose(eig.cpu().numpy()[0], w, atol=1e-9 * np.max(np.abs(w)))
    V = vec.cpu().numpy()[0]
    for r in (20, 21, 25, 28):
        assert np.max(np.abs(V[r])) < 1e-12
    # lower bound: no Ritz value below the smallest eigenvalue of A
    assert eig.cpu().numpy()[0].min() >= np.linalg.eigvalsh(A)[0] - 1e-9


def test_indefinite_leading_block_reports_status():
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    n = 10
    H = np.ascontiguousarray(np.eye(n, dtype=complex)[None])
    S = np.ascontiguousarray(np.eye(n, dtype=complex)[None])
    S[0, 1, 1] = -1.0
    st = torch.zeros((1,), dtype=torch.int32, device="cuda")
    pwk.eigh_batched(torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda(), 4, status=st)
    assert st.cpu().numpy()[0] == -6
