"""Argument checks of the reduced-eigensolver bindings (CPU, no library call).

The kernel behind pwk_eigh_batched and pwk_eigh_batched_noalloc trusts the sizes it is given,
so the binding refuses, before any pointer reaches the library, every argument whose dtype or
shape does not match (nprob, n, nev): a float32 eig, a vec smaller than [nprob][n][nev], a
status shorter than nprob, non-complex128 H or S, nev outside [1, n], a host tensor."""
import pytest

torch = pytest.importorskip("torch")

from paper_2412_01695_gb300 import pwk  # noqa: E402

NP, N, NEV = 3, 8, 4


def _args():
    H = torch.zeros((NP, N, N), dtype=torch.complex128)
    return dict(H=H, S=H.clone(), eig=torch.zeros((NP, NEV), dtype=torch.float64),
                vec=torch.zeros((NP, N, NEV), dtype=torch.complex128),
                status=torch.zeros((NP,), dtype=torch.int32))


BAD = {
    "eig float32": ("eig", lambda: torch.zeros((NP, NEV), dtype=torch.float32), "eig must be"),
    "eig too short": ("eig", lambda: torch.zeros((NP, NEV - 1), dtype=torch.float64), "eig must have shape"),
    "vec smaller": ("vec", lambda: torch.zeros((NP, N, NEV - 1), dtype=torch.complex128), "vec must have shape"),
    "vec complex64": ("vec", lambda: torch.zeros((NP, N, NEV), dtype=torch.complex64), "vec must be"),
    "status short": ("status", lambda: torch.zeros((NP - 1,), dtype=torch.int32), "status must have shape"),
    "status int64": ("status", lambda: torch.zeros((NP,), dtype=torch.int64), "status must be"),
    "H float64": ("H", lambda: torch.zeros((NP, N, N), dtype=torch.float64), "H must be"),
    "S wrong shape": ("S", lambda: torch.zeros((NP, N, N + 1), dtype=torch.complex128), "S must have shape"),
    "S complex64": ("S", lambda: torch.zeros((NP, N, N), dtype=torch.complex64), "S must be"),
    "H not square": ("H", lambda: torch.zeros((NP, N, N + 1), dtype=torch.complex128), "H must have shape"),
}


@pytest.mark.parametrize("case", sorted(BAD), ids=sorted(BAD))
def test_noalloc_refuses_mismatched_arguments(case):
    name, make, msg = BAD[case]
    a = _args()
    a[name] = make()
    with pytest.raises(ValueError, match=msg):
        pwk.eigh_batched_noalloc(a["H"], a["S"], NEV, a["eig"], a["vec"], status=a["status"])


@pytest.mark.parametrize("nev", [0, N + 1])
def test_nev_outside_the_problem_is_refused(nev):
    a = _args()
    with pytest.raises(ValueError, match="nev"):
        pwk.eigh_batched_noalloc(a["H"], a["S"], nev, a["eig"], a["vec"])
    with pytest.raises(ValueError, match="nev"):
        pwk.eigh_batched(a["H"], a["S"], nev)


def test_host_tensors_are_refused():
    a = _args()
    with pytest.raises(ValueError, match="CUDA"):
        pwk.eigh_batched_noalloc(a["H"], a["S"], NEV, a["eig"], a["vec"], status=a["status"])
    with pytest.raises(ValueError, match="CUDA"):
        pwk.eigh_batched(a["H"], a["S"], NEV)


def test_allocating_entry_point_checks_h_and_s():
    a = _args()
    with pytest.raises(ValueError, match="S must be"):
        pwk.eigh_batched(a["H"], a["S"].to(torch.complex64), NEV)
