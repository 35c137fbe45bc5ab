"""pwk_hpsi_multi: one launch over work items of several cells that share an FFT grid but
have uneven projector sets (9, 4 and 0 projectors), checked against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

from paper_2412_01695_gb300 import synth

from gpu_util import oracle_hpsi, torch_cuda

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 5e-6, "fp32_c128": 5e-6}


def _cells():
    """Three cells on a 24^3 grid: fcc with one atom and s, p, d projectors (9), simple cubic
    with two atoms and s, p projectors (8), and an fcc cell without projectors (0)."""
    out = []
    A1 = synth.fcc_lattice(7.5)
    B1 = synth.reciprocal_rows(A1)
    out.append(synth.build_problem(A1, np.zeros((1, 3)), (0, 1, 2), 24, 40.0,
                                   synth.mp_grid(B1, (2, 2, 2))[[0, 3, 5]], 5, 71))
    A2 = synth.sc_lattice(6.0)
    B2 = synth.reciprocal_rows(A2)
    out.append(synth.build_problem(A2, 6.0 * np.array([[0, 0, 0], [0.5, 0.5, 0.5]]), (0, 1), 24, 30.0,
                                   synth.mp_grid(B2, (2, 1, 1)), 3, 72))
    A3 = synth.fcc_lattice(7.0)
    B3 = synth.reciprocal_rows(A3)
    c3 = synth.build_problem(A3, np.zeros((1, 3)), (0,), 24, 35.0, synth.mp_grid(B3, (1, 1, 2)), 4, 73)
    out.append(dataclasses.replace(c3, beta=np.ascontiguousarray(c3.beta[:, :0, :]), D=np.zeros((0, 0))))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_c128"])
def test_multi_cell_work_list_matches_oracle(precision):
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    cells = _cells()
    assert [c.nkb for c in cells] == [9, 8, 0]
    plans = [pwk.plan_from_problem(c) for c in cells]
    prec = pwk.PRECISIONS[precision]
    dt = torch.complex64 if precision == "fp32" else torch.complex128
    psis, refs = [], []
    for c in cells:
        psi = c.psi.astype(np.complex64).astype(np.complex128) if precision == "fp32" else c.psi
        psis.append(torch.from_numpy(np.ascontiguousarray(psi)).to("cuda", dt))
        refs.append(oracle_hpsi(c, psi=psi))
    outs = [torch.full_like(x, complex(np.nan, np.nan)) for x in psis]
    # interleaved over the cells, an empty slot, and not every vector of every cell
    items = []
    for b in range(5):
        for ip, c in enumerate(cells):
            for ik in range(c.nk):
                if b < c.nb and (ip != 0 or b != 4 or ik != 1):
                    items.append((ip, ik, b, b))
        items.append((-1, 0, 0, 0))
    it = torch.tensor(items, dtype=torch.int32, device="cuda")
    pwk.hpsi_multi(plans, prec, psis, outs, it)
    torch.cuda.synchronize()
    assert plans[0].errors() == 0
    done = {(p, k, b) for p, k, b, _ in items if p >= 0}
    for ip, c in enumerate(cells):
        o = outs[ip].cpu().numpy().astype(np.complex128)
        for ik in range(c.nk):
            n = c.npw[ik]
            for b in range(c.nb):
                if (ip, ik, b) in done:
                    ref = refs[ip][ik][b, :n]
                    e = np.linalg.norm(o[ik, b, :n] - ref) / np.linalg.norm(ref)
                    assert e <= TOL[precision], (ip, ik, b, e)
                    assert np.all(o[ik, b, n:] == 0)
                else:
                    assert np.isnan(o[ik, b]).all(), (ip, ik, b)
    for p in plans:
        p.close()


def test_multi_in_place_and_invalid_entries():
    """In place on one cell, an entry naming a plan that does not exist and one with a k-point
    outside its plan: both skipped and flagged, the valid entries applied."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    cells = _cells()[:2]
    plans = [pwk.plan_from_problem(c) for c in cells]
    x0 = torch.from_numpy(np.ascontiguousarray(cells[0].psi)).cuda()
    x1 = torch.from_numpy(np.ascontiguousarray(cells[1].psi)).cuda()
    y1 = torch.full_like(x1, complex(np.nan, np.nan))
    items = torch.tensor([(0, 0, 1, 1), (1, 1, 2, 0), (5, 0, 0, 0), (1, 7, 0, 0)], dtype=torch.int32,
                         device="cuda")
    pwk.hpsi_multi(plans, pwk.PWK_FP64, [x0, x1], [x0, y1], items)
    torch.cuda.synchronize()
    assert plans[0].errors() == pwk.PWK_FLAG_ITEM_SKIPPED
    r0 = oracle_hpsi(cells[0], ks=[0])[0]
    r1 = oracle_hpsi(cells[1], ks=[1])[1]
    o0 = x0.cpu().numpy()
    o1 = y1.cpu().numpy()
    n0, n1 = cells[0].npw[0], cells[1].npw[1]
    assert np.linalg.norm(o0[0, 1, :n0] - r0[1, :n0]) <= 1e-12 * np.linalg.norm(r0[1, :n0])
    assert np.array_equal(o0[0, 0], cells[0].psi[0, 0])          # not listed: untouched
    assert np.linalg.norm(o1[1, 0, :n1] - r1[2, :n1]) <= 1e-12 * np.linalg.norm(r1[2, :n1])
    assert np.isnan(o1[0]).all()
    for p in plans:
        p.close()


def test_multi_rejects_plans_of_different_grids():
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    a = synth.make_config(1, k_subset=[0], nb=2)       # 16^3
    b = synth.make_config(2, k_subset=[0], nb=2)       # 24^3
    pa, pb = pwk.plan_from_problem(a), pwk.plan_from_problem(b)
    xa = torch.from_numpy(a.psi).cuda()
    xb = torch.from_numpy(b.psi).cuda()
    it = torch.tensor([(0, 0, 0, 0)], dtype=torch.int32, device="cuda")
    with pytest.raises(pwk.PwkError) as ei:
        pwk.hpsi_multi([pa, pb], pwk.PWK_FP64, [xa, xb], [xa.clone(), xb.clone()], it)
    assert ei.value.code == -1
    pa.close()
    pb.close()
