"""GPU parity of pwk_hpsi_batched / pwk_hpsi_items against the FP64 oracle (through the C ABI).

Tolerances: FP64 path <= 1e-12 relative per band-k (||dH psi||_2 / ||H psi||_2), the stated
bound of the FP64 path.  FP32 paths <= 5e-6: FP32 unit roundoff 6e-8 times the growth of
the transform pair (about 2 log2 N^3 ~ 30 rounding steps) and the ratio
max|V| ||psi|| / ||H psi|| (<= 4 on these cells) gives <= 7e-6 as a worst case; the
measured errors are about ten times smaller.
"""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from paper_2412_01695_gb300 import synth

from gpu_util import max_rel_err, oracle_hpsi, run_hpsi, torch_cuda

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 5e-6


@pytest.fixture(scope="module")
def cfg1():
    return synth.make_config(1)


def test_fp64_cfg1_all(cfg1):
    ref = oracle_hpsi(cfg1)
    out = run_hpsi(cfg1, "fp64")
    assert max_rel_err(out, ref, cfg1) <= TOL64


@pytest.mark.parametrize("precision", ["fp32", "fp32_c128"])
def test_fp32_cfg1_all(cfg1, precision):
    ref = oracle_hpsi(cfg1)
    psi = cfg1.psi.astype(np.complex64).astype(np.complex128) if precision == "fp32" else None
    out = run_hpsi(cfg1, precision, psi=psi)
    if psi is not None:
        ref = oracle_hpsi(cfg1, psi=psi)
    err = max_rel_err(out, ref, cfg1)
    assert err <= TOL32, err


@pytest.mark.parametrize("cfg,nks", [(2, 6), (3, 3), (4, 5)])
def test_fp64_subsets(cfg, nks):
    """Ragged npw(k), N = 24 / 36 / 20, nkb = 9 / 36 / 9; several tiles and chunks."""
    nkfull = int(np.prod(synth.CONFIGS[cfg]["mp"]))
    prob = synth.make_config(cfg, k_subset=synth.sample_k(nkfull, nks), nb=min(6, synth.CONFIGS[cfg]["nb"]))
    assert len(set(prob.npw.tolist())) > 1 or nks == 1
    ref = oracle_hpsi(prob)
    out = run_hpsi(prob, "fp64")
    assert max_rel_err(out, ref, prob) <= TOL64
    out32 = run_hpsi(prob, "fp32_c128")
    assert max_rel_err(out32, ref, prob) <= TOL32


def test_kq_points():
    """The k+q set of the DFPT cell (shifted grid, same spheres' shape)."""
    prob = synth.make_config(4, k_subset=[0, 1, 77, 4095], shift_q=True, nb=4)
    ref = oracle_hpsi(prob)
    assert max_rel_err(run_hpsi(prob, "fp64"), ref, prob) <= TOL64


def test_free_electron_exact():
    """V = 0, D = 0: H psi = |k+G|^2 psi up to the rounding of the transform pair of zeros."""
    prob = synth.make_config(1)
    prob.V_r = np.zeros_like(prob.V_r)
    prob.D = np.zeros_like(prob.D)
    out = run_hpsi(prob, "fp64")
    for ik in range(prob.nk):
        n = prob.npw[ik]
        g2 = ham.kinetic(prob.kpts[ik], prob.miller[ik, :n], prob.B)
        np.testing.assert_allclose(out[ik][:, :n], prob.psi[ik][:, :n] * g2, rtol=0, atol=1e-14)


def test_constant_potential_shift(cfg1):
    """Adding a constant c to V adds c psi exactly (up to rounding)."""
    a = run_hpsi(cfg1, "fp64")
    p2 = synth.make_config(1)
    p2.V_r = p2.V_r + 0.37
    b = run_hpsi(p2, "fp64")
    for ik in range(cfg1.nk):
        n = cfg1.npw[ik]
        np.testing.assert_allclose(b[ik][:, :n] - a[ik][:, :n], 0.37 * cfg1.psi[ik][:, :n], atol=1e-12)


def test_no_projectors_single_band_single_k():
    prob = synth.make_config(2, k_subset=[5], nb=1)
    prob.beta = prob.beta[:, :0, :]
    prob.D = np.zeros((0, 0))
    ref = oracle_hpsi(prob)
    assert max_rel_err(run_hpsi(prob, "fp64"), ref, prob) <= TOL64


def test_items_uneven_and_inplace():
    """pwk_hpsi_items on an uneven list: only listed vectors change; invalid entries are
    skipped; in-place (psi == hpsi) works for pwk_hpsi_batched."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(2, k_subset=[0, 100, 200, 511], nb=5)
    ref = oracle_hpsi(prob)
    plan = pwk.plan_from_problem(prob)
    x = torch.from_numpy(prob.psi.copy()).cuda()
    y = torch.zeros_like(x)
    items = np.array([[0, 0, 4], [3, 4, 0], [1, 2, 2], [2, 1, 3], [1, 3, 1],
                      [9, 0, 0], [0, 7, 0], [-1, 0, 0]], np.int32)   # last three invalid
    pwk.hpsi_items(plan, pwk.PWK_FP64, x, y, torch.from_numpy(items).cuda(), 5)
    torch.cuda.synchronize()
    out = y.cpu().numpy()
    touched = set()
    for k, i, o in items[:5]:
        n = prob.npw[k]
        e = ham.relative_error(out[k, o, :n], ref[k][i, :n])
        assert e <= TOL64
        touched.add((k, o))
    for k in range(4):
        for o in range(5):
            if (k, o) not in touched:
                assert np.all(out[k, o] == 0)
    # in place
    pwk.hpsi_batched(plan, pwk.PWK_FP64, x, x, 5)
    torch.cuda.synchronize()
    assert max_rel_err(x.cpu().numpy(), ref, prob) <= TOL64
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_full_size_cfg2_sampled(precision, tol):
    """Full 512 k x 20 bands batch in the launch configuration the benchmark times; the
    oracle checks a seeded sample of k-points (all their bands)."""
    prob = synth.make_config(2)
    psi = prob.psi.astype(np.complex64).astype(np.complex128) if precision == "fp32" else prob.psi
    out = run_hpsi(prob, precision, psi=psi)
    ks = synth.sample_k(prob.nk, 6, seed=11)
    ref = oracle_hpsi(prob, psi=psi, ks=ks)
    assert max_rel_err(out, ref, prob, ks=ks) <= tol
    assert np.all(np.isfinite(out))


def test_large_grid_n48():
    """Largest instantiated grid (N = 48) on a small simple-cubic cell."""
    A = synth.sc_lattice(6.0)
    B = synth.reciprocal_rows(A)
    k = synth.mp_grid(B, (2, 2, 2))[[0, 7]]
    prob = synth.build_problem(A, np.zeros((1, 3)), (0, 1, 2), 48, 40.0, k, 3, 9)
    ref = oracle_hpsi(prob)
    assert max_rel_err(run_hpsi(prob, "fp64"), ref, prob) <= TOL64
    assert max_rel_err(run_hpsi(prob, "fp32_c128"), ref, prob) <= TOL32


def test_sphere_too_large_for_shared_memory_is_rejected():
    """A sphere whose z-sticks do not fit in shared memory is refused at plan creation
    (PWK_ERR_UNSUPPORTED), never launched."""
    from paper_2412_01695_gb300 import pwk
    A = synth.sc_lattice(8.0)
    B = synth.reciprocal_rows(A)
    k = synth.mp_grid(B, (1, 1, 1))
    prob = synth.build_problem(A, np.zeros((1, 3)), (0,), 48, 75.0, k, 1, 9, with_psi=False)
    with pytest.raises(pwk.PwkError) as ei:
        pwk.plan_from_problem(prob)
    assert ei.value.code == -2


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_c128"])
def test_every_launch_shape_gives_identical_results(precision):
    """Every (kernel kind, threads, l3 chunk) the autotuner may pick computes the same H|psi>:
    bitwise identical within a kernel kind and between the two window kernels (kinds 1 and 2
    do the same arithmetic per line), every kind within the precision's tolerance of the
    oracle."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(2, k_subset=[0, 3, 300], nb=4)
    ref = oracle_hpsi(prob)
    plan = pwk.plan_from_problem(prob)
    prec = pwk.PRECISIONS[precision]
    dt = torch.complex64 if precision == "fp32" else torch.complex128
    x = torch.from_numpy(prob.psi).cuda().to(dt)
    tol = TOL64 if precision == "fp64" else TOL32
    outs = {}
    for kind in (0, 1, 2):
        for T in (96, 128, 192, 256):
            for L in ((24, 12, 8, 6, 5) if kind < 2 else (1, 2)):
                try:
                    plan.set_launch_shape(prec, kind, T, L)
                except pwk.PwkError as e:
                    assert e.code == -2
                    continue
                y = torch.full_like(x, complex(np.nan, np.nan))
                pwk.hpsi_batched(plan, prec, x, y, prob.nb)
                torch.cuda.synchronize()
                out = y.cpu().numpy().astype(np.complex128)
                assert max_rel_err(out, ref, prob) <= tol, (kind, T, L)
                key = min(kind, 1)   # kinds 1 and 2 agree bit for bit
                if key in outs:
                    assert np.array_equal(out, outs[key]), (kind, T, L)
                else:
                    outs[key] = out
    assert set(outs) == {0, 1}
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "fp32_c128"])
@pytest.mark.parametrize("cfg,nks,nb", [(2, 6, 20), (1, 8, 8), (4, 5, 12), (2, 3, 44), (3, 2, 40), (3, 2, 7),
                                       (3, 3, 64)])
def test_tensor_core_projections_match_cuda_cores_and_oracle(precision, cfg, nks, nb):
    """The FP32 projector contractions on the tensor cores (projection and add-back, three TF32
    products of a hi/lo split each) and on the CUDA cores both meet the FP32 bound against the
    oracle, and agree with each other to FP32 rounding: 4, 9 and 36 projectors (cell 3: four
    atoms), 7 to 64 bands, one and several tiles of 128 plane waves, ragged last tiles, the
    H C tile of the add-back staged in shared memory or (where it does not fit: complex128
    I/O with 40 bands, 64 bands) read in place, both depths of the projection's copy ring."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    nkfull = int(np.prod(synth.CONFIGS[cfg]["mp"]))
    prob = synth.make_config(cfg, k_subset=synth.sample_k(nkfull, nks), nb=nb)
    psi = prob.psi.astype(np.complex64).astype(np.complex128) if precision == "fp32" else prob.psi
    ref = oracle_hpsi(prob, psi=psi)
    plan = pwk.plan_from_problem(prob)
    prec = pwk.PRECISIONS[precision]
    dt = torch.complex64 if precision == "fp32" else torch.complex128
    x = torch.from_numpy(np.ascontiguousarray(psi)).to("cuda", dt)
    outs = []
    for path in (2, 1):
        plan.set_projector_path(path)
        y = torch.full_like(x, complex(np.nan, np.nan))
        pwk.hpsi_batched(plan, prec, x, y, prob.nb)
        torch.cuda.synchronize()
        outs.append(y.cpu().numpy().astype(np.complex128))
        assert max_rel_err(outs[-1], ref, prob) <= TOL32, (path, max_rel_err(outs[-1], ref, prob))
    d = max(np.linalg.norm(outs[0][ik] - outs[1][ik]) / np.linalg.norm(outs[1][ik]) for ik in range(prob.nk))
    assert d <= 2e-6, d
    plan.close()


def test_device_flags_report_skipped_items_and_wait_timeouts():
    """The plan's device flags: a work-list entry outside the plan is reported as skipped; a
    tensor-core wait that gives up (every wait bounded to zero polls, so no MMA is ever issued)
    is reported as a timeout; the plan then works again once the bound is restored."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(2, k_subset=[0, 7, 99], nb=4)
    plan = pwk.plan_from_problem(prob)
    assert plan.errors() == 0
    x = torch.from_numpy(prob.psi).cuda()
    y = torch.zeros_like(x)
    items = torch.tensor([[0, 0, 0], [5, 0, 0]], dtype=torch.int32, device="cuda")   # k = 5 outside
    pwk.hpsi_items(plan, pwk.PWK_FP64, x, y, items, prob.nb)
    torch.cuda.synchronize()
    assert plan.errors() & pwk.PWK_FLAG_ITEM_SKIPPED
    assert plan.errors() == 0   # cleared by the previous read
    x32 = x.to(torch.complex64)
    y32 = torch.zeros_like(x32)
    plan.set_projector_path(1)
    plan.set_wait_limit(0)
    pwk.hpsi_batched(plan, pwk.PWK_FP32, x32, y32, prob.nb)
    torch.cuda.synchronize()
    assert plan.errors() & pwk.PWK_FLAG_WAIT_TIMEOUT
    plan.set_wait_limit(1 << 24)
    pwk.hpsi_batched(plan, pwk.PWK_FP32, x32, y32, prob.nb)
    torch.cuda.synchronize()
    assert plan.errors() == 0
    ref = oracle_hpsi(prob, psi=x32.cpu().numpy().astype(np.complex128))
    assert max_rel_err(y32.cpu().numpy().astype(np.complex128), ref, prob) <= TOL32
    with pytest.raises(pwk.PwkError):
        plan.set_wait_limit(-1)
    plan.close()


def test_empty_and_invalid_requests():
    """Degenerate requests through the C ABI: nb = 0 and an unknown precision are errors
    (PWK_ERR_INVALID, nothing launched); an empty work list is a no-op that leaves the
    output as it was."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(1, k_subset=[0, 3], nb=2)
    plan = pwk.plan_from_problem(prob)
    x = torch.from_numpy(prob.psi.copy()).cuda()
    y = torch.full_like(x, 7.0 - 3.0j)
    empty = torch.empty((prob.nk, 0, prob.npw_max), dtype=torch.complex128, device="cuda")
    with pytest.raises(pwk.PwkError) as err:
        pwk.hpsi_batched(plan, pwk.PWK_FP64, empty, empty, 0)
    assert err.value.code == -1
    with pytest.raises(pwk.PwkError) as err:
        pwk.hpsi_batched(plan, 3, x, y, prob.nb)
    assert err.value.code == -1
    pwk.hpsi_items(plan, pwk.PWK_FP64, x, y, None, prob.nb)
    torch.cuda.synchronize()
    assert bool(torch.all(y == (7.0 - 3.0j)))
    # the plan still works after the rejected calls
    pwk.hpsi_batched(plan, pwk.PWK_FP64, x, y, prob.nb)
    torch.cuda.synchronize()
    assert max_rel_err(y.cpu().numpy(), oracle_hpsi(prob), prob) <= TOL64
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_c128"])
@pytest.mark.parametrize("cfg,nks,nb", [(1, 8, 8), (2, 4, 6), (3, 2, 4), (4, 5, 12)])
def test_projector_paths_match_the_oracle(precision, cfg, nks, nb):
    """The projector terms applied by separate CUDA-core kernels (path 2) and inside the local
    kernel (path 3: one HBM round trip per band-k, beta(k) staged in shared memory after the
    transforms) both meet the bound against the oracle, for the batched call and an uneven
    work list applied in place."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    nkfull = int(np.prod(synth.CONFIGS[cfg]["mp"]))
    prob = synth.make_config(cfg, k_subset=synth.sample_k(nkfull, nks), nb=nb)
    psi = prob.psi.astype(np.complex64).astype(np.complex128) if precision == "fp32" else prob.psi
    ref = oracle_hpsi(prob, psi=psi)
    plan = pwk.plan_from_problem(prob)
    prec = pwk.PRECISIONS[precision]
    tol = TOL64 if precision == "fp64" else TOL32
    dt = torch.complex64 if precision == "fp32" else torch.complex128
    x = torch.from_numpy(np.ascontiguousarray(psi)).to("cuda", dt)
    x_host = x.cpu().numpy().astype(np.complex128)
    for path in (2, 3):
        plan.set_projector_path(path)
        # path 3 stages beta(k) in shared memory in the window kernels; cell 3's does not fit
        # there, and the general kernel (kind 0) reads it through L1/L2 instead
        if path == 2 or cfg != 3:
            assert plan.projector_fused(prec) == (path == 3)
            assert plan.projector_choice(prec) == path
        y = torch.full_like(x, complex(np.nan, np.nan))
        pwk.hpsi_batched(plan, prec, x, y, prob.nb)
        torch.cuda.synchronize()
        out = y.cpu().numpy().astype(np.complex128)
        assert max_rel_err(out, ref, prob) <= tol, (path, max_rel_err(out, ref, prob))
        # uneven work list, in place: every other band of each k, the rest untouched
        items = np.array([[ik, b, b] for ik in range(prob.nk) for b in range(0, nb, 2)], np.int32)
        z = x.clone()
        pwk.hpsi_items(plan, prec, z, z, torch.from_numpy(items).cuda(), nb)
        torch.cuda.synchronize()
        zo = z.cpu().numpy().astype(np.complex128)
        for ik in range(prob.nk):
            n = prob.npw[ik]
            for b in range(nb):
                if b % 2 == 0:
                    e = np.linalg.norm(zo[ik, b, :n] - ref[ik][b, :n]) / np.linalg.norm(ref[ik][b, :n])
                    assert e <= tol, (path, ik, b, e)
                    assert np.all(zo[ik, b, n:] == 0)
                else:
                    assert np.array_equal(zo[ik, b], x_host[ik, b])
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_projectors_every_launch_shape_identical(precision):
    """With the projector terms inside the local kernel (path 3) every window-kernel shape
    gives the same bits: the projections are summed in an order that does not depend on the
    number of warps, the add-back per plane wave in projector order."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(2, k_subset=[0, 3, 300], nb=4)
    ref = oracle_hpsi(prob)
    plan = pwk.plan_from_problem(prob)
    plan.set_projector_path(3)
    prec = pwk.PRECISIONS[precision]
    dt = torch.complex64 if precision == "fp32" else torch.complex128
    x = torch.from_numpy(prob.psi).cuda().to(dt)
    first = None
    for kind in (1, 2):
        for T in (96, 128, 192, 256):
            for L in ((24, 12, 8, 6) if kind == 1 else (1, 2)):
                try:
                    plan.set_launch_shape(prec, kind, T, L)
                except pwk.PwkError as e:
                    assert e.code == -2
                    continue
                if not plan.projector_fused(prec):
                    continue
                y = torch.full_like(x, complex(np.nan, np.nan))
                pwk.hpsi_batched(plan, prec, x, y, prob.nb)
                torch.cuda.synchronize()
                out = y.cpu().numpy().astype(np.complex128)
                if first is None:
                    first = out
                    assert max_rel_err(out, ref, prob) <= (TOL64 if precision == "fp64" else TOL32)
                else:
                    assert np.array_equal(out, first), (kind, T, L)
    assert first is not None
    plan.close()


def test_launch_count_follows_the_projector_path():
    """pwk_launch_count counts the kernels the library queues: one H|psi> call is one launch
    with the projector terms inside the local kernel (path 3), three with the separate
    CUDA-core kernels (path 2), and none for an empty work list."""
    torch = torch_cuda()
    from paper_2412_01695_gb300 import pwk
    prob = synth.make_config(2, k_subset=[0, 3, 300], nb=4)
    plan = pwk.plan_from_problem(prob)
    x = torch.from_numpy(prob.psi).cuda().to(torch.complex64)
    y = torch.empty_like(x)
    for path, launches in ((3, 1), (2, 3)):
        plan.set_projector_path(path)
        pwk.hpsi_batched(plan, pwk.PWK_FP32, x, y, prob.nb)   # first call: any one-time set-up
        torch.cuda.synchronize()
        c0 = pwk.launch_count()
        pwk.hpsi_batched(plan, pwk.PWK_FP32, x, y, prob.nb)
        torch.cuda.synchronize()
        assert pwk.launch_count() - c0 == launches, (path, pwk.launch_count() - c0)
    c0 = pwk.launch_count()
    pwk.hpsi_items(plan, pwk.PWK_FP32, x, y, None, prob.nb)
    assert pwk.launch_count() == c0
    plan.close()
