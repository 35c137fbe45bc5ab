"""k-pool partition and the job-level aggregation of the multi-rank benchmark, with two gloo
ranks on CPU (the hot path itself has no collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2412_01695_gb300.pools import kpool_slice


@pytest.mark.parametrize("nk,world", [(512, 2), (513, 2), (7, 3), (1000, 8), (3, 4)])
def test_partition_covers_every_k_once(nk, world):
    seen = []
    for r in range(world):
        a, b = kpool_slice(nk, r, world)
        assert 0 <= a <= b <= nk
        seen += list(range(a, b))
    assert seen == list(range(nk))
    sizes = [kpool_slice(nk, r, world)[1] - kpool_slice(nk, r, world)[0] for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2412_01695_gb300.pools import aggregate, kpool_slice
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b = kpool_slice(512, rank, world)
    units = (b - a) * 20                 # band-k applications of this rank's pool
    seconds = 0.5 + 0.25 * rank           # a slower second rank
    total, tmax, w = aggregate(units, seconds)
    out[rank] = (total, tmax, w)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    total, tmax, w = res[0]
    assert w == 2 and total == 512 * 20 and abs(tmax - 0.75) < 1e-12


# ----------------------------------------------------------------------------- drho over pools
DRHO_KS = [0, 1, 517, 2049, 3000, 4095]     # six k-points of the DFPT cell, split over the pools
DRHO_NOCC = 2


def _drho_inputs():
    """Inputs of Eq. drho on the k-points DRHO_KS of the DFPT cell: the generator's orthonormal
    valence states at k and k+q, and a du with a conduction part (each valence vector's
    coefficients shifted by one plane wave)."""
    import numpy as np
    from paper_2412_01695_gb300 import synth
    pk = synth.make_config(4, k_subset=DRHO_KS, nb=DRHO_NOCC)
    pq = synth.make_config(4, k_subset=DRHO_KS, nb=DRHO_NOCC, shift_q=True)
    du = np.zeros_like(pq.psi)
    for i in range(pq.nk):
        n = pq.npw[i]
        du[i, :, :n] = np.roll(pq.psi[i, :, :n], 1, axis=1)
    return pk, pq, du


def _pool(prob, a, b):
    """The k-points [a, b) of a problem (the block a pool owns)."""
    import dataclasses
    return dataclasses.replace(prob, kpts=prob.kpts[a:b], npw=prob.npw[a:b], miller=prob.miller[a:b],
                               beta=prob.beta[a:b], psi=prob.psi[a:b])


def _pool_partial(a, b):
    """Pool [a, b)'s partial grid (a CPU stand-in for its pwk_drho_batched call), with the
    weights of the whole k-set."""
    import numpy as np
    from oracle import drho as odr
    pk, pq, du = _drho_inputs()
    pk, pq = _pool(pk, a, b), _pool(pq, a, b)
    return odr.drho(pk, pq, pk.psi, pq.psi, du[a:b], weights=np.full(b - a, 1.0 / len(DRHO_KS)))


def _drho_worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2412_01695_gb300.pools import kpool_slice, reduce_drho
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b = kpool_slice(len(DRHO_KS), rank, world)
    t = torch.from_numpy(np.ascontiguousarray(_pool_partial(a, b)))
    reduce_drho(t)
    out[rank] = t.numpy().copy()
    dist.barrier()
    dist.destroy_process_group()


def test_drho_summed_over_two_gloo_pools_equals_the_full_k_sum():
    """Eq. drho sums over every k: two pools, each holding three k-points, add their partial
    grids with one all-reduce, and both end with the oracle's sum over all six k-points."""
    import numpy as np
    from oracle import drho as odr
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_drho_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    pk, pq, du = _drho_inputs()
    ref = odr.drho(pk, pq, pk.psi, pq.psi, du)
    assert np.linalg.norm(ref) > 0
    for r in (0, 1):
        assert np.linalg.norm(res[r] - ref) <= 1e-13 * np.linalg.norm(ref)
    # one pool's grid alone is not the answer: the exchange is needed
    assert np.linalg.norm(_pool_partial(0, 3) - ref) > 1e-3 * np.linalg.norm(ref)


def test_reduce_drho_without_a_process_group_is_the_identity():
    import torch
    from paper_2412_01695_gb300.pools import reduce_drho
    t = torch.arange(8, dtype=torch.float64).reshape(2, 2, 2).to(torch.complex128)
    assert torch.equal(reduce_drho(t.clone()), t)
