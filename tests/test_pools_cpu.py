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
