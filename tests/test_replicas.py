"""Multi-GPU layout of the benchmarks (replicas): the shard of every rank, and the timing
reductions across ranks, run as two gloo processes on the CPU."""
import os
import socket

import pytest

from paper_2607_12656_b300 import replicas


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (64, 2), (64, 3), (7, 8), (1000, 4)])
def test_shards_partition_the_items(n, world):
    got = [i for r in range(world) for i in replicas.shard(n, r, world)]
    assert got == list(range(n))  # disjoint, in order, covering everything
    sizes = [len(replicas.shard(n, r, world)) for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_ranks():
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)
    with pytest.raises(ValueError):
        replicas.shard(10, 0, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = replicas.rank_info()
    mine = list(replicas.shard(10, r, w))
    t_max = replicas.max_over_ranks(1.5 + r)       # the slowest rank sets the time
    units = replicas.sum_over_ranks(len(mine))      # units decoded by the whole job
    out.put((r, w, local, mine, t_max, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing_and_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert res[0][3] + res[1][3] == list(range(10))
    assert all(r[4] == 2.5 for r in res) and all(r[5] == 10 for r in res)


def test_single_process_needs_no_group():
    assert replicas.max_over_ranks(3.0) == 3.0 and replicas.sum_over_ranks(4) == 4.0
