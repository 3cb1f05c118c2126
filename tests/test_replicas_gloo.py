"""The replica path's host logic with two ranks over gloo on CPU: barrier,
maximum of the ranks' times, sum of their work, and the instance shards."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2311_16935_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        info = replicas.RankInfo.from_env()
        g = replicas.RankGroup(info, device="cpu")
        g.barrier()
        ms = 100.0 + 50.0 * rank          # rank 1 is the slowest
        units = 1e9 * (rank + 1)          # work both ranks did
        thr, ms_max = replicas.aggregate_throughput(units, ms, g)
        mine = list(replicas.shard(512, info.rank, info.world))
        g.barrier()
        out.put((rank, thr, ms_max, mine[0], mine[-1], len(mine)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the same aggregate: 3e9 units over the slowest 150 ms
    for rank, thr, ms_max, first, last, n in got:
        assert ms_max == 150.0
        assert thr == pytest.approx(3e9 / 0.150)
    assert [(g[3], g[4], g[5]) for g in got] == [(0, 255, 256), (256, 511, 256)]


@pytest.mark.parametrize("count,world", [(0, 3), (7, 3), (512, 8), (5, 8), (1, 1)])
def test_shards_cover_disjointly(count, world):
    seen = []
    for r in range(world):
        s = replicas.shard(count, r, world)
        seen.extend(s)
    assert seen == list(range(count))
    sizes = [len(replicas.shard(count, r, world)) for r in range(world)]
    assert max(sizes) - min(sizes) <= (1 if count else 0)


def test_single_rank_needs_no_process_group():
    g = replicas.RankGroup(replicas.RankInfo(0, 1, 0))
    g.barrier()
    assert g.max(3.5) == 3.5 and g.sum(2.0) == 2.0
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)
