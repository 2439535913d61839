"""Multi-GPU host logic (one replica per GPU): the unit sharding and the
cross-rank timing calls of bench.py, run here as two gloo processes on CPU.
The depth stage has no exchange step, so these calls are all there is."""
import os
import socket

import pytest

from paper_2201_11924_gb300 import replicas


@pytest.mark.parametrize("n,world", [(1, 1), (4, 1), (8, 2), (9, 2), (7, 4), (3, 8), (0, 2)])
def test_shard_is_a_partition(n, world):
    parts = [replicas.shard(n, r, world) for r in range(world)]
    flat = sorted(u for p in parts for u in p)
    assert flat == list(range(n))                               # every unit once
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1                         # balanced


def test_single_process_needs_no_group(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    rep = replicas.from_env()
    assert (rep.world, rep.rank, rep.distributed) == (1, 0, False)
    rep.barrier()
    assert rep.max_over_ranks(3.25) == 3.25
    rep.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    rep = replicas.from_env(backend="gloo")
    rep.barrier()
    # each rank reports a different elapsed time; all must see the slowest
    got = rep.max_over_ranks(10.0 + rank)
    mine = replicas.shard(4 * world, rep.rank, rep.world)
    rep.barrier()
    rep.close()
    out.put((rank, rep.world, got, mine))


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == world for r in res)
    assert all(r[2] == 11.0 for r in res)                       # max over ranks
    owned = sorted(u for r in res for u in r[3])
    assert owned == list(range(4 * world))                      # pairs split, none shared
