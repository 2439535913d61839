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


def _rank_that_leaves(rank, world, port, out):
    # rank 1 joins the group and exits without reaching the barrier; rank 0
    # must get an error from its barrier well before any default timeout
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    rep = replicas.from_env(backend="gloo", timeout_s=5.0)

    def report_and_exit(*msg):
        out.put(msg)
        out.close()
        out.join_thread()            # the message is written before the process ends
        os._exit(0)                  # no interpreter shutdown around a broken group

    if rank == 1:
        report_and_exit(rank, "left", 0.0)
    t0 = time.perf_counter()
    try:
        rep.barrier()
        rep.max_over_ranks(1.0)
        outcome = "no error"
    except Exception as e:                       # gloo: timeout or connection closed
        outcome = type(e).__name__
    report_and_exit(rank, outcome, time.perf_counter() - t0)


def test_a_rank_that_leaves_ends_the_others_wait_with_an_error():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_that_leaves, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (o, t)) for r, o, t in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
    assert res[1][0] == "left"
    outcome, waited = res[0]
    assert outcome != "no error"
    assert waited < 60.0


def _lonely_rank(port, out):
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK="0", LOCAL_RANK="0")
    t0 = time.perf_counter()
    try:
        replicas.from_env(backend="gloo", timeout_s=3.0)
        outcome = "no error"
    except Exception as e:                       # the rendezvous gives up
        outcome = type(e).__name__
    out.put((outcome, time.perf_counter() - t0))
    out.close()
    out.join_thread()
    os._exit(0)


def test_a_rank_that_never_joins_ends_the_rendezvous_with_an_error():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_lonely_rank, args=(_free_port(), q))
    p.start()
    outcome, waited = q.get(timeout=120)
    p.join(timeout=60)
    assert outcome != "no error"
    assert waited < 60.0
