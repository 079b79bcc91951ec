"""The multi-process (replica) path of bench.py on the CPU: two ranks over
gloo on 127.0.0.1 get disjoint instance batches (independent solves shard with
no exchange), and the timing and count reductions over ranks give the max and
the sum.  Whole solves are the unit of work, so the only collectives are these
reductions and the barriers around the timed region."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), RMC_BENCH_BACKEND="gloo")
    import bench
    import torch
    w, r, local, pg = bench.dist_setup()
    seeds = bench.batch_seeds(r, 4, list(range(100, 108)))
    pg.barrier()
    mx = bench.reduce_max(pg, float(10 * (r + 1)), torch.device("cpu"))
    sm = bench.reduce_sum(pg, float(r + 1), torch.device("cpu"))
    q.put((r, w, seeds, mx, sm))
    pg.destroy_process_group()


def test_two_rank_replicas_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, mx0, sm0), (r1, w1, s1, mx1, sm1) = out
    assert (w0, w1) == (2, 2)
    assert set(s0).isdisjoint(s1) and len(s0) == len(s1) == 4
    assert s0 == [100, 101, 102, 103] and s1 == [104, 105, 106, 107]
    assert mx0 == mx1 == 20.0
    assert sm0 == sm1 == 3.0


def test_seeds_beyond_the_stored_batch_are_fresh():
    import bench
    s = bench.batch_seeds(1, 4, [1, 2, 3])
    assert len(set(s)) == 4 and not set(s) & {1, 2, 3}
