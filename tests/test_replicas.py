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
    seeds = bench.rf_seeds(r, 4)
    pg.barrier()
    mx = bench.reduce_op(pg, float(10 * (r + 1)), torch.device("cpu"), "max")
    sm = bench.reduce_op(pg, float(r + 1), torch.device("cpu"), "sum")
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
    base = 2609 * 100 + 4
    assert s0 == [base + 7919 * i for i in range(4)] and s1 == [base + 7919 * i for i in range(4, 8)]
    assert mx0 == mx1 == 20.0
    assert sm0 == sm1 == 3.0


def test_every_rank_of_the_xxz_batch_has_stored_oracle_energies():
    """Replicas of the XXZ batch take instances from the stored oracle set
    (wrapping around it), so every rank's solves can be validated: a rank past
    the stored set must not get seeds without a reference."""
    import bench
    gold = bench.load_gold_xxz()
    for rank in range(8):
        seeds = bench.xxz_seeds(rank, 32, gold.keys())
        assert len(seeds) == 32 and all(s in gold for s in seeds)
    assert bench.xxz_seeds(0, 32, gold.keys()) == sorted(gold)[:32]
