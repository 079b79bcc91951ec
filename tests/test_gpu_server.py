"""Batched and served solves (continuous batching over concurrent slots).

Each result is the same alone and in the mix: requests of different models,
sizes and k run concurrently on several slots, and every energy matches the
single-context solve of the same chain within the path's tolerance (and the
oracle).  Admission respects the memory budget; a request that can never fit
is refused at submission; a failing request does not disturb the others.
"""
import time

import numpy as np
import pytest

import instances as I
from oracle import rmc_oracle as O
from tests.gpu_util import torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu


def _mix():
    rng = np.random.default_rng(77)
    return [
        I.tfim(8, 1.0, 0.8, 2, 8, 4),
        I.xxz(12, list(rng.uniform(0.5, 1.5, 11)), 1.0, 3, 24, 6),
        I.tfim(16, 1.0, 0.7, 4, 16, 4),
        I.xxz(8, [1.0] * 7, 1.0, 4, 16, 8, fields=list(rng.uniform(-2, 2, 8))),
        I.tfim(24, 1.0, 1.4, 3, 32, 4),
        I.tfim(10, 1.0, 0.7, 5, 32, 6),
        I.xxz(16, list(rng.uniform(0.5, 1.5, 15)), 1.0, 4, 32, 5),
        I.tfim(3, 1.0, 0.5, 4, 8, 3),
    ]


@pytest.mark.parametrize("prec,rtol", [("mixed", 1e-8), ("fp64", 1e-10)])
def test_same_alone_and_in_the_mix(prec, rtol):
    torch_cuda()
    chains = _mix()
    with P.Context(precision=prec) as ctx:
        alone = [ctx.solve_chain(c) for c in chains]
    E, st = P.solve_chains(chains, slots=4, precision=prec)
    assert np.all(st == 0), st
    for i, c in enumerate(chains):
        got = E[i, :c.q]
        np.testing.assert_allclose(got, alone[i], rtol=0, atol=rtol * max(1, np.abs(alone[i]).max()))
        ref = O.solve(c).energies
        assert np.all(np.abs(got - ref) <= rtol * np.maximum(1, np.abs(ref)))


def test_server_poll_latency_and_stats():
    torch_cuda()
    chains = _mix()
    with P.Server(slots=3, precision="mixed") as srv:
        ids = [srv.submit(c) for c in chains]
        pending = set(ids)
        results = {}
        t0 = time.time()
        while pending and time.time() - t0 < 120:
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    results[t] = r
                    pending.discard(t)
            time.sleep(0.001)
        assert not pending
        st = srv.stats()
        assert st["submitted"] == len(chains) and st["completed"] == len(chains)
        assert st["running"] == 0 and st["queued"] == 0 and st["reserved_bytes"] == 0
        assert st["launches"] > 0
        for t, c in zip(ids, chains):
            E, status, lat, qd = results[t]
            assert status == 0 and lat >= qd >= 0
            ref = O.solve(c).energies
            assert np.all(np.abs(E - ref) <= 1e-8 * np.maximum(1, np.abs(ref)))


def test_admission_respects_the_memory_budget():
    torch_cuda()
    chains = [I.xxz(16, [1.0] * 15, 1.0, 4, 32, 4) for _ in range(4)]
    need = P.estimate_bytes(chains[0])
    # room for one solve at a time: the others wait in the queue
    with P.Server(slots=4, precision="mixed", mem_budget=int(1.5 * need)) as srv:
        ids = [srv.submit(c) for c in chains]
        max_running = 0
        t0 = time.time()
        while srv.stats()["completed"] < len(chains) and time.time() - t0 < 120:
            max_running = max(max_running, srv.stats()["running"])
            time.sleep(0.0005)
        assert max_running <= 1
        outs = [srv.poll(t, wait=True) for t in ids]
        assert all(o[1] == 0 for o in outs)
        np.testing.assert_array_equal(outs[0][0], outs[3][0])


def test_oversized_request_is_refused_and_failures_are_isolated():
    torch_cuda()
    big = I.rf_heisenberg_n128()
    with P.Server(slots=2, precision="mixed", mem_budget=64 << 20) as srv:
        with pytest.raises(P.RmcError) as e:
            srv.submit(big)
        assert e.value.status == P.RMC_ERR_NOMEM
        bad = I.tfim(8, 1.0, 0.8, 2, 8, 4)
        bad.onsite = [(0, "Y", 1.0)] + bad.onsite       # imaginary field: rejected by the solver
        good = I.tfim(8, 1.0, 0.8, 2, 8, 4)
        tb, tg = srv.submit(bad), srv.submit(good)
        rb, rg = srv.poll(tb, wait=True), srv.poll(tg, wait=True)
        assert rb[1] == P.RMC_ERR_INVAL
        assert rg[1] == 0
        np.testing.assert_allclose(rg[0], O.solve(good).energies, atol=1e-8 * 10)
