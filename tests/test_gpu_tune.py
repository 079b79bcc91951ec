"""Autotuned tile shapes: a tuning solve fills the process-wide table for
the solver's Gram and basis-combination products, solves after it still
match the oracle, repeat solves are bitwise identical, and every candidate
configuration (forced through the table) gives results within the path's
tolerance -- candidates differ only in summation order."""
import re

import numpy as np
import pytest

import instances as I
from oracle import rmc_oracle as O
from tests.gpu_util import torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu
RTOL = {"fp64": 1e-10, "mixed": 1e-8}


@pytest.fixture(autouse=True)
def empty_table():
    P.tune_clear()
    yield
    P.tune_clear()


def _chain():
    rng = np.random.default_rng(7)
    return I.xxz(16, list(rng.uniform(0.5, 1.5, 15)), 1.0, 4, 32, 4)


def _close(prec, got, ref):
    assert np.all(np.abs(got - ref) <= RTOL[prec] * np.maximum(1.0, np.abs(ref))), (got - ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tuning_fills_the_table_and_keeps_results(prec):
    torch_cuda()
    c = _chain()
    ref = O.solve(c).energies
    with P.Context(precision=prec) as ctx:
        _close(prec, ctx.autotune(c), ref)
        table = P.tune_dump()
        keys = [ln.split("=")[0] for ln in table.splitlines()]
        assert any(k.startswith("gram|") for k in keys) and any(k.startswith("comb|") for k in keys), table
        E1 = ctx.solve_chain(c)
        E2 = ctx.solve_chain(c)
    _close(prec, E1, ref)
    assert np.array_equal(E1, E2)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_candidate_is_correct(prec):
    torch_cuda()
    c = _chain()
    ref = O.solve(c).energies
    with P.Context(precision=prec) as ctx:
        ctx.autotune(c)
        keys = [ln.split("=")[0] for ln in P.tune_dump().splitlines()]
        for cand in range(9):
            P.tune_clear()
            lines = []
            for k in keys:
                n = 9 if k.startswith("gram|") else 3
                lines.append(f"{k}={cand % n}")
            assert P.tune_load("\n".join(lines)) == len(keys)
            _close(prec, ctx.solve_chain(c), ref)
