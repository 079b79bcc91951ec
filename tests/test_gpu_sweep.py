"""The batched TFIM sweep at full size: 256 parameter points h on a uniform
grid in [0.2, 2.0] (J = 1), chain lengths N in {16, 24, 32, 48} and k in
{32, 64, 128} mixed, 4 lowest states each, solved together through the
solve server in the mixed precision (the batched launch configuration).

Checks (Sec. II Eqs. (12)-(13), Sec. III Eqs. (18)-(19)):
* every solve succeeds and every energy is a variational upper bound of the
  exact free-fermion energy of its chain;
* a stratified sample -- one point per (N, k) with k <= 64 -- matches the
  oracle within 1e-8 relative;
* for k = 128 (effective dimension 16384, too large for the dense oracle) one
  point per N matches the plain FP64 GPU path within 1e-8 relative.
"""
import numpy as np
import pytest

import instances as I
from oracle import closed_forms as CF
from oracle import rmc_oracle as O
from tests.gpu_util import torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sweep():
    torch_cuda()
    chains = I.sweep_points()
    E, st = P.solve_chains(chains, slots=16, precision="mixed")
    return chains, E, st


def _meta(c):
    return c.n_sites, c.k, -float(c.onsite[0][2])  # N, k, h


def test_every_point_solves_and_is_an_upper_bound(sweep):
    chains, E, st = sweep
    assert np.all(st == 0), np.nonzero(st)
    for i, c in enumerate(chains):
        N, k, h = _meta(c)
        exact = CF.tfim_lowest(N, 1.0, h, 4)
        # upper bound up to the mixed path's stated energy tolerance (1e-8 relative)
        assert np.all(E[i] >= exact - 1e-8 * np.abs(exact)), (c.name, E[i] - exact)


def test_stratified_sample_matches_the_oracle(sweep):
    chains, E, st = sweep
    seen = set()
    for i, c in enumerate(chains):
        N, k, h = _meta(c)
        if k > 64 or (N, k) in seen:
            continue
        seen.add((N, k))
        ref = O.solve(c).energies
        assert np.all(np.abs(E[i] - ref) <= 1e-8 * np.maximum(1, np.abs(ref))), (c.name, E[i] - ref)
    assert len(seen) == 8


def test_k128_points_match_the_fp64_gpu_path(sweep):
    chains, E, st = sweep
    pick, seen = [], set()
    for i, c in enumerate(chains):
        N, k, h = _meta(c)
        if k == 128 and N not in seen:
            seen.add(N)
            pick.append(i)
    ref, st64 = P.solve_chains([chains[i] for i in pick], slots=4, precision="fp64")
    assert np.all(st64 == 0)
    for j, i in enumerate(pick):
        assert np.all(np.abs(E[i] - ref[j]) <= 1e-8 * np.maximum(1, np.abs(ref[j]))), (chains[i].name, E[i] - ref[j])
