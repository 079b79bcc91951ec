"""Whole-chain parity (the recursion loop of Algorithm 1) against the oracle:
energies within 1e-10 relative (FP64 path) or 1e-8 (mixed path), at the
workload sizes, plus free-fermion and exact-diagonalisation checks."""
import json
import os

import numpy as np
import pytest

import instances as I
from oracle import closed_forms as CF
from oracle import rmc_oracle as O
from tests.gpu_util import torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
RTOL = {"fp64": 1e-10, "mixed": 1e-8, "mixed_tf32": 1e-8}


@pytest.fixture(scope="module", params=["fp64", "mixed", "mixed_tf32"])
def ctx(request):
    torch_cuda()
    c = P.Context(precision=request.param)
    yield c
    c.close()


def _close(ctx, got, ref):
    tol = RTOL[ctx.precision] * np.maximum(1.0, np.abs(ref))
    assert np.all(np.abs(got - ref) <= tol), (got - ref, tol)


def test_tfim_n8_k8_and_exact(ctx):
    g = json.load(open(os.path.join(GOLD, "tfim_n8.json")))
    c = I.tfim_n8()
    _close(ctx, ctx.solve_chain(c), np.array(g["energies_k8"]))
    c.k = 16
    _close(ctx, ctx.solve_chain(c), np.array(g["exact"]))


def test_xxz_n32_k64(ctx):
    g = json.load(open(os.path.join(GOLD, "xxz_n32_k64.json")))
    _close(ctx, ctx.solve_chain(I.xxz_n32()), np.array(g["energies"]))


@pytest.mark.parametrize("chain", [
    I.tfim(10, 1.0, 0.7, 5, 32, 6),                      # full k: exact
    I.tfim(7, 1.0, 1.3, 2, 128, 6),                      # unbalanced tree
    I.tfim(16, 1.0, 0.7, 4, 16, 4),
    I.tfim(24, 1.0, 1.4, 3, 32, 4),                      # L0 = 3 leaves
    I.xxz(12, list(np.random.default_rng(1).uniform(0.5, 1.5, 11)), 1.0, 3, 24, 6),
    I.xxz(8, [1.0] * 7, 1.0, 4, 16, 8, fields=[0.5, -1.2, 1.9, 0.1, -0.7, 1.1, -1.8, 0.3]),
    I.tfim(3, 1.0, 0.5, 4, 8, 3),                        # a single leaf is the whole chain
    # unbalanced trees under truncation (floor/ceil halving; swapping the
    # halves moves these energies by ~0.1, so parity pins the GPU's tree)
    I.xxz(11, [1.0] * 10, 1.0, 4, 12, 4, fields=list(np.random.default_rng(3).uniform(-2, 2, 11))),
    I.xxz(13, list(np.random.default_rng(4).uniform(0.5, 1.5, 12)), 1.0, 4, 10, 4),
    I.xxz(7, [1.0] * 6, 1.0, 2, 3, 3, fields=list(np.random.default_rng(5).uniform(-2, 2, 7))),
])
def test_chain_matches_oracle(ctx, chain):
    _close(ctx, ctx.solve_chain(chain), O.solve(chain).energies)


def test_full_k_tfim_matches_free_fermions(ctx):
    c = I.tfim(12, 1.0, 0.9, 3, 64, 8)
    _close(ctx, ctx.solve_chain(c), CF.tfim_lowest(12, 1.0, 0.9, 8))


def test_k256_random_field_chain_is_exact(ctx):
    """Random-field Heisenberg, 16 sites, leaves of 4, k = 256: the first level
    keeps every state (256 of 256, wider than one Rayleigh-Ritz block, so it is
    solved chunk by chunk with locking) and the top merge (dimension 65536) is
    then the exact problem: its lowest energies are the chain's exact ones."""
    rng = np.random.default_rng(31)
    c = I.xxz(16, [1.0] * 15, 1.0, 4, 256, 8, fields=list(rng.uniform(-2, 2, 16)))
    _close(ctx, ctx.solve_chain(c), O.sparse_exact_lowest(c, 8))


def test_truncated_energies_are_upper_bounds(ctx):
    c = I.tfim(32, 1.0, 0.7, 4, 16, 4)
    E = ctx.solve_chain(c)
    assert np.all(E >= CF.tfim_lowest(32, 1.0, 0.7, 4) - 1e-9)


def test_degenerate_k256_chain_mixed_agrees_with_fp64():
    """A 50-site Heisenberg chain (random couplings, SU(2) multiplets) with
    k = 256 from the serving mix: every merge keeps 256 of up to 65536 states,
    so each is solved chunk by chunk with a one-vector tail chunk above 256
    locked vectors.  The mixed path must converge and agree with the FP64 path
    (no oracle: the merges are too wide for dense FP64 on the host)."""
    torch_cuda()
    c = I.serving_requests(48, seed=I.seed_for(5))[45]
    assert (c.n_sites, c.k) == (50, 256)
    with P.Context(precision="fp64") as c64, P.Context(precision="mixed") as cm:
        ref = c64.solve_chain(c)
        got = cm.solve_chain(c)
    assert np.all(np.abs(got - ref) <= 1e-8 * np.maximum(1.0, np.abs(ref))), got - ref


WIDE_LEAF_CHAINS = [
    I.tfim(18, 1.0, 0.9, 9, 64, 4),                       # two 9-site leaves (D = 512): 4 + 5 sub-leaves each
    I.xxz(16, list(np.random.default_rng(41).uniform(0.5, 1.5, 15)), 1.0, 8, 48, 4),  # 8-site leaves (D = 256)
    I.tfim(9, 1.0, 0.8, 9, 64, 4),                        # the whole chain is one 9-site leaf
]


@pytest.mark.parametrize("chain", WIDE_LEAF_CHAINS, ids=lambda c: c.name)
def test_wide_leaves_match_oracle(ctx, chain):
    """Leaves wider than the dense leaf solver (L0 = 8, 9: D = 256, 512) are
    built as two dense sub-leaves keeping every state plus one merge keeping
    min(k, D); the oracle diagonalises the D x D leaf densely (Algorithm 1,
    first step)."""
    _close(ctx, ctx.solve_chain(chain), O.solve(chain).energies)


GEOMETRY_CHAINS = [I.two_module_tfim(g, jp, k) for g, jp, k in
                   [("I", 0.8, 8), ("II", 0.8, 8), ("III", 1.0, 10), ("IV", 0.6, 8), ("NNN", 0.8, 10)]] + [
    I.tfim_nnn(20, 1.0, 0.7, 0.2, 5, 16, 4),   # next-nearest bonds across every boundary
    I.tfim_nnn(24, 1.0, 1.0, 0.2, 3, 32, 4),   # leaves of 3: carried operators on interior sites
]


@pytest.mark.parametrize("chain", GEOMETRY_CHAINS, ids=lambda c: c.name)
def test_coupling_geometries_match_oracle(ctx, chain):
    """The inter-module coupling geometries of Appendix C (A5-B1, A5-B2,
    A5-B3, A3-B3 and the next-nearest form with gamma = 0.2) and whole chains
    with next-nearest couplings: every term crossing a boundary carries its
    inside end, wherever that site is in the block."""
    _close(ctx, ctx.solve_chain(chain), O.solve(chain).energies)


def test_leaf_limits_are_rejected(ctx):
    with pytest.raises(P.RmcError) as e:
        ctx.solve_chain(I.tfim(16, 1.0, 0.9, 8, 256, 4))   # k keeps a whole 8-site leaf
    assert e.value.status == P.RMC_ERR_INVAL
    with pytest.raises(P.RmcError) as e:
        ctx.solve_chain(I.tfim(30, 1.0, 0.9, 15, 16, 4))   # leaves of 15 sites
    assert e.value.status == P.RMC_ERR_INVAL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_level_batches_equal_one_merge_at_a_time(precision):
    """rmc_solve_chain runs the merges of each level on the context's lanes;
    the energies equal those of one merge at a time (lanes = 1) bit for bit."""
    torch_cuda()
    c = I.xxz(32, [1.0] * 31, 1.0, 4, 32, 6, fields=list(np.random.default_rng(61).uniform(-2, 2, 32)))
    with P.Context(precision=precision, lanes=1) as one, P.Context(precision=precision) as many:
        np.testing.assert_array_equal(one.solve_chain(c), many.solve_chain(c))
