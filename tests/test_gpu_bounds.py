"""Per-merge truncation diagnostics on the GPU (Sec. IV and Appendix B):
a = lambda_min(PHP), b = ||PVQ||_2 in Kronecker form (Appendix B's
expression), bH = ||PHQ||_2 on the block's full space, gamma =
lambda_min(QHQ) - a, the bound r(bH, gamma) and the merged block's exact
ground energy E0, merge by merge, against the oracle's dense definitions
(oracle/error_bounds.py: merge_bound and b_from_products) for the paper's
ten-site validation (J = 1, h = 0.7, 5 + 5 sites, every k) and for deeper
Ising and Heisenberg trees (where the modules are themselves truncated, so b
and bH differ); the twenty-site validation, beyond the oracle's dense
matrices, against the free-fermion ground energies and the bound chain
0 <= a - E0 <= r <= bH^2 / gamma the paper states."""
import numpy as np
import pytest

import instances as I
from oracle import closed_forms as CF
from oracle import error_bounds as EB
from oracle import rmc_oracle as O
from tests.gpu_util import torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu

# energies: the path's own tolerance; b, gamma and r inherit the retained
# bases' accuracy (first order in them), E0 only the Krylov solve's
TOL = {"fp64": {"a": 1e-10, "b": 1e-9}, "mixed": {"a": 1e-8, "b": 1e-7}}


@pytest.fixture(scope="module", params=["fp64", "mixed"])
def ctx(request):
    torch_cuda()
    c = P.Context(precision=request.param)
    yield c
    c.close()


def oracle_merges(chain):
    """(A, B) of every merge of the oracle's recursion, children first."""
    out = []

    def walk(blk):
        if blk.is_leaf:
            return
        A, B = blk.children
        walk(A)
        walk(B)
        out.append((A, B))

    walk(O.solve(chain).top)
    return out


def check_bound_chain(d, tol):
    assert d["gamma"] > 0
    assert -tol <= d["a"] - d["E0"] <= d["r"] + tol
    assert d["r"] <= d["bH"] ** 2 / d["gamma"] + tol


def compare(ctx, chain, full_sites):
    E, diag = ctx.solve_chain_bounds(chain, full_space_sites=full_sites)
    refs = oracle_merges(chain)
    assert len(diag) == len(refs)
    t = TOL[ctx.precision]
    for d, (A, B) in zip(diag, refs):
        assert (d["lo"], d["mid"], d["hi"]) == (A.lo, A.hi, B.hi)
        assert (d["kA"], d["kB"]) == (len(A.E), len(B.E))
        ref = EB.merge_bound(chain, A, B)
        bv = EB.b_from_products(chain, A, B)
        assert abs(d["a"] - ref["a"]) <= t["a"] * max(1.0, abs(ref["a"])), (d, ref)
        # compared squared: the oracle's b of a fully kept sector is the square
        # root of rounding noise (~1e-8), the GPU's is exactly 0
        assert abs(d["b"] ** 2 - bv ** 2) <= t["b"] * max(1.0, bv ** 2), (d, bv)
        assert abs(d["bH"] - ref["b"]) <= t["b"] * max(1.0, ref["b"]), (d, ref)
        if A.is_leaf and B.is_leaf:   # Appendix B: P H Q = P V Q for exact module eigenstates
            assert abs(d["b"] - d["bH"]) <= t["b"] * max(1.0, d["b"])
        assert abs(d["E0"] - ref["E0"]) <= 1e-10 * max(1.0, abs(ref["E0"])), (d, ref)
        if np.isinf(ref["gamma"]):
            assert np.isinf(d["gamma"]) and d["r"] == 0.0
        else:
            assert abs(d["gamma"] - ref["gamma"]) <= t["b"] * max(1.0, abs(ref["gamma"])), (d, ref)
            assert abs(d["r"] - ref["r"]) <= t["b"] * max(1.0, ref["r"]), (d, ref)
            check_bound_chain(d, 1e-9)
    return E, diag


@pytest.mark.parametrize("k", [2, 3, 4, 8, 16, 24])
def test_ten_site_validation(ctx, k):
    """Appendix B figure, L = 10: two five-site modules, every k."""
    compare(ctx, I.tfim(10, 1.0, 0.7, 5, k, 4), 10)


@pytest.mark.parametrize("chain", [
    I.tfim(10, 1.0, 0.9, 3, 5, 4),                                               # merges of merges
    I.xxz(8, [0.7, 1.1, 0.9, 1.4, 0.6, 1.2, 1.0], 1.0, 2, 6, 4),                 # three operators a bond
    I.xxz(8, [1.0] * 7, 1.0, 2, 5, 4, fields=[0.3, -1.2, 0.8, 1.9, -0.4, 0.1, -1.5, 0.6]),
], ids=["tfim10_L3", "xxz8_L2", "rf8_L2"])
def test_deeper_trees(ctx, chain):
    compare(ctx, chain, chain.n_sites)


def test_full_retention_gives_zero_b(ctx):
    """k = the full leaf dimension: P = I on the merged block, b = 0, Q = 0."""
    E, diag = compare(ctx, I.tfim(8, 1.0, 0.9, 4, 16, 4), 8)
    d = diag[0]
    assert d["b"] == 0.0 and d["bH"] == 0.0 and np.isinf(d["gamma"]) and d["r"] == 0.0


@pytest.mark.parametrize("k", [4, 8, 16])
def test_twenty_site_validation(ctx, k):
    """Appendix B figure, L = 20 (5-site leaves, 10-site halves): E0 of every
    merged block equals the free-fermion ground energy of its open chain, and
    the bound chain holds with gamma > 0 for every merge."""
    c = I.tfim(20, 1.0, 0.7, 5, k, 4)
    E, diag = ctx.solve_chain_bounds(c, full_space_sites=20)
    assert [(d["lo"], d["mid"], d["hi"]) for d in diag] == [(0, 5, 10), (10, 15, 20), (0, 10, 20)]
    for d in diag:
        L = d["hi"] - d["lo"]
        ref = CF.tfim_ground_energy(L, 1.0, 0.7)
        assert abs(d["E0"] - ref) <= 1e-10 * abs(ref), (d, ref)
        check_bound_chain(d, 1e-9)
    assert diag[-1]["a"] == pytest.approx(E[0], abs=1e-12)


def test_merge_bound_on_blocks(ctx):
    """rmc_merge_bound on two Heisenberg leaves equals the dense definition."""
    Js = [0.8, 1.3, 0.9, 1.1, 0.7, 1.2, 1.0]
    c = I.xxz(8, Js, 1.0, 4, 6, 4)
    def leaf(lo):
        bonds = [(i - lo, j - lo, pi, pj, v) for i, j, pi, pj, v in c.bonds if lo <= i and j < lo + 4]
        carry = [(3, p) for p in "XYZ"] if lo == 0 else [(0, p) for p in "XYZ"]
        return ctx.build_leaf_pauli(4, 6, [], bonds, carry)
    A, B = leaf(0), leaf(4)
    coefs = {p: v for i, j, p, _, v in c.bonds if (i, j) == (3, 4)}
    # Y Y = -(iY)(iY); both leaves carry X, Y, Z in that order
    terms = [(coefs["X"], 0, 0), (-coefs["Y"], 1, 1), (coefs["Z"], 2, 2)]
    b = ctx.merge_bound(A, B, terms)
    OA, OB = O.leaf_block(c, 0, 4, 6), O.leaf_block(c, 4, 8, 6)
    ref = EB.merge_bound(c, OA, OB)["b"]
    assert abs(b - ref) <= TOL[ctx.precision]["b"] * max(1.0, ref), (b, ref)
    # a product across two sites of one module is not carried: rejected
    with pytest.raises(P.RmcError):
        C = ctx.build_leaf_pauli(4, 6, [], [], [(2, "Z"), (3, "Z")])
        ctx.merge_bound(C, B, [(1.0, 0, 2), (1.0, 1, 2)])
