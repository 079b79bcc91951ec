"""Per-step parity of the GPU path against the oracle on identical inputs.

* Leaf build (Algorithm 1, first step) from Pauli terms.
* One merge (Algorithm 1, inner loop) on blocks imported from the oracle:
  retained energies, the cut, the retained subspace (gauge-invariant overlap)
  and the rotated operators.
* Edge cases: no coupling term (J' = 0, Eq. (7) without V), ragged k_A != k_B,
  the dense case k_A k_B <= block size, a top merge, invalid inputs, the
  memory budget and the iteration cap.
"""
import numpy as np
import pytest

import instances as I
from oracle import rmc_oracle as O
from tests.gpu_util import overlap_singular_values, torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-10, 1e-9), "mixed": (1e-8, 1e-7), "mixed_tf32": (1e-8, 1e-7)}


@pytest.fixture(scope="module", params=["fp64", "mixed", "mixed_tf32"])
def ctx(request):
    torch_cuda()
    c = P.Context(precision=request.param)
    yield c
    c.close()


def _import(ctx, blk):
    keys = sorted(blk.ops)
    h = ctx.block_import(blk.E, [blk.ops[k] for k in keys], keys)
    return h, keys


def _leaf_terms(chain, lo, hi):
    ons = [(s - lo, p, c) for s, p, c in chain.onsite if lo <= s < hi]
    bnd = [(i - lo, j - lo, a, b, c) for i, j, a, b, c in chain.bonds if lo <= i and j < hi]
    return ons, bnd


@pytest.mark.parametrize("chain,lo,hi", [
    (I.tfim(8, 1.0, 0.8, 2, 8, 4), 0, 2),
    (I.tfim(16, 1.0, 0.7, 4, 16, 4), 4, 8),
    (I.xxz(8, [0.7, 1.1, 0.9, 1.4, 0.6, 1.2, 1.0], 1.0, 4, 16, 8), 4, 8),
    (I.xxz(8, [1.0] * 7, 1.0, 4, 16, 8, fields=[0.5, -1.2, 1.9, 0.1, -0.7, 1.1, -1.8, 0.3]), 0, 4),
    (I.xxz(12, [0.9] * 11, 0.5, 6, 40, 8), 0, 6),
])
def test_leaf_matches_oracle(ctx, chain, lo, hi):
    ref = O.leaf_block(chain, lo, hi, chain.k)
    carry = [(s - lo, p) for s, p in O.boundary_ops(chain, lo, hi)]
    ons, bnd = _leaf_terms(chain, lo, hi)
    blk = ctx.build_leaf_pauli(hi - lo, chain.k, ons, bnd, carry)
    E, ops, basis = blk.export()
    assert len(E) == len(ref.E)
    np.testing.assert_allclose(E, ref.E, atol=1e-12 * max(1, np.abs(ref.E).max()))
    sv = overlap_singular_values(ref.U, basis.T)
    assert sv.min() >= 1 - 1e-12
    G = ref.U.T @ basis.T                      # maps the oracle basis onto the GPU one
    for j, (s, p) in enumerate(carry):
        o_ref = ref.ops[(s + lo, p)]
        np.testing.assert_allclose(ops[j], G.T @ o_ref @ G, atol=1e-11)
    blk.free()


def rotated_op_tolerance(C_ref, C_gpu, o_norm=1.0):
    """Bound on |C_g^T O C_g - G^T (C_or^T O C_or) G| for G = C_or^T C_g.

    Write C_g = C_or G + E with E = (I - C_or C_or^T) C_g, so |E|_2 = sin(phi),
    phi the largest principal angle between the two retained subspaces.
    Expanding gives G^T C_or^T O E + E^T O C_or G + E^T O E, of norm at most
    |O| (2 sin(phi) + sin(phi)^2) since |G| <= 1; |O| = |o (x) I| = |o| <= 1
    for a projected Pauli operator.  sin(phi) is measured directly as |E|_2
    (not from 1 - sigma_min, which FP64 cannot resolve below ~1e-8), and the
    tolerance adds the FP64 rounding of the k x k products."""
    G = C_ref.T @ C_gpu
    sin_phi = np.linalg.norm(C_gpu - C_ref @ G, 2)
    return o_norm * (2 * sin_phi + sin_phi ** 2) + 1e-13 * C_gpu.shape[1]


def _merge_case(chain, A_rng, B_rng, k, top):
    A = O.leaf_block(chain, *A_rng, chain.k) if A_rng[1] - A_rng[0] <= chain.leaf_sites else None
    B = O.leaf_block(chain, *B_rng, chain.k) if B_rng[1] - B_rng[0] <= chain.leaf_sites else None
    return A, B


MERGES = [
    # chain, A range, B range, keep, top
    (I.tfim(8, 1.0, 0.8, 2, 8, 4), (0, 2), (2, 4), 8, False),                  # dense: n = 16
    (I.tfim(10, 1.0, 0.7, 5, 7, 4), (0, 5), (5, 10), 4, True),                 # the paper's 5 + 5 chain, k = 7
    (I.xxz(8, [0.7, 1.1, 0.9, 1.4, 0.6, 1.2, 1.0], 1.0, 4, 16, 8), (0, 4), (4, 8), 24, False),
    (I.xxz(16, list(np.random.default_rng(4).uniform(0.5, 1.5, 15)), 1.0, 8, 40, 8), (0, 8), (8, 16), 64, False),
    (I.xxz(16, [1.0] * 15, 1.0, 8, 36, 8, fields=list(np.random.default_rng(9).uniform(-2, 2, 16))),
     (0, 8), (8, 16), 48, False),
    (I.tfim(12, 1.0, 1.1, 6, 50, 6), (0, 6), (6, 12), 6, True),
]


@pytest.mark.parametrize("case", range(len(MERGES)))
def test_merge_matches_oracle(ctx, case):
    chain, Ar, Br, keep, top = MERGES[case]
    A = O.leaf_block(chain, *Ar, chain.k)
    B = O.leaf_block(chain, *Br, chain.k)
    ref, rec = O.merge_blocks(chain, A, B, keep, top)
    hA, kA_keys = _import(ctx, A)
    hB, kB_keys = _import(ctx, B)
    terms = [(c, kA_keys.index(ka), kB_keys.index(kb)) for c, ka, kb in O.merge_terms(chain, *Ar, *Br)]
    keys = O.boundary_ops(chain, Ar[0], Br[1]) if not top else []
    carry = [(0, kA_keys.index(k)) if k[0] < Ar[1] else (1, kB_keys.index(k)) for k in keys]
    blk = ctx.couple(hA, hB, terms, keep, carry, top=top)
    E, ops, basis = blk.export()
    etol, stol = TOL[ctx.precision]
    assert len(E) == len(ref.E)
    np.testing.assert_allclose(E, ref.E, atol=etol * max(1, np.abs(ref.E).max()))
    sv = overlap_singular_values(ref.U, basis.T)
    assert sv.min() >= 1 - stol, sv.min()
    G = ref.U.T @ basis.T
    for j, key in enumerate(keys):
        np.testing.assert_allclose(ops[j], G.T @ ref.ops[key] @ G, atol=rotated_op_tolerance(ref.U, basis.T))
    # the retained basis is orthonormal and diagonalises the projected H_eff
    np.testing.assert_allclose(basis @ basis.T, np.eye(len(E)), atol=1e-12)
    H = O.effective_hamiltonian(A.E, B.E, [(c, A.ops[ka], B.ops[kb]) for c, ka, kb in
                                           O.merge_terms(chain, *Ar, *Br)])
    np.testing.assert_allclose(basis @ H @ basis.T, np.diag(E), atol=1e-10 * max(1, np.abs(E).max()))
    for h in (blk, hA, hB):
        h.free()


LARGE_MERGES = [
    # kept counts wider than one Rayleigh-Ritz block: solved chunk by chunk with locking
    (I.xxz(16, list(np.random.default_rng(21).uniform(0.5, 1.5, 15)), 1.0, 8, 50, 8), (0, 8), (8, 16), 220),
    (I.xxz(16, [1.0] * 15, 1.0, 8, 48, 8, fields=list(np.random.default_rng(22).uniform(-2, 2, 16))),
     (0, 8), (8, 16), 300),
    # 256 kept from 64 x 64: two full chunks and a one-vector tail chunk right
    # above 256 locked vectors (the filter must not amplify the locked span)
    (I.xxz(16, list(np.random.default_rng(23).uniform(0.5, 1.5, 15)), 1.0, 8, 64, 8), (0, 8), (8, 16), 256),
]


@pytest.mark.parametrize("case", range(len(LARGE_MERGES)))
def test_wide_merge_with_locking_matches_oracle(ctx, case):
    chain, Ar, Br, keep = LARGE_MERGES[case]
    A = O.leaf_block(chain, *Ar, chain.k)
    B = O.leaf_block(chain, *Br, chain.k)
    ref, rec = O.merge_blocks(chain, A, B, keep, False)
    hA, kA_keys = _import(ctx, A)
    hB, kB_keys = _import(ctx, B)
    terms = [(c, kA_keys.index(ka), kB_keys.index(kb)) for c, ka, kb in O.merge_terms(chain, *Ar, *Br)]
    keys = O.boundary_ops(chain, Ar[0], Br[1])
    carry = [(0, kA_keys.index(k)) if k[0] < Ar[1] else (1, kB_keys.index(k)) for k in keys]
    blk = ctx.couple(hA, hB, terms, keep, carry)
    E, ops, basis = blk.export()
    etol, stol = TOL[ctx.precision]
    assert len(E) == len(ref.E)
    np.testing.assert_allclose(E, ref.E, atol=etol * max(1, np.abs(ref.E).max()))
    sv = overlap_singular_values(ref.U, basis.T)
    assert sv.min() >= 1 - stol, sv.min()
    G = ref.U.T @ basis.T
    for j, key in enumerate(keys):
        np.testing.assert_allclose(ops[j], G.T @ ref.ops[key] @ G, atol=rotated_op_tolerance(ref.U, basis.T))
    np.testing.assert_allclose(basis @ basis.T, np.eye(len(E)), atol=1e-12)
    for h in (blk, hA, hB):
        h.free()


def test_zero_coupling_is_sorted_sums(ctx):
    c = I.tfim(8, 1.0, 0.8, 4, 16, 20)
    A = O.leaf_block(c, 0, 4, 16)
    B = O.leaf_block(c, 4, 8, 16)
    hA, _ = _import(ctx, A)
    hB, _ = _import(ctx, B)
    blk = ctx.couple(hA, hB, [], 20, [], top=True)
    E = ctx.lowest(blk, 20)
    sums = np.sort(np.add.outer(A.E, B.E).reshape(-1))[:20]
    np.testing.assert_allclose(E, sums, atol=1e-10 * max(1, np.abs(sums).max()))


def test_homogeneous_reuse_same_block_twice(ctx):
    """A and B may be the same block (identical modules, the paper's reuse):
    an interior leaf of a uniform chain carries Z on its first and last site,
    and the merge couples A's last-site Z to B's first-site Z."""
    c = I.tfim(8, 1.0, 0.9, 4, 16, 4)
    ref = O.solve(c).energies
    U = O.leaf_block(c, 0, 4, 16).U
    Z = O.pauli_matrix("Z")
    z0 = U.T @ O.site_operator(Z, 0, 0, 4) @ U
    z3 = U.T @ O.site_operator(Z, 3, 0, 4) @ U
    E = O.leaf_block(c, 0, 4, 16).E
    h = ctx.block_import(E, [z0, z3], [(0, "Z"), (3, "Z")])
    blk = ctx.couple(h, h, [(-1.0, 1, 0)], 4, [], top=True)
    tol = TOL[ctx.precision][0] * np.abs(ref).max()
    np.testing.assert_allclose(ctx.lowest(blk, 4), ref, atol=tol)


def test_invalid_inputs_are_rejected(ctx):
    H = np.array([[0.0, 1.0], [0.5, 0.0]])
    with pytest.raises(P.RmcError) as e:
        ctx.build_leaf(H, 2)
    assert e.value.status == P.RMC_ERR_INVAL
    with pytest.raises(P.RmcError) as e:
        ctx.build_leaf(np.array([[np.nan]]), 1)
    assert e.value.status == P.RMC_ERR_INVAL
    with pytest.raises(P.RmcError) as e:
        ctx.block_import([1.0, 0.0])                       # not ascending
    assert e.value.status == P.RMC_ERR_INVAL
    A = ctx.block_import([0.0, 1.0], [np.eye(2)], [(0, "Z")])
    with pytest.raises(P.RmcError) as e:
        ctx.couple(A, A, [(1.0, 0, 5)], 2)                 # missing operator
    assert e.value.status == P.RMC_ERR_INVAL
    A.free()


def test_memory_budget_is_enforced():
    torch_cuda()
    with P.Context(precision="fp64", mem_budget=1 << 20) as c:
        chain = I.xxz(16, [1.0] * 15, 1.0, 8, 40, 8)
        A = O.leaf_block(chain, 0, 8, 40)
        B = O.leaf_block(chain, 8, 16, 40)
        hA, ka = _import(c, A)
        hB, kb = _import(c, B)
        terms = [(cc, ka.index(x), kb.index(y)) for cc, x, y in O.merge_terms(chain, 0, 8, 8, 16)]
        with pytest.raises(P.RmcError) as e:
            c.couple(hA, hB, terms, 40)
        assert e.value.status == P.RMC_ERR_NOMEM
        assert c.mem_in_use() < (1 << 20)


def test_iteration_cap_reports_noconv():
    torch_cuda()
    with P.Context(precision="fp64", max_iter=1) as c:
        chain = I.xxz(16, [1.0] * 15, 1.0, 8, 40, 8)
        A = O.leaf_block(chain, 0, 8, 40)
        B = O.leaf_block(chain, 8, 16, 40)
        hA, ka = _import(c, A)
        hB, kb = _import(c, B)
        terms = [(cc, ka.index(x), kb.index(y)) for cc, x, y in O.merge_terms(chain, 0, 8, 8, 16)]
        with pytest.raises(P.RmcError) as e:
            c.couple(hA, hB, terms, 40)
        assert e.value.status == P.RMC_ERR_NOCONV
        blk = c.couple(hA, hB, terms, 40, allow_noconv=True)   # best iterate still returned
        assert blk.info()[0] >= 1


def _prepare(ctx, case):
    chain, Ar, Br, keep, top = MERGES[case]
    A = O.leaf_block(chain, *Ar, chain.k)
    B = O.leaf_block(chain, *Br, chain.k)
    ref, _ = O.merge_blocks(chain, A, B, keep, top)
    hA, kA_keys = _import(ctx, A)
    hB, kB_keys = _import(ctx, B)
    terms = [(c, kA_keys.index(ka), kB_keys.index(kb)) for c, ka, kb in O.merge_terms(chain, *Ar, *Br)]
    keys = O.boundary_ops(chain, Ar[0], Br[1]) if not top else []
    carry = [(0, kA_keys.index(k)) if k[0] < Ar[1] else (1, kB_keys.index(k)) for k in keys]
    return (hA, hB, terms, keep, carry, top), ref, keys


def test_batched_merges_match_one_at_a_time_and_the_oracle(ctx):
    """rmc_couple_batch runs the independent merges at once (one stream and
    host thread per lane, up to 8): every result equals the same merge run
    alone (the kernels are deterministic) and the oracle's."""
    cases = list(range(len(MERGES))) * 2
    prep = [_prepare(ctx, c) for c in cases]
    blocks = ctx.couple_batch([p[0] for p in prep])
    etol, stol = TOL[ctx.precision]
    for (args, ref, keys), blk in zip(prep, blocks):
        E, ops, basis = blk.export()
        alone = ctx.couple(*args[:5], top=args[5])
        E1, ops1, basis1 = alone.export()
        np.testing.assert_array_equal(E, E1)
        np.testing.assert_array_equal(basis, basis1)
        np.testing.assert_allclose(E, ref.E, atol=etol * max(1, np.abs(ref.E).max()))
        assert overlap_singular_values(ref.U, basis.T).min() >= 1 - stol
        for h in (blk, alone, args[0], args[1]):
            h.free()


def test_batch_reports_a_failing_merge_and_keeps_the_others(ctx):
    prep = [_prepare(ctx, c) for c in (0, 2, 3)]
    merges = [p[0] for p in prep]
    bad = list(merges[1])
    bad[2] = [(1.0, 99, 0)]                          # a term naming a missing operator
    merges[1] = tuple(bad)
    with pytest.raises(P.RmcError) as e:
        ctx.couple_batch(merges)
    assert e.value.status == P.RMC_ERR_INVAL
    assert "missing operator" in ctx.last_error()


def test_batch_lanes_share_the_budget():
    """Lanes draw on their context's budget: a budget that holds the inputs
    but not the merges' workspaces fails with NOMEM, and every byte the lanes
    drew is returned to the context."""
    torch_cuda()
    with P.Context(precision="mixed", mem_budget=4 << 20) as c:
        prep = [_prepare(c, 3) for _ in range(4)]
        base = c.mem_in_use()
        with pytest.raises(P.RmcError) as e:
            c.couple_batch([p[0] for p in prep])
        assert e.value.status == P.RMC_ERR_NOMEM
        assert c.mem_in_use() == base
