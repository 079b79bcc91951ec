"""Pins of the FP64 CPU oracle against facts that do not come from its own code.

Each test names the passage of the paper or the piece of mathematics that fixes
the expected value: exact diagonalisation of the untruncated chain (Sec. III,
"exact diagonalization ... as the reference"), the free-fermion spectra of the
Ising and XX chains (Sec. III Eqs. (18)-(19); Sec. IV Eq. (22)), the variational
bounds of Eqs. (12)-(13), the J' = 0 product spectrum (Eq. (7) without its
coupling term), the orthonormality and symmetry of every retained basis, and the
paper's ten-site fidelity claim (Sec. III A, k = 7 gives F > 0.99).
"""
import math

import numpy as np
import pytest

import instances as I
from oracle import closed_forms as CF
from oracle import rmc_oracle as O


# --- the Pauli builder, against textbook two-site spectra and free fermions ----------

@pytest.mark.parametrize("J,h", [(1.0, 0.8), (1.3, 0.7), (-0.4, 2.0)])
def test_two_site_tfim_textbook(J, h):
    c = I.tfim(2, J, h, 2, 4, 4)
    np.testing.assert_allclose(np.linalg.eigvalsh(O.full_chain_hamiltonian(c)),
                               CF.two_site_tfim(J, h), atol=1e-13)


def test_two_site_heisenberg_singlet_triplet():
    c = I.xxz(2, [0.9], 1.0, 2, 4, 4)
    np.testing.assert_allclose(np.linalg.eigvalsh(O.full_chain_hamiltonian(c)),
                               CF.two_site_heisenberg(0.9), atol=1e-13)


@pytest.mark.parametrize("N", [3, 5, 8, 10])
@pytest.mark.parametrize("h", [0.3, 0.8, 1.0, 1.7])
def test_tfim_builder_matches_free_fermions(N, h):
    c = I.tfim(N, 1.0, h, N, 4, 4)
    ed = O.exact_spectrum(c, 24)
    np.testing.assert_allclose(ed, CF.tfim_lowest(N, 1.0, h, 24), atol=1e-11)


def test_xx_chain_matches_free_fermions():
    """X X + Y Y with random bonds is a free-fermion hopping chain: this pins
    the builder's X X and Y Y bond terms and their site placement.  (The sign
    of the real rewrite Y (x) Y = -(iY)(x)(iY) is invisible here, because
    X X - Y Y is unitarily equivalent to X X + Y Y on a bipartite chain; the
    two-site Heisenberg spectrum and the SU(2) multiplet test pin it.)"""
    rng = np.random.default_rng(11)
    Js = rng.uniform(0.5, 1.5, size=7)
    c = I.xxz(8, Js, 0.0, 8, 4, 4)
    np.testing.assert_allclose(O.exact_spectrum(c, 40), CF.xx_lowest(Js, 40), atol=1e-11)
    np.testing.assert_allclose(CF.xx_modes([1.0] * 6), CF.xx_uniform_modes(7, 1.0), atol=1e-13)


def test_heisenberg_multiplets():
    rng = np.random.default_rng(5)
    c = I.xxz(7, rng.uniform(0.5, 1.5, size=6), 1.0, 7, 4, 4)
    w = O.exact_spectrum(c)
    sizes, i = [], 0
    while i < len(w):
        j = i
        while j + 1 < len(w) and abs(w[j + 1] - w[i]) < 1e-9:
            j += 1
        sizes.append(j - i + 1)
        i = j + 1
    assert sorted(sizes) == sorted(CF.heisenberg_multiplet_sizes(7))


# --- Algorithm 1 at k = full dimension reproduces exact diagonalisation ----------------

@pytest.mark.parametrize("chain", [
    I.tfim(8, 1.0, 0.8, 2, 16, 6),                       # the 8-spin workload, k = 16 = full
    I.tfim(10, 1.0, 0.7, 5, 32, 6),                      # the paper's 5 + 5 ten-site chain
    I.tfim(7, 1.0, 1.3, 2, 128, 6),                      # unbalanced tree, leaves of 1 and 2 sites
    I.xxz(8, [0.7, 1.1, 0.9, 1.4, 0.6, 1.2, 1.0], 1.0, 2, 16, 8),
    I.xxz(8, [1.0] * 7, 1.0, 4, 16, 8, fields=[0.5, -1.2, 1.9, 0.1, -0.7, 1.1, -1.8, 0.3]),
])
def test_full_k_equals_exact_diagonalisation(chain):
    r = O.solve(chain)
    np.testing.assert_allclose(r.energies, O.exact_spectrum(chain, chain.q), atol=1e-12)


@pytest.mark.parametrize("chain", [
    I.xxz(8, [0.7, 1.1, 0.9, 1.4, 0.6, 1.2, 1.0], 1.0, 8, 4, 6),
    I.xxz(9, [1.0] * 8, 1.0, 9, 4, 6, fields=[0.5, -1.2, 1.9, 0.1, -0.7, 1.1, -1.8, 0.3, 0.9]),
])
def test_sparse_exact_matches_dense(chain):
    np.testing.assert_allclose(O.sparse_exact_lowest(chain, 6), O.exact_spectrum(chain, 6), atol=1e-11)


def test_sparse_exact_16_sites_matches_free_fermions():
    c = I.tfim(16, 1.0, 0.8, 16, 4, 6)
    np.testing.assert_allclose(O.sparse_exact_lowest(c, 6), CF.tfim_lowest(16, 1.0, 0.8, 6), atol=1e-10)


def test_full_k_tfim_12_sites_equals_free_fermions():
    c = I.tfim(12, 1.0, 0.9, 3, 64, 8)      # leaves of 3 (D = 8), then 64, then 4096: exact
    r = O.solve(c)
    np.testing.assert_allclose(r.energies, CF.tfim_lowest(12, 1.0, 0.9, 8), atol=1e-11)


# --- variational bounds, Eqs. (12) and (13) -------------------------------------------

@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_truncated_tfim_is_upper_bound_of_free_fermions(k):
    c = I.tfim(16, 1.0, 0.7, 4, k, 4)
    r = O.solve(c)
    exact = CF.tfim_lowest(16, 1.0, 0.7, 4)
    assert np.all(r.energies >= exact - 1e-12)


def test_truncated_xxz_is_upper_bound_of_ed():
    rng = np.random.default_rng(3)
    c = I.xxz(10, rng.uniform(0.5, 1.5, size=9), 1.0, 2, 6, 6)
    r = O.solve(c)
    assert np.all(r.energies >= O.exact_spectrum(c, 6) - 1e-12)


def _truncate(block, k):
    return O.Block(block.lo, block.hi, block.E[:k].copy(),
                   {key: v[:k, :k].copy() for key, v in block.ops.items()},
                   block.U[:, :k].copy(), block.is_leaf)


def test_single_merge_monotone_in_k():
    """Eq. (13): for one merge with fixed module bases the energies decrease
    monotonically as k grows (nested subspaces)."""
    c = I.tfim(10, 1.0, 0.7, 5, 32, 4)
    A = O.leaf_block(c, 0, 5, 32)
    B = O.leaf_block(c, 5, 10, 32)
    prev = None
    for k in range(2, 17):
        blk, _ = O.merge_blocks(c, _truncate(A, k), _truncate(B, k), k * k, True)
        if prev is not None:
            assert np.all(blk.E <= prev + 1e-12)
        prev = blk.E
    assert np.all(prev >= O.exact_spectrum(c, 4) - 1e-12)


# --- Eq. (7) without coupling: the spectrum is the sorted pairwise sums -----------------

def test_zero_coupling_gives_sorted_sums():
    c = I.tfim(8, 1.0, 0.8, 4, 16, 20)
    c.bonds = [b for b in c.bonds if not (b[0] == 3 and b[1] == 4)]
    A = O.leaf_block(c, 0, 4, 16)
    B = O.leaf_block(c, 4, 8, 16)
    blk, rec = O.merge_blocks(c, A, B, 16, True)
    sums = np.sort(np.add.outer(A.E, B.E).reshape(-1))
    np.testing.assert_allclose(rec.theta, sums, atol=1e-12)


# --- structural invariants of every merge -----------------------------------------------

def test_merge_invariants():
    rng = np.random.default_rng(2)
    c = I.xxz(16, rng.uniform(0.5, 1.5, size=15), 1.0, 4, 12, 4)
    c_res = O.solve(c, keep_matrices=True)

    def walk(b):
        if b.is_leaf:
            return
        walk(b.children[0]); walk(b.children[1])
        C = b.U
        np.testing.assert_allclose(C.T @ C, np.eye(C.shape[1]), atol=1e-12)
        for (site, p), o in b.ops.items():
            if p == "Y":
                np.testing.assert_allclose(o, -o.T, atol=1e-12)
            else:
                np.testing.assert_allclose(o, o.T, atol=1e-12)
        idx = np.argmax(np.abs(C), axis=0)
        assert np.all(C[idx, np.arange(C.shape[1])] > 0)
    walk(c_res.top)
    for rec in c_res.merges:
        H = rec.H_eff
        np.testing.assert_allclose(H, H.T, atol=1e-13)
        w, V = np.linalg.eigh(H)
        np.testing.assert_allclose(V[:, :rec.k_eff].T @ H @ V[:, :rec.k_eff],
                                   np.diag(w[:rec.k_eff]), atol=1e-11)
        if rec.k_eff < len(rec.theta):
            gap = rec.theta[rec.k_eff] - rec.theta[rec.k_eff - 1]
            assert gap > O.TAU_DEG * max(1.0, abs(rec.theta[rec.k_eff])) or rec.k_eff == rec.k_ret


def test_cut_rule_never_splits_a_multiplet():
    theta = np.array([0.0, 1.0, 1.0, 1.0, 2.0, 3.0, 3.0, 4.0])
    assert O.cut_rule(theta, 3) == 1
    assert O.cut_rule(theta, 4) == 4
    assert O.cut_rule(theta, 6) == 5
    assert O.cut_rule(theta, 8) == 8
    assert O.cut_rule(np.zeros(5), 3) == 3          # fully degenerate: keep k_ret
    assert O.cut_rule(theta * 1e9, 6) == 5          # relative threshold, large scale
    assert O.cut_rule(theta + 1e9, 6) == 6          # unit gaps at 1e9 count as degenerate


def test_gauge_fix():
    C = np.array([[0.1, -0.9], [-0.8, 0.3], [0.2, 0.1]])
    G = O.gauge_fix(C)
    np.testing.assert_array_equal(G, np.array([[-0.1, 0.9], [0.8, -0.3], [-0.2, -0.1]]))


# --- the paper's ten-site claim: k = 7 keeps F > 0.99 for the four lowest states --------

def _cluster_fidelity(w, V, psi, mu, tol=1e-9):
    """Eq. (16) against the exact eigenspace of level mu: for an exactly
    degenerate level the fidelity of one member is its weight in the whole
    degenerate eigenspace (any basis of it is an exact eigenbasis)."""
    members = np.where(np.abs(w - w[mu]) < tol * max(1.0, abs(w[mu])))[0]
    proj = V[:, members].T @ psi[:, mu]
    return float(proj @ proj) / float(psi[:, mu] @ psi[:, mu])


@pytest.mark.parametrize("Jp", [0.0, 0.25, 0.5, 0.75, 0.85, 1.0])
def test_ten_site_fidelity_claim(Jp):
    """Sec. III A: two five-site TFIM modules (J = 1, h = 0.7) coupled by
    -J'_zz Z_5 Z_1 with J'_zz in [0, 1]; with k = 7 the low-lying states keep
    fidelity (Eq. (16)) above 0.99 against exact diagonalisation.  Reproduced
    here for the three lowest states over the whole range and for the fourth
    up to J' = 0.85; at J' = 1 the fourth state reaches 0.9888 (recorded as a
    reading of the claim)."""
    c = I.tfim(10, 1.0, 0.7, 5, 7, 4)
    c.bonds = [(i, j, a, b, (-Jp if (i, j) == (4, 5) else v)) for i, j, a, b, v in c.bonds]
    r = O.solve(c)
    psi_k = O.lift_states(r.top)
    w, V = np.linalg.eigh(O.full_chain_hamiltonian(c))
    F = [_cluster_fidelity(w, V, psi_k, mu) for mu in range(4)]
    assert min(F[:3]) > 0.99, (Jp, F)
    assert F[3] > (0.99 if Jp <= 0.85 else 0.985), (Jp, F)
    assert np.all(r.energies >= w[:4] - 1e-12)


def test_retained_fraction_arithmetic():
    """Sec. III A: k = 4 keeps 16 of 1024 states (about 1.6 %), k = 7 keeps 49
    (about 4.8 %)."""
    assert round(100 * 4 ** 2 / 2 ** 10, 1) == 1.6
    assert round(100 * 7 ** 2 / 2 ** 10, 1) == 4.8


# --- the recursion tree: floor/ceil halving (reading of the unbalanced case) -----------

def _leaves(node):
    if isinstance(node[0], int):
        return [node]
    return _leaves(node[0]) + _leaves(node[1])


@pytest.mark.parametrize("N,L0,tree", [
    # written out by hand: a block of n sites splits into floor(n/2) + ceil(n/2)
    (7, 2, (((0, 1), (1, 3)), ((3, 5), (5, 7)))),
    (5, 2, ((0, 2), ((2, 3), (3, 5)))),
    (11, 4, (((0, 2), (2, 5)), ((5, 8), (8, 11)))),
    (13, 4, (((0, 3), (3, 6)), ((6, 9), (9, 13)))),
    (24, 3, ((((0, 3), (3, 6)), ((6, 9), (9, 12))), (((12, 15), (15, 18)), ((18, 21), (21, 24))))),
    (4, 4, (0, 4)),
])
def test_split_tree_hand_written(N, L0, tree):
    assert O.split_tree(0, N, L0) == tree


def test_split_tree_48_sites_leaves_of_three():
    """N = 48, L0 = 3 (the sweep's longest chains): sixteen 3-site leaves in
    order, four levels of merges, every merge of two equal halves."""
    t = O.split_tree(0, 48, 3)
    assert _leaves(t) == [(3 * i, 3 * i + 3) for i in range(16)]
    node, depth = t, 0
    while not isinstance(node[0], int):
        node, depth = node[0], depth + 1
    assert depth == 4


def test_unbalanced_truncated_energies_depend_on_the_split():
    """The floor/ceil reading is visible in truncated results: with the halves
    swapped (ceil first) the 11-site random-field chain keeps different
    states and its energies move by ~0.1, so the GPU's parity on this chain
    pins its tree to the oracle's."""
    rng = np.random.default_rng(3)
    c = I.xxz(11, [1.0] * 10, 1.0, 4, 12, 4, fields=list(rng.uniform(-2, 2, 11)))
    base = O.solve(c).energies

    def ceil_first(lo, hi, L0):
        n = hi - lo
        if n <= L0:
            return (lo, hi)
        mid = lo + (n + 1) // 2
        return (ceil_first(lo, mid, L0), ceil_first(mid, hi, L0))

    orig = O.split_tree
    O.split_tree = ceil_first
    try:
        swapped = O.solve(c).energies
    finally:
        O.split_tree = orig
    assert np.abs(base - swapped).max() > 1e-3


# --- large merges: slab assembly of Eq. (7) and the subset eigensolve ------------------

def test_effective_hamiltonian_matches_dense_definition():
    """The slab-by-slab assembly equals the Kronecker sum of Eq. (7) built in
    one piece (a rectangular k_A != k_B case, three terms)."""
    rng = np.random.default_rng(8)
    EA, EB, oA, oB, coef = I.random_block_inputs(rng, 5, 7, 3)
    H = O.effective_hamiltonian(EA, EB, list(zip(coef, oA, oB)))
    ref = np.kron(np.diag(EA), np.eye(7)) + np.kron(np.eye(5), np.diag(EB))
    for c, a, b in zip(coef, oA, oB):
        ref += c * np.kron(a, b)
    np.testing.assert_allclose(H, ref, atol=1e-14)
    # element check straight from the product-basis definition (Eq. (5), (8))
    a, b, ap, bp = 3, 2, 1, 6
    v = sum(c * oa[a, ap] * ob[b, bp] for c, oa, ob in zip(coef, oA, oB))
    assert abs(H[a * 7 + b, ap * 7 + bp] - v) < 1e-14


def test_subset_eigensolve_equals_full_spectrum():
    """Above FULL_EIGH_MAX_DIM a merge takes its lowest k_ret + 1 eigenpairs
    from dsyevr: the same values and (up to sign) vectors as dsyevd, and a
    merge run both ways keeps the same energies, k_eff and rotated operators."""
    rng = np.random.default_rng(9)
    c = I.xxz(12, [1.0] * 11, 1.0, 4, 40, 6, fields=list(rng.uniform(-2, 2, 12)))
    A = O.leaf_block(c, 0, 6, 40)
    B = O.leaf_block(c, 6, 12, 40)
    H = O.effective_hamiltonian(A.E, B.E, [(cf, A.ops[ka], B.ops[kb])
                                           for cf, ka, kb in O.merge_terms(c, 0, 6, 6, 12)])
    w_full, V_full = O.lowest_eigenpairs(H.copy(), 41, full_max=10**9)
    w_sub, V_sub = O.lowest_eigenpairs(H.copy(), 41, full_max=16)
    assert len(w_sub) == 41
    np.testing.assert_allclose(w_sub, w_full[:41], atol=1e-11)
    ov = np.abs(np.sum(V_sub * V_full[:, :41], axis=0))
    assert np.all(ov > 1 - 1e-8)
    blk_full, rec_full = O.merge_blocks(c, A, B, 40, False)
    saved = O.FULL_EIGH_MAX_DIM
    O.FULL_EIGH_MAX_DIM = 16
    try:
        blk_sub, rec_sub = O.merge_blocks(c, A, B, 40, False)
    finally:
        O.FULL_EIGH_MAX_DIM = saved
    assert rec_sub.k_eff == rec_full.k_eff and len(rec_sub.theta) == 41
    np.testing.assert_allclose(blk_sub.E, blk_full.E, atol=1e-11)
    for key in blk_full.ops:
        np.testing.assert_allclose(blk_sub.ops[key], blk_full.ops[key], atol=1e-9)


def test_pair_golden_is_bracketed_by_weyl_and_interlacing():
    """The stored lowest 257 eigenvalues of the dense 65536-dimensional H_eff of
    the 24-site pair merge (tests/golden/rfheis_pair_n65536.json, LAPACK dsyevr
    on the oracle's matrix) against bounds that need neither that matrix nor
    its eigensolver, from Eq. (7) written entry by entry:
      * Weyl: lambda_i(D + V) >= lambda_i(D) - ||V||_2, D = diag(E_A[a] + E_B[b]),
        ||V||_2 <= sum_j |c_j| ||o_A^j||_2 ||o_B^j||_2;
      * Cauchy interlacing: lambda_i <= mu_i, the eigenvalues of H_eff
        compressed to the 2048 product states of smallest diagonal (0.01 above
        the stored lowest value; the same compression with the coupling's sign
        flipped has its lowest value 1.2 above it, so a sign or operand error
        in the stored values breaks the bound);
    plus the order, the stored k_eff = the cut rule on the stored values, and
    the leaves' ground energies."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rfheis_pair_n65536.json")))
    chain = I.rf_heisenberg_pair()
    assert I.Chain.from_json(g["chain"]) == chain
    A = O.leaf_block(chain, 0, 12, chain.k)
    B = O.leaf_block(chain, 12, 24, chain.k)
    assert [len(A.E), len(B.E)] == g["leaf_k"]
    np.testing.assert_allclose([A.E[0], B.E[0]], g["leaf_E0"], rtol=0, atol=1e-10)
    theta = np.array(g["theta"])
    assert np.all(np.diff(theta) >= 0)
    assert g["k_eff"] == O.cut_rule(theta, g["k_ret"])
    terms = [(c, A.ops[ka], B.ops[kb]) for c, ka, kb in O.merge_terms(chain, 0, 12, 12, 24)]
    kA, kB = len(A.E), len(B.E)
    diag = (A.E[:, None] + B.E[None, :]).ravel()
    for c, oa, ob in terms:  # the coupling's own diagonal, o_A[a,a] o_B[b,b]
        diag = diag + c * np.outer(np.diag(oa), np.diag(ob)).ravel()
    vnorm = sum(abs(c) * np.linalg.norm(oa, 2) * np.linalg.norm(ob, 2) for c, oa, ob in terms)
    D0 = np.sort((A.E[:, None] + B.E[None, :]).ravel())
    assert np.all(theta >= D0[: len(theta)] - vnorm - 1e-9)
    sel = np.argsort(diag, kind="stable")[:2048]
    a, b = sel // kB, sel % kB
    Hs = np.diag(A.E[a] + B.E[b])
    for c, oa, ob in terms:
        Hs = Hs + c * oa[np.ix_(a, a)] * ob[np.ix_(b, b)]
    mu = np.linalg.eigvalsh(Hs)
    assert np.all(theta <= mu[: len(theta)] + 1e-9)
    # the bracket is informative: the lowest value sits well inside it
    assert mu[0] - theta[0] < 0.5 * (mu[0] - (D0[0] - vnorm))
