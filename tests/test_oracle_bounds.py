"""Pins of the single-merge error bound (Sec. IV, Appendix B) as the oracle
computes it: the two expressions of b agree, the bound chain
0 <= a - E0 <= r(b, gamma) <= b^2 / gamma holds with gamma > 0 for the
paper's ten-site validation (J = 1, h = 0.7, every k), and the special
cases -- full retention (P = I) and no coupling -- give b = 0 and a = E0."""
import numpy as np
import pytest

import instances as I
from oracle import error_bounds as EB
from oracle import rmc_oracle as O


def _two_leaves(chain, lo, mid, hi, k):
    return O.leaf_block(chain, lo, mid, k), O.leaf_block(chain, mid, hi, k)


@pytest.mark.parametrize("k", [2, 3, 4, 6, 8, 12, 16, 24])
def test_ten_site_bound_holds_for_every_k(k):
    c = I.tfim(10, 1.0, 0.7, 5, k, 4)
    A, B = _two_leaves(c, 0, 5, 10, k)
    d = EB.merge_bound(c, A, B)
    assert d["gamma"] > 0
    assert -1e-12 <= d["a"] - d["E0"] <= d["r"] + 1e-12
    assert d["r"] <= d["b"] ** 2 / d["gamma"] + 1e-12
    # the merge's projected ground energy is the lowest eigenvalue of Eq. (7)
    ref, _ = O.merge_blocks(c, A, B, k, True)
    assert abs(d["a"] - ref.E[0]) < 1e-11


@pytest.mark.parametrize("chain,mid", [
    (I.tfim(8, 1.0, 0.9, 4, 5, 4), 4),
    (I.xxz(8, [0.7, 1.1, 0.9, 1.4, 0.6, 1.2, 1.0], 1.0, 4, 6, 4), 4),
    (I.tfim_nnn(9, 1.0, 0.8, 0.3, 5, 7, 4), 4),
])
def test_two_expressions_of_b_agree(chain, mid):
    A, B = _two_leaves(chain, 0, mid, chain.n_sites, chain.k)
    d = EB.merge_bound(chain, A, B)
    assert abs(d["b"] - EB.b_from_products(chain, A, B)) < 1e-10 * max(1.0, d["b"])
    assert d["b"] > 1e-3


def test_full_retention_and_zero_coupling():
    c = I.tfim(8, 1.0, 0.9, 4, 16, 4)
    A, B = _two_leaves(c, 0, 4, 8, 16)           # every state kept: P = I
    d = EB.merge_bound(c, A, B)
    assert d["b"] == 0.0 and abs(d["a"] - d["E0"]) < 1e-11
    c0 = I.tfim(8, 1.0, 0.9, 4, 3, 4)
    c0.bonds = [(i, j, a, b_, 0.0 if (i, j) == (3, 4) else v) for i, j, a, b_, v in c0.bonds]
    A, B = _two_leaves(c0, 0, 4, 8, 3)
    d = EB.merge_bound(c0, A, B)
    assert d["b"] < 1e-12 and abs(d["a"] - d["E0"]) < 1e-11


# Products of the real single-site Paulis (Y carried as iY): p1 p2 = sign * p.
PAULI_PRODUCT = {("X", "X"): ("I", 1), ("X", "Y"): ("Z", -1), ("X", "Z"): ("Y", -1),
                 ("Y", "X"): ("Z", 1), ("Y", "Y"): ("I", -1), ("Y", "Z"): ("X", -1),
                 ("Z", "X"): ("Y", 1), ("Z", "Y"): ("X", 1), ("Z", "Z"): ("I", 1)}


def test_pauli_product_table():
    """The table the Kronecker form of b rests on, against the matrix products."""
    for (p1, p2), (p, sign) in PAULI_PRODUCT.items():
        assert np.array_equal(O.pauli_matrix(p1) @ O.pauli_matrix(p2), sign * O.pauli_matrix(p))


@pytest.mark.parametrize("chain", [
    I.xxz(8, [0.7, 1.1, 0.9, 1.4, 0.6, 1.2, 1.0], 1.0, 4, 6, 4),
    I.tfim(10, 1.0, 0.7, 5, 4, 4),
    I.xxz(8, [1.0] * 7, 1.0, 4, 5, 4, fields=[0.3, -1.2, 0.8, 1.9, -0.4, 0.1, -1.5, 0.6]),
])
def test_kronecker_form_of_b(chain):
    """Appendix B's b^2 = lambda_max(P V^2 P - (P V P)^2) assembled in the
    product basis from the carried operators alone: P V^2 P = sum_{s,t} c_s c_t
    [O_A^s O_A^t] (x) [O_B^s O_B^t], each same-site product a carried Pauli
    (up to sign) or the identity, and (P V P)^2 from the projected operators.
    Equals the dense ||P V Q||_2 of the lifted sector."""
    mid = chain.n_sites // 2
    A = O.leaf_block(chain, 0, mid, chain.k)
    B = O.leaf_block(chain, mid, chain.n_sites, chain.k)
    terms = O.merge_terms(chain, 0, mid, mid, chain.n_sites)
    kA, kB = len(A.E), len(B.E)
    M = np.zeros((kA * kB,) * 2)
    for cs, (sa, pa), (sb, pb) in terms:
        for ct, (ta, qa), (tb, qb) in terms:
            assert sa == ta and sb == tb
            ra, ga = PAULI_PRODUCT[(pa, qa)]
            rb, gb = PAULI_PRODUCT[(pb, qb)]
            mA = np.eye(kA) if ra == "I" else A.ops[(sa, ra)]
            mB = np.eye(kB) if rb == "I" else B.ops[(sb, rb)]
            M += cs * ct * ga * gb * np.kron(mA, mB)
            M -= cs * ct * np.kron(A.ops[(sa, pa)] @ A.ops[(ta, qa)], B.ops[(sb, pb)] @ B.ops[(tb, qb)])
    b = np.sqrt(max(0.0, np.linalg.eigvalsh(M)[-1]))
    ref = EB.b_from_products(chain, A, B)
    assert abs(b - ref) < 1e-10 * max(1.0, ref)
    assert abs(b - EB.merge_bound(chain, A, B)["b"]) < 1e-10 * max(1.0, ref)   # leaves: ||PHQ|| = ||PVQ||
