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
