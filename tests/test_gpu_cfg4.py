"""Parity at the size of the 128-site random-field Heisenberg workload.

* The whole 128-site chain (h_i ~ U[-2,2], leaves of 4 sites) at k = 128:
  fifteen merges of dimension 16384, every one of them checked densely by the
  oracle (Algorithm 1 with the dense H_eff of Eq. (7); stored energies in
  tests/golden/rfheis_n128_k128.json, written by make_golden.py).
* One merge of two 256-state blocks (dimension 65536, three boundary
  operators): the shape of every merge above the first level at k = 256.  The
  inputs are the oracle's own 12-site leaves (dense 4096 x 4096 eigensolves,
  imported into the GPU), and the expected values are the lowest 257
  eigenvalues of the dense 65536 x 65536 H_eff (LAPACK dsyevr on the host,
  stored in tests/golden/rfheis_pair_n65536.json).
"""
import json
import os

import numpy as np
import pytest

import instances as I
from oracle import rmc_oracle as O
from tests.gpu_util import torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
RTOL = {"fp64": 1e-10, "mixed": 1e-8}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rfheis_n128_k128_matches_oracle(precision):
    torch_cuda()
    g = json.load(open(os.path.join(GOLD, "rfheis_n128_k128.json")))
    chain = I.rf_heisenberg_n128(k=128)
    assert I.Chain.from_json(g["chain"]) == chain
    ref = np.array(g["energies"])
    with P.Context(precision=precision) as ctx:
        E = ctx.solve_chain(chain)
    tol = RTOL[precision] * np.maximum(1.0, np.abs(ref))
    assert np.all(np.abs(E - ref) <= tol), (E - ref) / np.maximum(1.0, np.abs(ref))


@pytest.fixture(scope="module")
def pair_inputs():
    g = json.load(open(os.path.join(GOLD, "rfheis_pair_n65536.json")))
    chain = I.rf_heisenberg_pair()
    assert I.Chain.from_json(g["chain"]) == chain
    A = O.leaf_block(chain, 0, 12, chain.k)
    B = O.leaf_block(chain, 12, 24, chain.k)
    assert [len(A.E), len(B.E)] == g["leaf_k"]
    return chain, A, B, g


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_merge_of_two_256_state_blocks_matches_dense_eigensolve(precision, pair_inputs):
    torch_cuda()
    chain, A, B, g = pair_inputs
    ref = np.array(g["theta"])
    with P.Context(precision=precision) as ctx:
        keysA, keysB = sorted(A.ops), sorted(B.ops)
        hA = ctx.block_import(A.E, [A.ops[k] for k in keysA], keysA)
        hB = ctx.block_import(B.E, [B.ops[k] for k in keysB], keysB)
        terms = [(c, keysA.index(ka), keysB.index(kb)) for c, ka, kb in O.merge_terms(chain, 0, 12, 12, 24)]
        assert len(terms) == 3
        blk = ctx.couple(hA, hB, terms, chain.k, [])
        E, _, basis = blk.export()
        assert len(E) == g["k_eff"]
        tol = RTOL[precision] * np.maximum(1.0, np.abs(ref[: len(E)]))
        err = np.abs(E - ref[: len(E)])
        assert np.all(err <= tol), (err / np.maximum(1.0, np.abs(ref[: len(E)]))).max()
        # the retained basis is orthonormal (65536-long vectors)
        np.testing.assert_allclose(basis @ basis.T, np.eye(len(E)), atol=1e-11)
        for h in (blk, hA, hB):
            h.free()
