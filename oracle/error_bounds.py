"""Single-merge truncation-error bound (Sec. IV and Appendix B), dense, small N.

TEST INFRASTRUCTURE ONLY -- imported by ``tests/`` and never by the product.

For a merge of blocks A and B, let P project the Hilbert space of the merged
block onto the retained product sector span{|a>|b>} (the kept states of A and
B, lifted to the physical basis) and Q = I - P.  With H the merged block's own
Hamiltonian and V its inter-module coupling (Eq. (3)):

* a     = lowest eigenvalue of P H P on range(P) (the merge's projected
          ground energy, the lowest eigenvalue of Eq. (7));
* b     = || P H Q ||_2 = || P V Q ||_2 (H_A (x) I + I (x) H_B does not couple
          the two sectors; Appendix B);
* gamma = lowest eigenvalue of Q H Q on range(Q) minus a (the discarded
          sector's separation, Appendix B);
* r     = (sqrt(gamma^2 + 4 b^2) - gamma) / 2, the bound of Eq. (single-merge
          bound): 0 <= a - E0 <= r <= b^2 / gamma when gamma > 0, E0 the
          merged block's exact ground energy.

Every quantity is computed from its definition with dense matrices of the
merged block (2^(sites) square), so only blocks of up to ~12 sites are
practical.  ``b_from_products`` evaluates b the second way the paper writes
it, lambda_max(P V^2 P - (P V P)^2), as an independent check.
"""
from __future__ import annotations

import numpy as np

from oracle.rmc_oracle import (Block, _bond_real, block_hamiltonian, carried_matrix, lift_states,
                               merge_terms, site_operator)


def _retained_basis(A: Block, B: Block) -> np.ndarray:
    """Orthonormal columns spanning P: kron of the lifted kept states (slow index from A)."""
    return np.kron(lift_states(A), lift_states(B))


def coupling_operator(chain, A: Block, B: Block) -> np.ndarray:
    """V of the merge as a dense operator on the merged block's sites."""
    lo, hi = A.lo, B.hi
    V = np.zeros((2 ** (hi - lo),) * 2)
    for c, (sa, pa), (sb, pb) in merge_terms(chain, A.lo, A.hi, B.lo, B.hi):
        V += c * site_operator(carried_matrix(pa), sa, lo, hi) @ site_operator(carried_matrix(pb), sb, lo, hi)
    return V


def merge_bound(chain, A: Block, B: Block) -> dict:
    """a, b, gamma, r and the exact E0 of the merge of A and B (definitions above)."""
    H = block_hamiltonian(chain, A.lo, B.hi)
    W = _retained_basis(A, B)
    D, m = W.shape
    HW = H @ W
    a = np.linalg.eigvalsh(W.T @ HW)[0]
    # P H Q = W^T H (I - W W^T); its 2-norm
    PHQ = HW.T - (W.T @ HW) @ W.T
    b = np.linalg.norm(PHQ, 2) if m < D else 0.0
    if m < D:
        # orthonormal basis of range(Q): the left singular vectors of I - W W^T with unit singular value
        Qm = np.eye(D) - W @ W.T
        u, s, _ = np.linalg.svd(Qm)
        Qb = u[:, s > 0.5]
        gamma = np.linalg.eigvalsh(Qb.T @ H @ Qb)[0] - a
    else:
        gamma = np.inf
    E0 = np.linalg.eigvalsh(H)[0]
    r = 0.0 if b == 0 else (np.sqrt(gamma * gamma + 4 * b * b) - gamma) / 2
    return {"a": a, "b": b, "gamma": gamma, "r": r, "E0": E0}


def b_from_products(chain, A: Block, B: Block) -> float:
    """b = sqrt(lambda_max(P V^2 P - (P V P)^2)) with P V^2 P and P V P the
    restrictions to range(P) (Appendix B's expression of || P V Q ||^2)."""
    W = _retained_basis(A, B)
    V = coupling_operator(chain, A, B)
    PVP = W.T @ V @ W
    PV2P = W.T @ V @ V @ W
    M = PV2P - PVP @ PVP
    return float(np.sqrt(max(0.0, np.linalg.eigvalsh(0.5 * (M + M.T))[-1])))
