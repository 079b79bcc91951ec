"""Plain FP64 CPU oracle: Algorithm 1 (modular projected eigensolver) as written.

TEST INFRASTRUCTURE ONLY -- imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product.

What it computes, step by step, in the paper's order (Sec. II, Algorithm 1):

1. Leaves (Algorithm 1, first step; Eq. (4)): build the dense leaf Hamiltonian
   from its Pauli terms, diagonalise it densely (LAPACK ``dsyevd`` through
   ``numpy.linalg.eigh``), keep the lowest states, and project every operator
   the block must carry into that basis, o = U^T O U (Eq. (9)).
2. Each merge of two neighbouring blocks A, B (Algorithm 1, inner loop):
   form the product basis |alpha>|beta> (Eq. (5)), evaluate the projected
   couplings <alpha beta|V|alpha' beta'> = sum coef o_A (x) o_B (Eq. (8)),
   assemble the dense k_A k_B x k_A k_B effective Hamiltonian
   diag(E_A + E_B) + sum coef kron(o_A, o_B) (Eq. (7)), diagonalise it fully
   (Eq. (10); above FULL_EIGH_MAX_DIM rows only its lowest k_ret + 1
   eigenpairs, from LAPACK's dsyevr on the same dense matrix), keep the lowest
   states (cut and gauge rules below) and rotate
   every carried boundary operator into the new basis,
   o_new = C^T kron(o, I) C or C^T kron(I, o) C.
3. The top block returns its lowest q eigenpairs.

The dense ``eigh`` of the full k_A k_B matrix is the paper's own cost model
(Appendix A: Theta(k^6) per merge); there is no blocking, no Krylov method and
no reordering here, so the code can be checked against Algorithm 1 by eye.

Readings of points the paper leaves open (each also listed in the design notes):

* Index order of the product basis: alpha (module A) is the slow index,
  row = alpha * k_B + beta, which matches numpy's ``kron`` (Eq. (5)).
* Real arithmetic: Y (x) Y = -(iY) (x) (iY) with iY = [[0, 1], [-1, 0]], so a
  YY bond of coefficient c becomes the real term -c * iY (x) iY.
* Retained count: k_ret = min(k, dim) below the top, q at the top, min(k, D)
  at a leaf (the paper's "lowest k" with k > dim impossible otherwise).
* Degenerate cut (the paper says only "lowest k"): below the top, keep the
  largest k' <= k_ret with theta[k'] - theta[k'-1] > tau * max(1, |theta[k']|),
  tau = 1e-7, so no degenerate multiplet is split; if none exists keep k_ret.
  The top level keeps exactly q (energies only are reported there).
* Eigenvector sign (not fixed by the paper): each retained column is flipped
  so that its entry of largest magnitude (first one on exact ties) is positive.
* Tree: a block of n sites is split into floor(n/2) + ceil(n/2) until n <= L0
  (the paper only uses L = L0 * 2^m).
* Operators carried by a block: one per (site, Pauli) end of every two-site
  term with exactly one end inside the block (nearest-neighbour chains carry
  the first and last site's operators; the general coupling of Eq. (3) is
  covered by the same rule).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

import numpy as np

from instances import Chain

TAU_DEG = 1e-7

# --- Pauli algebra, written out (real representation) ---------------------------------

_I2 = np.eye(2)
_X = np.array([[0.0, 1.0], [1.0, 0.0]])
_IY = np.array([[0.0, 1.0], [-1.0, 0.0]])  # i * sigma_y, real antisymmetric
_Z = np.array([[1.0, 0.0], [0.0, -1.0]])


def pauli_matrix(label: str) -> np.ndarray:
    """Real 2x2 matrix carried for a Pauli label ('Y' is carried as iY)."""
    return {"I": _I2, "X": _X, "Y": _IY, "Z": _Z}[label].copy()


def site_operator(mat: np.ndarray, site: int, lo: int, hi: int) -> np.ndarray:
    """mat acting on ``site`` of the block [lo, hi); site lo is the most
    significant tensor factor."""
    out = np.ones((1, 1))
    for s in range(lo, hi):
        out = np.kron(out, mat if s == site else _I2)
    return out


def _bond_real(pi: str, pj: str, coef: float) -> Tuple[np.ndarray, np.ndarray, float]:
    """Real factors and coefficient of the term coef * P_i P_j."""
    if pi == "Y" and pj == "Y":
        return _IY, _IY, -coef
    return pauli_matrix(pi), pauli_matrix(pj), coef


def block_hamiltonian(chain: Chain, lo: int, hi: int) -> np.ndarray:
    """Dense Hamiltonian of sites [lo, hi): all on-site terms on those sites and
    all two-site terms with both ends inside (the module Hamiltonian H_A of
    Eq. (2))."""
    dim = 2 ** (hi - lo)
    H = np.zeros((dim, dim))
    for s, p, c in chain.onsite:
        if lo <= s < hi:
            H += c * site_operator(pauli_matrix(p), s, lo, hi)
    for i, j, pi, pj, c in chain.bonds:
        if lo <= i and j < hi:
            a, b, cc = _bond_real(pi, pj, c)
            H += cc * (site_operator(a, i, lo, hi) @ site_operator(b, j, lo, hi))
    return H


def full_chain_hamiltonian(chain: Chain) -> np.ndarray:
    return block_hamiltonian(chain, 0, chain.n_sites)


def exact_spectrum(chain: Chain, n_low: Optional[int] = None) -> np.ndarray:
    """Exact diagonalisation of the whole chain (small N only)."""
    w = np.linalg.eigh(full_chain_hamiltonian(chain))[0]
    return w if n_low is None else w[:n_low]


def sparse_exact_lowest(chain: Chain, count: int) -> np.ndarray:
    """Lowest ``count`` eigenvalues of the whole chain from its sparse
    Hamiltonian (the same Pauli sums as ``block_hamiltonian``, assembled with
    scipy.sparse Kronecker products) by Lanczos (ARPACK ``eigsh``): exact
    diagonalisation for chains too large for a dense matrix (N <= ~20)."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import eigsh

    N = chain.n_sites

    def op(mat, site):
        out = sp.identity(1, format="csr")
        for s in range(N):
            out = sp.kron(out, sp.csr_matrix(mat if s == site else _I2), format="csr")
        return out

    dim = 2 ** N
    H = sp.csr_matrix((dim, dim))
    for s, p, c in chain.onsite:
        H = H + c * op(pauli_matrix(p), s)
    for i, j, pi, pj, c in chain.bonds:
        a, b, cc = _bond_real(pi, pj, c)
        H = H + cc * (op(a, i) @ op(b, j))
    w = eigsh(H, k=count, which="SA", tol=1e-14, ncv=max(4 * count, 40))[0]
    return np.sort(w)


# --- recursion tree and carried operators ---------------------------------------------

def split_tree(lo: int, hi: int, L0: int):
    """Binary tree over sites: a leaf is (lo, hi); a node is (left, right)."""
    n = hi - lo
    if n <= L0:
        return (lo, hi)
    mid = lo + n // 2
    return (split_tree(lo, mid, L0), split_tree(mid, hi, L0))


def boundary_ops(chain: Chain, lo: int, hi: int) -> List[Tuple[int, str]]:
    """(site, Pauli) pairs the block [lo, hi) must carry: the inside end of
    every two-site term that crosses the block's boundary.  Sorted."""
    need = set()
    for i, j, pi, pj, _ in chain.bonds:
        i_in, j_in = lo <= i < hi, lo <= j < hi
        if i_in and not j_in:
            need.add((i, pi))
        if j_in and not i_in:
            need.add((j, pj))
    return sorted(need)


def carried_matrix(label: str) -> np.ndarray:
    return pauli_matrix(label)


def merge_terms(chain: Chain, A_lo: int, A_hi: int, B_lo: int, B_hi: int):
    """Coupling terms of a merge: (coef, (site_a, P_a), (site_b, P_b)) for every
    two-site term with one end in A and the other in B (Eq. (3) with the sign
    folded into coef and Y Y written as -iY iY)."""
    out = []
    for i, j, pi, pj, c in chain.bonds:
        if A_lo <= i < A_hi and B_lo <= j < B_hi:
            _, _, cc = _bond_real(pi, pj, c)
            out.append((cc, (i, pi), (j, pj)))
    return out


# --- blocks ---------------------------------------------------------------------------

@dataclasses.dataclass
class Block:
    lo: int
    hi: int
    E: np.ndarray                      # retained energies, ascending
    ops: Dict[Tuple[int, str], np.ndarray]   # carried operators in the retained basis
    U: np.ndarray                      # leaf: D x k eigenvectors; merge: C (kA kB x k)
    is_leaf: bool
    children: Optional[Tuple["Block", "Block"]] = None


@dataclasses.dataclass
class MergeRecord:
    lo: int
    mid: int
    hi: int
    H_eff: Optional[np.ndarray]
    theta: np.ndarray      # spectrum of H_eff (ascending): all of it, or the lowest
                           # k_ret + 1 above FULL_EIGH_MAX_DIM
    k_ret: int
    k_eff: int


@dataclasses.dataclass
class OracleResult:
    energies: np.ndarray
    top: Block
    merges: List[MergeRecord]


def _is_symmetric(H: np.ndarray, atol: float) -> bool:
    """|H - H^T| <= atol everywhere, checked one row slab at a time."""
    n = H.shape[0]
    step = max(1, (1 << 24) // max(1, n))
    for r in range(0, n, step):
        if np.max(np.abs(H[r:r + step, :] - H[:, r:r + step].T), initial=0.0) > atol:
            return False
    return True


def cut_rule(theta: np.ndarray, k_ret: int, tau: float = TAU_DEG) -> int:
    """Largest k' <= k_ret such that theta[k'] - theta[k'-1] > tau*max(1,|theta[k']|),
    so a (near-)degenerate multiplet is never split; k_ret when it keeps all
    states or no such k' exists."""
    n = len(theta)
    if k_ret >= n:
        return n
    for kp in range(k_ret, 0, -1):
        if theta[kp] - theta[kp - 1] > tau * max(1.0, abs(theta[kp])):
            return kp
    return k_ret


def gauge_fix(C: np.ndarray) -> np.ndarray:
    """Flip each column so that its largest-|.| entry (first on ties) is > 0."""
    C = C.copy()
    idx = np.argmax(np.abs(C), axis=0)
    signs = np.sign(C[idx, np.arange(C.shape[1])])
    signs[signs == 0] = 1.0
    return C * signs


def leaf_block(chain: Chain, lo: int, hi: int, k: int, is_top: bool = False) -> Block:
    """Algorithm 1, first step: dense ED of the leaf, keep the lowest states,
    project the carried operators (Eqs. (4), (9))."""
    H = block_hamiltonian(chain, lo, hi)
    w, U = np.linalg.eigh(H)
    D = H.shape[0]
    if is_top:
        k_eff = min(chain.q, D)
    else:
        k_eff = cut_rule(w, min(k, D))
    U = gauge_fix(U[:, :k_eff])
    ops = {}
    if not is_top:
        for site, p in boundary_ops(chain, lo, hi):
            O = site_operator(carried_matrix(p), site, lo, hi)
            ops[(site, p)] = U.T @ O @ U
    return Block(lo, hi, w[:k_eff].copy(), ops, U, True)


def effective_hamiltonian(EA: np.ndarray, EB: np.ndarray, coupling) -> np.ndarray:
    """Eq. (7) written out: diag(E_A[a] + E_B[b]) + sum coef * kron(o_A, o_B),
    with ``coupling`` a list of (coef, o_A, o_B) in the retained bases.

    The matrix is filled one row slab at a time: the k_B rows of product
    states (a, .) are diag(E_A[a] + E_B) on the diagonal block plus
    sum coef * kron(o_A[a, :], o_B), i.e. the rows a*k_B .. a*k_B + k_B - 1 of
    the Kronecker products, so no temporary as large as H is ever made (a
    merge of two 256-state blocks gives a 65536 x 65536 matrix of 34 GB)."""
    kA, kB = len(EA), len(EB)
    n = kA * kB
    H = np.zeros((n, n))
    for a in range(kA):
        rows = slice(a * kB, (a + 1) * kB)
        for coef, oA, oB in coupling:
            H[rows, :] += coef * np.kron(oA[a:a + 1, :], oB)
        H[rows, rows] += np.diag(EA[a] + EB)
    return H


# Above this dimension a merge computes only the eigenpairs it needs (the
# lowest k_ret + 1: the kept ones and the one the cut rule compares with).
FULL_EIGH_MAX_DIM = 4096


def lowest_eigenpairs(H: np.ndarray, count: int, full_max: Optional[int] = None):
    """Eigenvalues (ascending) and eigenvectors of the symmetric H (Eq. (10)).

    Up to ``full_max`` rows: the whole spectrum from LAPACK dsyevd
    (``numpy.linalg.eigh``), the paper's full dense eigendecomposition.  Larger:
    the lowest ``count`` pairs from LAPACK dsyevr (``scipy.linalg.eigh`` with
    ``subset_by_index``) on the same dense matrix -- the same eigenpairs, without
    the eigenvectors nobody keeps.  H may be overwritten in that case."""
    n = H.shape[0]
    lim = FULL_EIGH_MAX_DIM if full_max is None else full_max
    if n <= lim or count >= n:
        return np.linalg.eigh(H)
    import scipy.linalg as sl
    # H is symmetric, so its transpose view is the same matrix; that view is
    # Fortran-ordered, which LAPACK takes without a copy (a 65536-row matrix is
    # 34 GB)
    return sl.eigh(H.T, subset_by_index=[0, count - 1], driver="evr", overwrite_a=True, check_finite=False)


def rotate_operator(C: np.ndarray, o: np.ndarray, side: int, kA: int, kB: int) -> np.ndarray:
    """Algorithm 1's operator transform: C^T kron(o, I) C for an operator of
    module A (side 0), C^T kron(I, o) C for one of module B (side 1)."""
    big = np.kron(o, np.eye(kB)) if side == 0 else np.kron(np.eye(kA), o)
    return C.T @ big @ C


def merge_blocks(chain: Chain, A: Block, B: Block, k: int, is_top: bool,
                 keep_matrix: bool = False) -> Tuple[Block, MergeRecord]:
    """One merge of Algorithm 1: product basis, projected couplings, dense
    H_eff (Eq. (7)), full eigendecomposition (Eq. (10)), keep, rotate."""
    kA, kB = len(A.E), len(B.E)
    n = kA * kB
    H = effective_hamiltonian(A.E, B.E, [(coef, A.ops[ka], B.ops[kb])
                                         for coef, ka, kb in merge_terms(chain, A.lo, A.hi, B.lo, B.hi)])
    if not _is_symmetric(H, 1e-12):
        raise AssertionError("effective Hamiltonian is not symmetric")
    k_ret = min(chain.q, n) if is_top else min(k, n)
    theta, V = lowest_eigenpairs(H.copy() if keep_matrix else H, min(n, k_ret + 1))
    if is_top:
        k_eff = k_ret
    else:
        k_eff = cut_rule(theta, k_ret)
    C = gauge_fix(V[:, :k_eff])
    ops = {}
    if not is_top:
        for key in boundary_ops(chain, A.lo, B.hi):
            site, _ = key
            if A.lo <= site < A.hi:
                ops[key] = rotate_operator(C, A.ops[key], 0, kA, kB)
            else:
                ops[key] = rotate_operator(C, B.ops[key], 1, kA, kB)
    blk = Block(A.lo, B.hi, theta[:k_eff].copy(), ops, C, False, (A, B))
    rec = MergeRecord(A.lo, A.hi, B.hi, H if keep_matrix else None, theta, k_ret, k_eff)
    return blk, rec


def solve(chain: Chain, keep_matrices: bool = False) -> OracleResult:
    """Algorithm 1 over the whole chain; returns the lowest q energies of the top
    block, the block tree and one record per merge (post-order)."""
    chain.validate()
    merges: List[MergeRecord] = []
    tree = split_tree(0, chain.n_sites, chain.leaf_sites)

    def build(node, is_top):
        if isinstance(node[0], int):
            return leaf_block(chain, node[0], node[1], chain.k, is_top)
        A = build(node[0], False)
        B = build(node[1], False)
        blk, rec = merge_blocks(chain, A, B, chain.k, is_top, keep_matrices)
        merges.append(rec)
        return blk

    top = build(tree, True)
    return OracleResult(top.E[: chain.q].copy(), top, merges)


def lift_states(block: Block) -> np.ndarray:
    """Physical-basis vectors of a block's retained states (Eq. (11)), applied
    recursively: psi = (U_A (x) U_B) C.  Small N only."""
    if block.is_leaf:
        return block.U
    A, B = block.children
    PA, PB = lift_states(A), lift_states(B)
    k = block.U.shape[1]
    out = np.empty((PA.shape[0] * PB.shape[0], k))
    for mu in range(k):
        Xmu = block.U[:, mu].reshape(PA.shape[1], PB.shape[1])
        out[:, mu] = (PA @ Xmu @ PB.T).reshape(-1)
    return out
