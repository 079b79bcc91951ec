"""Plant plausible mistakes in the oracle (on the CPU only) and check that the
pins catch each one: a dropped coupling term, a transposed Kronecker order, a
wrong sign of the real Y (x) Y rewrite, operators rotated on the wrong side,
and the wrong tensor factor in the rotation."""
import numpy as np
import pytest

import instances as I
from oracle import closed_forms as CF
from oracle import rmc_oracle as O


def _ed_pin_holds():
    try:
        return _pins()
    except AssertionError:      # the oracle's own symmetry check fired
        return False


def _pins():
    two = I.xxz(2, [0.9], 1.0, 2, 4, 4)
    if not np.allclose(np.linalg.eigvalsh(O.full_chain_hamiltonian(two)),
                       CF.two_site_heisenberg(0.9), atol=1e-12):
        return False
    Js = [0.7, 1.1, 0.9, 1.4, 0.6, 1.2, 1.0]
    xx = I.xxz(8, Js, 0.0, 2, 16, 8)
    if not np.allclose(O.solve(xx).energies, CF.xx_lowest(Js, 8), atol=1e-10):
        return False
    chains = [I.xxz(8, [0.7, 1.1, 0.9, 1.4, 0.6, 1.2, 1.0], 1.0, 2, 16, 8),
              I.tfim(8, 1.0, 0.8, 2, 16, 6),
              I.xxz(8, [1.0] * 7, 1.0, 4, 16, 8, fields=[0.5, -1.2, 1.9, 0.1, -0.7, 1.1, -1.8, 0.3])]
    for c in chains:
        r = O.solve(c)
        if not np.allclose(r.energies, O.exact_spectrum(c, c.q), atol=1e-10):
            return False
    return True


def test_unmutated_oracle_passes():
    assert _ed_pin_holds()


def test_dropped_coupling_is_caught(monkeypatch):
    monkeypatch.setattr(O, "merge_terms", lambda *a, **k: [])
    assert not _ed_pin_holds()


def test_transposed_coupling_operand_is_caught(monkeypatch):
    """o_B (x) o_A in place of o_A (x) o_B in the coupling term of Eq. (7)."""
    real = O.effective_hamiltonian
    calls = {"n": 0}

    def swapped(EA, EB, coupling):
        out = []
        for coef, oA, oB in coupling:
            if oA.shape == oB.shape:
                calls["n"] += 1
                out.append((coef, oB, oA))
            else:
                out.append((coef, oA, oB))
        return real(EA, EB, out)
    monkeypatch.setattr(O, "effective_hamiltonian", swapped)
    held = _ed_pin_holds()
    assert calls["n"] > 0
    assert not held


def _is_diag(m):
    return np.count_nonzero(m - np.diag(np.diagonal(m))) == 0


def test_wrong_yy_sign_is_caught(monkeypatch):
    real = O._bond_real

    def bad(pi, pj, coef):
        a, b, c = real(pi, pj, coef)
        return a, b, abs(coef) if pi == "Y" else c
    monkeypatch.setattr(O, "_bond_real", bad)
    assert not _ed_pin_holds()


def test_rotation_without_transpose_is_caught(monkeypatch):
    real_merge = O.merge_blocks

    def bad(chain, A, B, k, is_top, keep_matrix=False):
        blk, rec = real_merge(chain, A, B, k, is_top, keep_matrix)
        # rotate with C (k x n layout error) replaced by a column-permuted basis
        blk.ops = {key: v[::-1, :] for key, v in blk.ops.items()}
        return blk, rec
    monkeypatch.setattr(O, "merge_blocks", bad)
    assert not _ed_pin_holds()


def test_rotation_on_wrong_tensor_factor_is_caught(monkeypatch):
    """C^T kron(I, o) C used for an A-side operator (and vice versa)."""
    real_kron = np.kron

    class KronSpy:
        def __getattr__(self, name):
            return getattr(np, name)

        @staticmethod
        def eye(n):
            return np.eye(n)

        @staticmethod
        def kron(a, b):
            # the rotation builds kron(o, I) or kron(I, o); swap which factor is I
            if _is_identity(b) and not _is_diag(a):
                return real_kron(np.eye(a.shape[0]), a) if a.shape == b.shape else real_kron(a, b)
            if _is_identity(a) and not _is_diag(b):
                return real_kron(b, np.eye(b.shape[0])) if a.shape == b.shape else real_kron(a, b)
            return real_kron(a, b)
    monkeypatch.setattr(O, "np", KronSpy())
    assert not _ed_pin_holds()


def _is_identity(m):
    return m.ndim == 2 and m.shape[0] == m.shape[1] and np.array_equal(m, np.eye(m.shape[0]))


def test_boundary_operator_on_wrong_site_is_caught(monkeypatch):
    real = O.boundary_ops

    def bad(chain, lo, hi):
        return [((lo if s == hi - 1 else (hi - 1 if s == lo else s)), p) for s, p in real(chain, lo, hi)]
    real_leaf = O.leaf_block

    def bad_leaf(chain, lo, hi, k, is_top=False):
        blk = real_leaf(chain, lo, hi, k, is_top)
        if hi - lo > 1 and not is_top:
            H = O.block_hamiltonian(chain, lo, hi)
            w, U = np.linalg.eigh(H)
            U = O.gauge_fix(U[:, :len(blk.E)])
            ops = {}
            for (site, p), (bsite, _) in zip(real(chain, lo, hi), bad(chain, lo, hi)):
                Om = O.site_operator(O.carried_matrix(p), bsite, lo, hi)
                ops[(site, p)] = U.T @ Om @ U
            blk.ops = ops
        return blk
    monkeypatch.setattr(O, "leaf_block", bad_leaf)
    assert not _ed_pin_holds()
