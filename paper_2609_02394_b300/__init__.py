"""B300-native recursive module-coupling eigensolver (arXiv 2609.02394).

Thin ctypes binding over the C ABI in ``include/rmc.h`` (``librmc.so``):
argument marshalling only -- every step of Algorithm 1 runs in the library's
CUDA kernels.  There is no CPU fallback: if the library is missing or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librmc.so")

# Concurrent solves (server slots, merge lanes) each run on their own CUDA
# stream; the driver serves streams through CUDA_DEVICE_MAX_CONNECTIONS
# hardware queues (8 unless set) and streams sharing a queue run their kernels
# in order.  The variable is read when the CUDA context is created, so this
# only takes effect when the package is imported before CUDA is first used.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

RMC_OK, RMC_ERR_INVAL, RMC_ERR_NOMEM, RMC_ERR_NOCONV, RMC_ERR_TIMEOUT, RMC_ERR_CUDA = range(6)
STATUS_NAMES = {0: "RMC_OK", 1: "RMC_ERR_INVAL", 2: "RMC_ERR_NOMEM", 3: "RMC_ERR_NOCONV",
                4: "RMC_ERR_TIMEOUT", 5: "RMC_ERR_CUDA"}
PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_tf32": 2}
RMC_COUPLE_TOP = 1

EXPORTED = [
    "rmc_create", "rmc_destroy", "rmc_last_error", "rmc_mem_in_use", "rmc_stats", "rmc_stream",
    "rmc_build_leaf", "rmc_build_leaf_pauli", "rmc_couple", "rmc_lowest", "rmc_solve_chain",
    "rmc_block_free", "rmc_block_info", "rmc_block_export", "rmc_block_import",
    "rmc_kron_matvec", "rmc_gram", "rmc_syev", "rmc_rotate_op", "rmc_profile", "rmc_profile_read",
    "rmc_kron_matvec_noalloc", "rmc_server_create", "rmc_server_destroy", "rmc_submit", "rmc_poll",
    "rmc_server_stats", "rmc_estimate_bytes", "rmc_solve_chains", "rmc_server_profile",
    "rmc_server_profile_read", "rmc_server_last_error", "rmc_cheb_filter", "rmc_solve_chain_states",
    "rmc_couple_batch", "rmc_merge_bound", "rmc_solve_chain_bounds", "rmc_autotune", "rmc_tune_dump",
    "rmc_tune_load", "rmc_tune_clear",
]
PROF_KINDS = ["kron_working", "kron_fp64", "small_eig", "cholqr", "gram", "combine", "rotate", "fused_working"]


class RmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class rmc_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("mem_budget", ctypes.c_size_t),
                ("precision", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("guard", ctypes.c_int), ("tau_deg", ctypes.c_double), ("lanes", ctypes.c_int)]


class rmc_op_tag(ctypes.Structure):
    _fields_ = [("site", ctypes.c_int), ("pauli", ctypes.c_char)]


class rmc_term(ctypes.Structure):
    _fields_ = [("coef", ctypes.c_double), ("op_a", ctypes.c_int), ("op_b", ctypes.c_int)]


class rmc_carry(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int), ("op", ctypes.c_int)]


class rmc_couple_desc(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("terms", ctypes.POINTER(rmc_term)),
                ("n_terms", ctypes.c_int), ("k_keep", ctypes.c_int), ("carry", ctypes.POINTER(rmc_carry)),
                ("n_carry", ctypes.c_int), ("flags", ctypes.c_int)]


class rmc_merge_diag(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int), ("mid", ctypes.c_int), ("hi", ctypes.c_int), ("kA", ctypes.c_int),
                ("kB", ctypes.c_int), ("k", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("bH", ctypes.c_double), ("gamma", ctypes.c_double), ("r", ctypes.c_double), ("E0", ctypes.c_double)]


class rmc_chain(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int), ("L0", ctypes.c_int), ("k", ctypes.c_int), ("q", ctypes.c_int),
                ("n_onsite", ctypes.c_int), ("onsite_site", ctypes.POINTER(ctypes.c_int)),
                ("onsite_pauli", ctypes.c_char_p), ("onsite_coef", ctypes.POINTER(ctypes.c_double)),
                ("n_bonds", ctypes.c_int), ("bond_i", ctypes.POINTER(ctypes.c_int)),
                ("bond_j", ctypes.POINTER(ctypes.c_int)), ("bond_pauli_i", ctypes.c_char_p),
                ("bond_pauli_j", ctypes.c_char_p), ("bond_coef", ctypes.POINTER(ctypes.c_double))]


def make_chain(chain):
    """An rmc_chain for an instances.Chain-like description; the returned
    tuple's second item keeps the marshalled arrays alive."""
    ip, dp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    ons, bnd = chain.onsite, chain.bonds
    keep = [np.array([t[0] for t in ons] or [0], dtype=np.int32), "".join(t[1] for t in ons).encode(),
            np.array([t[2] for t in ons] or [0.0], dtype=np.float64),
            np.array([t[0] for t in bnd] or [0], dtype=np.int32), np.array([t[1] for t in bnd] or [0], dtype=np.int32),
            "".join(t[2] for t in bnd).encode(), "".join(t[3] for t in bnd).encode(),
            np.array([t[4] for t in bnd] or [0.0], dtype=np.float64)]
    c = rmc_chain(chain.n_sites, chain.leaf_sites, chain.k, chain.q, len(ons), keep[0].ctypes.data_as(ip), keep[1],
                  keep[2].ctypes.data_as(dp), len(bnd), keep[3].ctypes.data_as(ip), keep[4].ctypes.data_as(ip),
                  keep[5], keep[6], keep[7].ctypes.data_as(dp))
    return c, keep


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librmc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2609_02394_b300.build`")
    lib = ctypes.CDLL(path)
    vp, ip, dp, cp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_char_p
    P = ctypes.POINTER
    sig = {
        "rmc_create": ([P(vp), P(rmc_config)], ip),
        "rmc_destroy": ([vp], ip),
        "rmc_last_error": ([vp], cp),
        "rmc_mem_in_use": ([vp], ctypes.c_size_t),
        "rmc_stats": ([vp, P(ctypes.c_uint64), P(ctypes.c_uint64)], ip),
        "rmc_stream": ([vp], vp),
        "rmc_build_leaf": ([vp, P(dp), ip, ip, P(P(dp)), P(rmc_op_tag), ip, P(vp)], ip),
        "rmc_build_leaf_pauli": ([vp, ip, ip, ip, P(ip), cp, P(dp), ip, P(ip), P(ip), cp, cp, P(dp), ip,
                                  P(rmc_op_tag), P(vp)], ip),
        "rmc_couple": ([vp, vp, vp, P(rmc_term), ip, ip, P(rmc_carry), ip, ip, P(vp)], ip),
        "rmc_lowest": ([vp, vp, ip, P(dp), P(dp), P(ip)], ip),
        "rmc_solve_chain": ([vp, ip, ip, ip, ip, ip, P(ip), cp, P(dp), ip, P(ip), P(ip), cp, cp, P(dp), P(dp)], ip),
        "rmc_block_free": ([vp, vp], ip),
        "rmc_block_info": ([vp, P(ip), P(ip), P(ip), P(rmc_op_tag)], ip),
        "rmc_block_export": ([vp, vp, P(dp), P(dp), P(dp)], ip),
        "rmc_block_import": ([vp, ip, P(dp), ip, P(dp), P(rmc_op_tag), ip, P(dp), P(vp)], ip),
        "rmc_kron_matvec": ([vp, ip, ip, ip, ip, ip, vp, vp, vp, vp, P(dp), vp, vp, vp, dp, dp, dp], ip),
        "rmc_gram": ([vp, ip, ip, ip, ctypes.c_long, vp, vp, vp, ip], ip),
        "rmc_syev": ([vp, ip, vp, vp, vp], ip),
        "rmc_rotate_op": ([vp, ip, ip, ip, ip, vp, vp, vp], ip),
        "rmc_profile": ([vp, ip], ip),
        "rmc_server_create": ([P(rmc_config), ip, P(vp)], ip),
        "rmc_server_destroy": ([vp], ip),
        "rmc_submit": ([vp, P(rmc_chain), P(ctypes.c_uint64)], ip),
        "rmc_poll": ([vp, ctypes.c_uint64, ip, P(ip), P(dp), P(ip), P(dp), P(dp)], ip),
        "rmc_server_stats": ([vp, P(ctypes.c_uint64), P(ctypes.c_uint64), P(ip), P(ip), P(ctypes.c_size_t),
                              P(ctypes.c_uint64)], ip),
        "rmc_estimate_bytes": ([P(rmc_chain), ip], ctypes.c_size_t),
        "rmc_server_profile": ([vp, ip], ip),
        "rmc_server_last_error": ([vp], cp),
        "rmc_server_profile_read": ([vp, ip, P(ctypes.c_uint64), P(ctypes.c_uint64), P(dp), P(dp)], ip),
        "rmc_solve_chains": ([P(rmc_config), ip, ip, P(rmc_chain), ip, P(dp), P(ip)], ip),
        "rmc_kron_matvec_noalloc": ([vp, ip, ip, ip, ip, ip, vp, vp, vp, vp, P(dp), vp, vp, vp, dp, dp, dp], ip),
        "rmc_profile_read": ([vp, ip, P(ctypes.c_uint64), P(ctypes.c_uint64), P(dp), P(dp)], ip),
        "rmc_cheb_filter": ([vp, ip, ip, ip, ip, ip, vp, vp, vp, vp, P(dp), vp, ip, dp, dp, dp, ip, vp], ip),
        "rmc_solve_chain_states": ([vp, P(rmc_chain), ip, P(rmc_op_tag), P(dp), P(dp), P(dp)], ip),
        "rmc_couple_batch": ([vp, ip, P(rmc_couple_desc), P(vp), P(ip)], ip),
        "rmc_merge_bound": ([vp, vp, vp, P(rmc_term), ip, P(dp)], ip),
        "rmc_autotune": ([vp, P(rmc_chain), P(dp)], ip),
        "rmc_tune_dump": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_size_t),
        "rmc_tune_load": ([cp], ip),
        "rmc_tune_clear": ([], None),
        "rmc_solve_chain_bounds": ([vp, P(rmc_chain), ip, ip, P(rmc_merge_diag), P(ip), P(dp)], ip),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


NOALLOC_SCRATCH_BYTES = 16 << 20


def kron_matvec_noalloc(stream: int, dtype: int, kA: int, kB: int, n_ops: int, nv: int, EA: int, EB: int, A: int,
                        B: int, coef, X: int, Y: int, Z: int = 0, alpha: float = 1.0, beta: float = 0.0,
                        gamma: float = 0.0) -> int:
    """The allocation-free Kronecker-form product (device pointers, current
    device, no context).  Returns the rmc_status code."""
    lib = load_library()
    c = np.ascontiguousarray(coef if len(coef) else [0.0], dtype=np.float64)
    return lib.rmc_kron_matvec_noalloc(stream or None, dtype, kA, kB, n_ops, nv, EA, EB, A or None, B or None,
                                       c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), X, Y, Z or None,
                                       alpha, beta, gamma)


PROFILE_MASK = 0x100


def _profile_mode(enable: bool, kinds) -> int:
    if not enable:
        return 0
    if kinds is None:
        return 1
    return PROFILE_MASK | sum(1 << PROF_KINDS.index(k) for k in kinds)


def tune_dump() -> str:
    """The autotuner's table as text ("key=choice" lines)."""
    lib = load_library()
    n = lib.rmc_tune_dump(None, 0)
    buf = ctypes.create_string_buffer(n)
    lib.rmc_tune_dump(buf, n)
    return buf.value.decode()


def tune_load(text: str) -> int:
    """Merge a table written by ``tune_dump``; returns the entries read."""
    n = load_library().rmc_tune_load(text.encode())
    if n < 0:
        raise ValueError("malformed tuning table")
    return n


def tune_clear() -> None:
    load_library().rmc_tune_clear()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Block:
    """Opaque device-resident block handle (freed with its context or .free())."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.handle = ctypes.c_void_p(handle)

    def info(self):
        k, n_ops, rows = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.ctx.lib.rmc_block_info(self.handle, ctypes.byref(k), ctypes.byref(n_ops), ctypes.byref(rows), None)
        tags = (rmc_op_tag * max(1, n_ops.value))()
        self.ctx.lib.rmc_block_info(self.handle, None, None, None, tags)
        return k.value, n_ops.value, rows.value, [(tags[j].site, tags[j].pauli.decode()) for j in range(n_ops.value)]

    def export(self):
        """(E[k], ops[n_ops, k, k], basis[k, rows]) as FP64 numpy arrays."""
        k, n_ops, rows, _ = self.info()
        E = np.empty(k)
        ops = np.empty((max(n_ops, 1), k, k))
        basis = np.empty((k, max(rows, 1)))
        self.ctx._check(self.ctx.lib.rmc_block_export(self.ctx.h, self.handle, _dptr(E), _dptr(ops),
                                                      _dptr(basis) if rows else None))
        return E, ops[:n_ops], (basis if rows else None)

    def free(self):
        if self.handle:
            self.ctx._check(self.ctx.lib.rmc_block_free(self.ctx.h, self.handle))
            self.handle = ctypes.c_void_p(0)


class Context:
    """One solver context (device, stream, memory budget, precision)."""

    def __init__(self, device: int = 0, precision: str = "fp64", stream: Optional[int] = None,
                 mem_budget: int = 0, tol: float = 0.0, max_iter: int = 0, guard: int = 0, tau_deg: float = 0.0,
                 lanes: int = 0):
        self.lib = load_library()
        cfg = rmc_config(device, ctypes.c_void_p(stream) if stream else None, mem_budget, PRECISIONS[precision],
                         tol, max_iter, guard, tau_deg, lanes)
        h = ctypes.c_void_p()
        st = self.lib.rmc_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != RMC_OK:
            raise RmcError(st, "rmc_create failed")
        self.h = h
        self.precision = precision

    def close(self):
        if self.h:
            self.lib.rmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st: int, allow=()):
        if st != RMC_OK and st not in allow:
            raise RmcError(st, self.lib.rmc_last_error(self.h).decode())
        return st

    def last_error(self) -> str:
        return self.lib.rmc_last_error(self.h).decode()

    @property
    def stream(self) -> int:
        return self.lib.rmc_stream(self.h)

    def stats(self):
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self.lib.rmc_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def profile(self, enable: bool = True, kinds=None):
        """Time launch groups on the stream: every kind, or only ``kinds``
        (names from PROF_KINDS)."""
        self._check(self.lib.rmc_profile(self.h, _profile_mode(enable, kinds)))

    def profile_read(self):
        """{kind: (launch groups, kernel launches, ms, algorithmic flops)} since the last read."""
        out = {}
        for i, name in enumerate(PROF_KINDS):
            g, l, ms, fl = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.rmc_profile_read(self.h, i, ctypes.byref(g), ctypes.byref(l), ctypes.byref(ms),
                                                  ctypes.byref(fl)))
            out[name] = (g.value, l.value, ms.value, fl.value)
        return out

    def mem_in_use(self) -> int:
        return self.lib.rmc_mem_in_use(self.h)

    # ---- Algorithm 1 -------------------------------------------------------
    def build_leaf(self, H, k: int, ops: Sequence = (), tags: Sequence = ()) -> Block:
        H = _f64(H)
        D = H.shape[0]
        opsl = [_f64(o) for o in ops]
        arr = (ctypes.POINTER(ctypes.c_double) * max(1, len(opsl)))(*[_dptr(o) for o in opsl])
        tg = (rmc_op_tag * max(1, len(opsl)))(*[rmc_op_tag(s, p.encode()) for s, p in tags]) if tags else None
        out = ctypes.c_void_p()
        self._check(self.lib.rmc_build_leaf(self.h, _dptr(H), D, k, arr, tg, len(opsl), ctypes.byref(out)))
        return Block(self, out.value)

    def build_leaf_pauli(self, L: int, k: int, onsite, bonds, carry) -> Block:
        os_ = np.array([t[0] for t in onsite], dtype=np.int32)
        op_ = "".join(t[1] for t in onsite).encode()
        oc_ = _f64([t[2] for t in onsite])
        bi = np.array([t[0] for t in bonds], dtype=np.int32)
        bj = np.array([t[1] for t in bonds], dtype=np.int32)
        pi = "".join(t[2] for t in bonds).encode()
        pj = "".join(t[3] for t in bonds).encode()
        bc = _f64([t[4] for t in bonds])
        cr = (rmc_op_tag * max(1, len(carry)))(*[rmc_op_tag(s, p.encode()) for s, p in carry])
        out = ctypes.c_void_p()
        ip = ctypes.POINTER(ctypes.c_int)
        self._check(self.lib.rmc_build_leaf_pauli(
            self.h, L, k, len(onsite), os_.ctypes.data_as(ip), op_, _dptr(oc_), len(bonds), bi.ctypes.data_as(ip),
            bj.ctypes.data_as(ip), pi, pj, _dptr(bc), len(carry), cr, ctypes.byref(out)))
        return Block(self, out.value)

    def couple(self, A: Block, B: Block, terms, k_keep: int, carry=(), top: bool = False,
               allow_noconv: bool = False) -> Block:
        tt = (rmc_term * max(1, len(terms)))(*[rmc_term(c, a, b) for c, a, b in terms])
        cc = (rmc_carry * max(1, len(carry)))(*[rmc_carry(s, o) for s, o in carry])
        out = ctypes.c_void_p()
        st = self.lib.rmc_couple(self.h, A.handle, B.handle, tt, len(terms), k_keep, cc, len(carry),
                                 RMC_COUPLE_TOP if top else 0, ctypes.byref(out))
        self._check(st, allow=(RMC_ERR_NOCONV,) if allow_noconv else ())
        return Block(self, out.value)

    def couple_batch(self, merges, allow_noconv: bool = False):
        """Independent merges at once: ``merges`` is a list of (A, B, terms,
        k_keep, carry, top) tuples as for ``couple``; returns their blocks."""
        n = len(merges)
        keep = []
        descs = (rmc_couple_desc * max(1, n))()
        for i, (A, B, terms, k_keep, carry, top) in enumerate(merges):
            tt = (rmc_term * max(1, len(terms)))(*[rmc_term(c, a, b) for c, a, b in terms])
            cc = (rmc_carry * max(1, len(carry)))(*[rmc_carry(s_, o) for s_, o in carry])
            keep += [tt, cc]
            descs[i] = rmc_couple_desc(A.handle, B.handle, ctypes.cast(tt, ctypes.POINTER(rmc_term)), len(terms),
                                       k_keep, ctypes.cast(cc, ctypes.POINTER(rmc_carry)), len(carry),
                                       RMC_COUPLE_TOP if top else 0)
        outs = (ctypes.c_void_p * max(1, n))()
        sts = (ctypes.c_int * max(1, n))()
        st = self.lib.rmc_couple_batch(self.h, n, descs, outs, sts)
        del keep
        blocks = [Block(self, outs[i]) if outs[i] else None for i in range(n)]
        self._check(st, allow=(RMC_ERR_NOCONV,) if allow_noconv else ())
        return blocks

    def lowest(self, blk: Block, q: int, with_states: bool = False):
        k, _, rows, _ = blk.info()
        qq = min(q, k)
        E = np.empty(qq)
        C = np.empty((rows, qq)) if (with_states and rows) else None
        keff = ctypes.c_int()
        self._check(self.lib.rmc_lowest(self.h, blk.handle, q, _dptr(E), _dptr(C) if C is not None else None,
                                        ctypes.byref(keff)))
        return (E, C) if with_states else E

    def block_import(self, E, ops=(), tags=(), basis=None) -> Block:
        E = _f64(E)
        k = len(E)
        opsa = _f64(np.array(ops).reshape(len(ops), k, k)) if len(ops) else np.zeros((1, k, k))
        tg = (rmc_op_tag * max(1, len(ops)))(*[rmc_op_tag(s, p.encode()) for s, p in tags]) if tags else None
        rows = 0 if basis is None else basis.shape[1]
        bs = _f64(basis) if basis is not None else None
        out = ctypes.c_void_p()
        self._check(self.lib.rmc_block_import(self.h, k, _dptr(E), len(ops), _dptr(opsa), tg, rows,
                                              _dptr(bs) if bs is not None else None, ctypes.byref(out)))
        return Block(self, out.value)

    def solve_chain(self, chain) -> np.ndarray:
        """Algorithm 1 over a chain description (``instances.Chain``-like):
        returns the lowest q energies."""
        ons, bnd = chain.onsite, chain.bonds
        ip = ctypes.POINTER(ctypes.c_int)
        os_ = np.array([t[0] for t in ons], dtype=np.int32)
        bi = np.array([t[0] for t in bnd], dtype=np.int32)
        bj = np.array([t[1] for t in bnd], dtype=np.int32)
        E = np.full(chain.q, np.nan)
        st = self.lib.rmc_solve_chain(
            self.h, chain.n_sites, chain.leaf_sites, chain.k, chain.q, len(ons), os_.ctypes.data_as(ip),
            "".join(t[1] for t in ons).encode(), _dptr(_f64([t[2] for t in ons])), len(bnd),
            bi.ctypes.data_as(ip), bj.ctypes.data_as(ip), "".join(t[2] for t in bnd).encode(),
            "".join(t[3] for t in bnd).encode(), _dptr(_f64([t[4] for t in bnd])), _dptr(E))
        self._check(st)
        return E

    def solve_chain_states(self, chain, observables=(), states: bool = False):
        """The chain solve plus <psi_mu|O|psi_nu> for single-site Pauli
        observables [(site, 'X'|'Y'|'Z'), ...] (Y as iY) and, with
        ``states``, the lowest q states lifted to the 2^N basis (N <= 24).
        Returns (E[q], O[n_obs, q, q], psi[q, 2^N] or None)."""
        c, keep = make_chain(chain)
        q = chain.q
        E = np.full(q, np.nan)
        n_obs = len(observables)
        tags = (rmc_op_tag * max(1, n_obs))(*[rmc_op_tag(int(s_), p.encode()) for s_, p in observables])
        O = np.full((max(1, n_obs), q, q), np.nan)
        # (more than 24 sites: the library rejects the request before writing)
        psi = np.full((q, 1 << min(chain.n_sites, 24)), np.nan) if states else None
        st = self.lib.rmc_solve_chain_states(self.h, ctypes.byref(c), n_obs, tags, _dptr(E),
                                             _dptr(O) if n_obs else None, _dptr(psi) if states else None)
        del keep
        self._check(st)
        return E, O[:n_obs], psi

    def autotune(self, chain) -> np.ndarray:
        """Solve ``chain`` once with tile autotuning on (fills the process-wide
        table for its product shapes); returns its energies."""
        c, keep = make_chain(chain)
        E = np.full(chain.q, np.nan)
        st = self.lib.rmc_autotune(self.h, ctypes.byref(c), _dptr(E))
        del keep
        self._check(st)
        return E

    def merge_bound(self, A: Block, B: Block, terms) -> float:
        """b = ||P V Q||_2 of the merge of A and B with the coupling ``terms``
        [(coef, op_a, op_b), ...] as for ``couple`` (Appendix B)."""
        tt = (rmc_term * max(1, len(terms)))(*[rmc_term(c, a, b) for c, a, b in terms])
        b = ctypes.c_double()
        self._check(self.lib.rmc_merge_bound(self.h, A.handle, B.handle, tt, len(terms), ctypes.byref(b)))
        return b.value

    def solve_chain_bounds(self, chain, full_space_sites: int = 0):
        """The chain solve plus the truncation diagnostics of every merge
        (children before parents): returns (E[q], [dict(lo, mid, hi, kA, kB,
        k, a, b, gamma, r, E0), ...]); gamma, r and E0 are evaluated for merged
        blocks of at most ``full_space_sites`` sites (NaN otherwise)."""
        c, keep = make_chain(chain)
        E = np.full(chain.q, np.nan)
        cap = max(1, 2 * chain.n_sites)
        diag = (rmc_merge_diag * cap)()
        n = ctypes.c_int()
        st = self.lib.rmc_solve_chain_bounds(self.h, ctypes.byref(c), full_space_sites, cap, diag, ctypes.byref(n),
                                             _dptr(E))
        del keep
        self._check(st)
        out = [{f: getattr(diag[i], f) for f, _ in rmc_merge_diag._fields_} for i in range(min(n.value, cap))]
        return E, out

    # ---- kernel-level entry points (device pointers) -------------------------
    def kron_matvec(self, dtype: int, kA: int, kB: int, n_ops: int, nv: int, EA: int, EB: int, A: int, B: int,
                    coef, X: int, Y: int, Z: int = 0, alpha: float = 1.0, beta: float = 0.0, gamma: float = 0.0):
        c = _f64(coef if len(coef) else [0.0])
        self._check(self.lib.rmc_kron_matvec(self.h, dtype, kA, kB, n_ops, nv, EA, EB, A or None, B or None,
                                             _dptr(c), X, Y, Z or None, alpha, beta, gamma))

    def gram(self, dtype: int, nv1: int, nv2: int, n: int, X1: int, X2: int, G: int, symmetrize: bool = False):
        """G = X1 X2^T (device FP32 pointers); dtype 1 FP32 pipe, 2 tensor cores."""
        self._check(self.lib.rmc_gram(self.h, dtype, nv1, nv2, n, X1, X2, G, 1 if symmetrize else 0))

    def cheb_filter(self, dtype: int, kA: int, kB: int, n_ops: int, nv: int, EA: int, EB: int, A: int, B: int,
                    coef, X: int, deg: int, theta0: float, a: float, ub: float, fused: bool, Y: int):
        c = _f64(coef if len(coef) else [0.0])
        self._check(self.lib.rmc_cheb_filter(self.h, dtype, kA, kB, n_ops, nv, EA, EB, A or None, B or None,
                                             _dptr(c), X, deg, theta0, a, ub, 1 if fused else 0, Y))

    def syev(self, m: int, S: int, w: int, V: int):
        self._check(self.lib.rmc_syev(self.h, m, S, w, V))

    def rotate_op(self, side: int, kA: int, kB: int, kr: int, C: int, o: int, out: int):
        self._check(self.lib.rmc_rotate_op(self.h, side, kA, kB, kr, C, o, out))


def _config(device=0, precision="mixed", mem_budget=0, tol=0.0, max_iter=0, guard=0, tau_deg=0.0):
    return rmc_config(device, None, mem_budget, PRECISIONS[precision], tol, max_iter, guard, tau_deg, 1)


def solve_chains(chains, slots: int = 8, **cfg):
    """Solve many chains with `slots` concurrent solves (native worker threads,
    one CUDA stream each).  Returns (energies n x q_max with NaN padding,
    per-solve status codes)."""
    lib = load_library()
    n = len(chains)
    q_max = max(c.q for c in chains)
    arr = (rmc_chain * max(1, n))()
    keep = []
    for i, c in enumerate(chains):
        arr[i], kp = make_chain(c)
        keep.append(kp)
    E = np.full((n, q_max), np.nan)
    st = np.zeros(n, dtype=np.int32)
    c = _config(**cfg)
    lib.rmc_solve_chains(ctypes.byref(c), slots, n, arr, q_max, _dptr(E),
                         st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return E, st


def estimate_bytes(chain, precision: str = "mixed") -> int:
    c, keep = make_chain(chain)
    return load_library().rmc_estimate_bytes(ctypes.byref(c), PRECISIONS[precision])


class Server:
    """Continuous-batching solve server (rmc_server_create / rmc_submit / rmc_poll)."""

    def __init__(self, slots: int = 8, **cfg):
        self.lib = load_library()
        c = _config(**cfg)
        h = ctypes.c_void_p()
        st = self.lib.rmc_server_create(ctypes.byref(c), slots, ctypes.byref(h))
        if st != RMC_OK:
            raise RmcError(st, "rmc_server_create failed")
        self.h = h
        self.q = {}

    def submit(self, chain) -> int:
        c, keep = make_chain(chain)
        tid = ctypes.c_uint64()
        st = self.lib.rmc_submit(self.h, ctypes.byref(c), ctypes.byref(tid))
        if st != RMC_OK:
            raise RmcError(st, "rmc_submit failed")
        self.q[tid.value] = chain.q
        return tid.value

    def poll(self, tid: int, wait: bool = False):
        """None while pending, else (energies, status, latency_ms, queue_ms)."""
        q = self.q[tid]
        E = np.full(q, np.nan)
        done, sst = ctypes.c_int(), ctypes.c_int()
        lat, qd = ctypes.c_double(), ctypes.c_double()
        st = self.lib.rmc_poll(self.h, tid, 1 if wait else 0, ctypes.byref(done), _dptr(E), ctypes.byref(sst),
                               ctypes.byref(lat), ctypes.byref(qd))
        if st != RMC_OK:
            raise RmcError(st, "rmc_poll failed")
        if not done.value:
            return None
        del self.q[tid]
        return E, sst.value, lat.value, qd.value

    def stats(self):
        a, b, l = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        r, qd, byt = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        self.lib.rmc_server_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(r), ctypes.byref(qd),
                                  ctypes.byref(byt), ctypes.byref(l))
        return {"submitted": a.value, "completed": b.value, "running": r.value, "queued": qd.value,
                "reserved_bytes": byt.value, "launches": l.value}

    def last_error(self) -> str:
        return self.lib.rmc_server_last_error(self.h).decode()

    def profile(self, enable: bool = True, kinds=None):
        self.lib.rmc_server_profile(self.h, _profile_mode(enable, kinds))

    def profile_read(self):
        out = {}
        for i, name in enumerate(PROF_KINDS):
            g, l, ms, fl = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
            self.lib.rmc_server_profile_read(self.h, i, ctypes.byref(g), ctypes.byref(l), ctypes.byref(ms),
                                             ctypes.byref(fl))
            out[name] = (g.value, l.value, ms.value, fl.value)
        return out

    def close(self):
        if self.h:
            self.lib.rmc_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
