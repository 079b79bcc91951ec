"""Parity of single kernels against the oracle's explicit formulas.

* Kronecker-form product (Eq. (7)) against the oracle's dense H_eff times X,
  including the Chebyshev three-term form alpha H X + beta X + gamma Z.
* Small symmetric eigensolver (FP32 Jacobi + FP64 refinement) against LAPACK.
* Operator rotation against C^T kron(o, I) C / C^T kron(I, o) C.
"""
import numpy as np
import pytest

import instances as I
from oracle import rmc_oracle as O
from tests.gpu_util import dev, host, torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1, 3), (4, 4, 1, 5), (5, 7, 2, 9), (16, 16, 3, 72), (62, 60, 3, 33), (64, 64, 3, 96),
          (64, 64, 1, 1), (128, 96, 1, 17), (3, 130, 2, 4)]


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    c = P.Context(precision="fp64")
    yield c
    c.close()


def _dense_reference(EA, EB, oA, oB, coef, X, alpha, beta, gamma, Z):
    H = O.effective_hamiltonian(EA, EB, [(coef[j], oA[j], oB[j]) for j in range(len(coef))])
    nv, kA, kB = X.shape
    Xf = X.reshape(nv, -1)
    Y = alpha * (Xf @ H.T) + beta * Xf
    if gamma:
        Y = Y + gamma * Z.reshape(nv, -1)
    return Y.reshape(nv, kA, kB)


@pytest.mark.parametrize("kA,kB,n_ops,nv", SHAPES)
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_kron_matvec_matches_dense_heff(ctx, kA, kB, n_ops, nv, dtype):
    """dtype 0: FP64; 1: FP32 on the FP32 pipe; 2: FP32 data on the tcgen05
    tensor cores (3xTF32), defined for n_ops >= 1, n_ops*kB <= 256, kA <= 256."""
    if dtype == 2 and not (n_ops >= 1 and n_ops * kB <= 256 and kA <= 256):
        pytest.skip("outside the tensor-core kernel's shapes")
    rng = np.random.default_rng(kA * 1000 + kB * 10 + n_ops + dtype)
    EA, EB, oA, oB, coef = I.random_block_inputs(rng, kA, kB, n_ops)
    X = rng.standard_normal((nv, kA, kB))
    Z = rng.standard_normal((nv, kA, kB))
    for alpha, beta, gamma in [(1.0, 0.0, 0.0), (0.37, -1.3, 0.0), (0.21, 0.5, -0.8)]:
        ref = _dense_reference(EA, EB, oA, oB, coef, X, alpha, beta, gamma, Z)
        npdt = np.float64 if dtype == 0 else np.float32
        d = [dev(a, npdt) for a in (EA, EB, oA, oB, X, Z)]
        Y = dev(np.zeros_like(X), npdt)
        torch_cuda().cuda.synchronize()
        ctx.kron_matvec(dtype, kA, kB, n_ops, nv, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                        d[3].data_ptr(), coef, d[4].data_ptr(), Y.data_ptr(), d[5].data_ptr(), alpha, beta, gamma)
        got = host(Y)
        scale = max(1.0, np.abs(ref).max())
        tol = 1e-12 if dtype == 0 else 3e-5
        assert np.abs(got - ref).max() <= tol * scale, (alpha, beta, gamma, np.abs(got - ref).max() / scale)


def test_tensor_core_product_rejects_shapes_it_cannot_hold(ctx):
    kA, kB, n_ops, nv = 8, 130, 2, 2
    d = [dev(np.zeros(s), np.float32) for s in (kA, kB, (n_ops, kA, kA), (n_ops, kB, kB), (nv, kA, kB), (nv, kA, kB))]
    torch_cuda().cuda.synchronize()
    with pytest.raises(P.RmcError) as e:
        ctx.kron_matvec(2, kA, kB, n_ops, nv, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(),
                        [1.0, 1.0], d[4].data_ptr(), d[5].data_ptr())
    assert e.value.status == P.RMC_ERR_INVAL


def test_kron_matvec_without_coupling(ctx):
    rng = np.random.default_rng(3)
    EA, EB, oA, oB, coef = I.random_block_inputs(rng, 6, 9, 1)
    X = rng.standard_normal((4, 6, 9))
    d = [dev(a) for a in (EA, EB, X)]
    Y = dev(np.zeros_like(X))
    torch_cuda().cuda.synchronize()
    ctx.kron_matvec(0, 6, 9, 0, 4, d[0].data_ptr(), d[1].data_ptr(), 0, 0, [], d[2].data_ptr(), Y.data_ptr())
    ref = (EA[:, None] + EB[None, :])[None] * X
    np.testing.assert_allclose(host(Y), ref, atol=1e-13)


def _sym(rng, m, spectrum=None):
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    w = rng.uniform(-10, 10, m) if spectrum is None else np.asarray(spectrum, float)
    return (Q * w) @ Q.T


@pytest.mark.parametrize("m", [1, 2, 3, 7, 16, 33, 64, 96, 127, 160])
def test_syev_matches_lapack(ctx, m):
    rng = np.random.default_rng(m)
    S = _sym(rng, m)
    S = 0.5 * (S + S.T)
    dS, dw, dV = dev(S), dev(np.zeros(m)), dev(np.zeros((m, m)))
    torch_cuda().cuda.synchronize()
    ctx.syev(m, dS.data_ptr(), dw.data_ptr(), dV.data_ptr())
    w, V = host(dw), host(dV)
    wr = np.linalg.eigvalsh(S)
    nrm = np.abs(S).max()
    assert np.abs(w - wr).max() <= 1e-12 * nrm
    assert np.abs(V.T @ V - np.eye(m)).max() <= 1e-13
    assert np.abs(S @ V - V * w).max() <= 1e-12 * nrm


def test_syev_degenerate_clusters(ctx):
    """Exact multiplets (as in SU(2)-symmetric spectra): eigenvalues exact and
    the eigenvector matrix orthonormal; any basis of a cluster is valid."""
    rng = np.random.default_rng(7)
    spec = [-3.0] * 1 + [-1.0] * 3 + [0.5] * 5 + [2.0] * 3 + list(rng.uniform(3, 5, 12))
    m = len(spec)
    S = _sym(rng, m, spec)
    S = 0.5 * (S + S.T)
    dS, dw, dV = dev(S), dev(np.zeros(m)), dev(np.zeros((m, m)))
    torch_cuda().cuda.synchronize()
    ctx.syev(m, dS.data_ptr(), dw.data_ptr(), dV.data_ptr())
    w, V = host(dw), host(dV)
    np.testing.assert_allclose(w, np.sort(spec), atol=1e-12 * 5)
    assert np.abs(V.T @ V - np.eye(m)).max() <= 1e-13
    assert np.abs(S @ V - V * w).max() <= 1e-12 * 5


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("kA,kB,kr", [(4, 4, 8), (16, 16, 64), (62, 60, 64), (7, 3, 5)])
def test_rotate_op_matches_explicit(ctx, side, kA, kB, kr):
    rng = np.random.default_rng(side * 100 + kA + kB + kr)
    n = kA * kB
    C, _ = np.linalg.qr(rng.standard_normal((n, kr)))
    k = kA if side == 0 else kB
    o = rng.standard_normal((k, k))
    o = 0.5 * (o + o.T)
    ref = O.rotate_operator(C, o, side, kA, kB)
    dC, do, dout = dev(C.T.copy()), dev(o), dev(np.zeros((kr, kr)))
    torch_cuda().cuda.synchronize()
    ctx.rotate_op(side, kA, kB, kr, dC.data_ptr(), do.data_ptr(), dout.data_ptr())
    np.testing.assert_allclose(host(dout), ref, atol=1e-13 * max(1, np.abs(ref).max()))
