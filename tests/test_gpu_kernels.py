"""Parity of single kernels against the oracle's explicit formulas.

* Kronecker-form product (Eq. (7)) against the oracle's dense H_eff times X,
  including the Chebyshev three-term form alpha H X + beta X + gamma Z.
* Chebyshev filter (single-launch shared-memory form and multi-launch form)
  against the scaled three-term recurrence on the oracle's dense H_eff.
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


def tc_shape_ok(kA, kB, n_ops):
    """Stage 1 (contraction over kB, N = n_ops*kB) runs on the TMA-fed kernel
    when kB is a multiple of 4 (16-byte row pitch), else on the plain-load one
    (N <= 256); stage 2 (contraction over n_ops*kA, N = kA) likewise."""
    s1 = kB % 4 == 0 or n_ops * kB <= 256
    s2 = (n_ops * kA) % 4 == 0 or kA <= 256
    return n_ops >= 1 and s1 and s2


def _kron_reference(EA, EB, oA, oB, coef, X, alpha, beta, gamma, Z):
    """Eq. (7) applied in Kronecker form, FP64: Y_v = D o X_v + sum_j c_j A_j X_v B_j^T,
    then alpha Y + beta X + gamma Z (for shapes whose dense H_eff is too large)."""
    Y = (EA[:, None] + EB[None, :])[None] * X
    for j in range(len(coef)):
        Y = Y + coef[j] * np.einsum("ab,vbc,dc->vad", oA[j], X, oB[j], optimize=True)
    return alpha * Y + beta * X + gamma * Z


WIDE_SHAPES = [(256, 256, 3, 5), (200, 256, 3, 7), (256, 192, 2, 9), (128, 128, 3, 40), (96, 250, 3, 3)]


@pytest.mark.parametrize("kA,kB,n_ops,nv", WIDE_SHAPES)
@pytest.mark.parametrize("dtype", [1, 2])
def test_wide_kron_matvec_matches_kronecker_form(ctx, kA, kB, n_ops, nv, dtype):
    """The shapes of the 256-state merges (stage-1 N = n_ops*kB up to 768, split
    into N tiles; ragged kA = 200 -> a 208-column tile; kB = 250 is not a
    multiple of 4, so stage 1 falls back or is refused) against Eq. (7) in
    Kronecker form in FP64."""
    if dtype == 2 and not tc_shape_ok(kA, kB, n_ops):
        pytest.skip("outside the tensor-core kernels' shapes")
    rng = np.random.default_rng(kA * 3 + kB * 5 + n_ops + 11 * dtype)
    EA, EB, oA, oB, coef = I.random_block_inputs(rng, kA, kB, n_ops)
    X = rng.standard_normal((nv, kA, kB))
    Z = rng.standard_normal((nv, kA, kB))
    for alpha, beta, gamma in [(1.0, 0.0, 0.0), (0.21, 0.5, -0.8)]:
        ref = _kron_reference(EA, EB, oA, oB, coef, X, alpha, beta, gamma, Z)
        d = [dev(a, np.float32) for a in (EA, EB, oA, oB, X, Z)]
        Y = dev(np.full_like(X, np.nan), np.float32)
        torch_cuda().cuda.synchronize()
        ctx.kron_matvec(dtype, kA, kB, n_ops, nv, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                        d[3].data_ptr(), coef, d[4].data_ptr(), Y.data_ptr(), d[5].data_ptr(), alpha, beta, gamma)
        got = host(Y)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(got - ref).max() <= 3e-5 * scale, (alpha, beta, gamma, np.abs(got - ref).max() / scale)


@pytest.mark.parametrize("nv1,nv2,n,sym", [(160, 160, 65536, True), (128, 160, 65536, False), (288, 288, 16384, True),
                                          (37, 200, 4096, False), (5, 7, 1000, False), (96, 96, 4100, True)])
@pytest.mark.parametrize("dtype", [1, 2])
def test_gram_matches_numpy(ctx, nv1, nv2, n, sym, dtype):
    """G = X1 X2^T over long contractions (the Gram products of the wide
    merges: split-K over many CTAs, ragged M and N tiles, the split partial
    sums reduced in a fixed order) against an FP64 product; FP32 and 3xTF32
    both within 2e-5 of max |G| (contractions of up to 65536 terms)."""
    if dtype == 2 and n % 4:
        pytest.skip("the tensor-core form needs n % 4 == 0")
    rng = np.random.default_rng(nv1 * 7 + nv2 * 13 + n + dtype)
    X1 = rng.standard_normal((nv1, n)) / np.sqrt(n)
    X2 = X1.copy() if sym else rng.standard_normal((nv2, n)) / np.sqrt(n)
    ref = X1 @ X2.T
    if sym:
        ref = 0.5 * (ref + ref.T)
    d1, d2 = dev(X1, np.float32), dev(X2, np.float32)
    G = dev(np.full((nv1, nv2), np.nan), np.float32)
    torch_cuda().cuda.synchronize()
    ctx.gram(dtype, nv1, nv2, n, d1.data_ptr(), d2.data_ptr(), G.data_ptr(), sym)
    got = host(G)
    scale = max(1.0, np.abs(ref).max())
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 2e-5 * scale, np.abs(got - ref).max() / scale
    if sym:  # formed from one triangle (FP32 pipe) or averaged (tensor cores): exactly symmetric
        assert np.array_equal(got, got.T)


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
    tensor cores (3xTF32), defined where each stage fits one of the two
    tensor-core kernels (tc_shape_ok)."""
    if dtype == 2 and not tc_shape_ok(kA, kB, n_ops):
        pytest.skip("outside the tensor-core kernels' shapes")
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


def _dense_filter(H, X, deg, theta0, a, ub):
    """Scaled Chebyshev filter (Zhou and Saad) written out on the dense H,
    then column normalisation; deg = 0 is the plain product."""
    nv = X.shape[0]
    Xf = X.reshape(nv, -1)
    if deg == 0:
        return (Xf @ H.T).reshape(X.shape)
    e, c = (ub - a) / 2, (ub + a) / 2
    sigma1 = e / (theta0 - c)
    Y0, Y1 = Xf, (sigma1 / e) * (Xf @ H.T - c * Xf)
    sigma, tau = sigma1, 2.0 / sigma1
    for _ in range(2, deg + 1):
        s1 = 1.0 / (tau - sigma)
        Y0, Y1 = Y1, (2 * s1 / e) * (Y1 @ H.T - c * Y1) - sigma * s1 * Y0
        sigma = s1
    Y1 = Y1 / np.linalg.norm(Y1, axis=1, keepdims=True)
    return Y1.reshape(X.shape)


FILTER_CASES = [(16, 16, 3, 40, 8), (64, 64, 3, 9, 6), (24, 40, 1, 7, 5), (7, 13, 2, 3, 1), (64, 64, 0, 5, 4),
                (20, 30, 3, 6, 0), (62, 60, 3, 11, 12), (1, 1, 1, 2, 3)]


@pytest.mark.parametrize("kA,kB,n_ops,nv,deg", FILTER_CASES)
@pytest.mark.parametrize("dtype", [0, 1, 3])
@pytest.mark.parametrize("fused", [True, False])
def test_chebyshev_filter_matches_dense_recurrence(ctx, kA, kB, n_ops, nv, deg, dtype, fused):
    """Both forms of the filter against the recurrence on the dense H_eff:
    damped interval [theta_m, ub] from the exact spectrum, scaled at its lowest
    eigenvalue; ragged shapes, several vectors per CTA, no coupling, degrees
    0 (plain product), 1 and up to 12.  dtype 3 (FP64 data, double-FP32
    products, single-launch form only) is held to 5e-12."""
    if dtype == 3 and not fused:
        pytest.skip("double-FP32 arithmetic exists in the single-launch form only")
    rng = np.random.default_rng(kA * 7919 + kB * 31 + n_ops * 7 + nv + deg)
    EA, EB, oA, oB, coef = I.random_block_inputs(rng, kA, kB, n_ops)
    H = O.effective_hamiltonian(EA, EB, [(coef[j], oA[j], oB[j]) for j in range(n_ops)])
    lam = np.linalg.eigvalsh(H)
    m = min(len(lam) - 1, max(1, len(lam) // 4))
    theta0, a, ub = lam[0] - 1e-3, lam[m] + 1e-3, lam[-1] + 0.1
    X = rng.standard_normal((nv, kA, kB))
    ref = _dense_filter(H, X, deg, theta0, a, ub)
    npdt = np.float32 if dtype == 1 else np.float64
    d = [dev(v, npdt) for v in (EA, EB, oA, oB, X)]
    Y = dev(np.zeros_like(X), npdt)
    torch_cuda().cuda.synchronize()
    ctx.cheb_filter(dtype, kA, kB, n_ops, nv, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(),
                    coef, d[4].data_ptr(), deg, theta0, a, ub, fused, Y.data_ptr())
    got = host(Y)
    scale = max(1.0, np.abs(ref).max())
    tol = {0: 1e-11, 1: 2e-4, 3: 5e-12}[dtype]
    assert np.abs(got - ref).max() <= tol * scale, np.abs(got - ref).max() / scale


def test_chebyshev_filter_in_place_and_limits(ctx):
    """Y may alias X; the single-launch form rejects vectors it cannot hold
    (128 x 128 with three operators); theta0 < a < ub is required."""
    rng = np.random.default_rng(5)
    kA, kB, n_ops, nv = 16, 12, 2, 5
    EA, EB, oA, oB, coef = I.random_block_inputs(rng, kA, kB, n_ops)
    H = O.effective_hamiltonian(EA, EB, [(coef[j], oA[j], oB[j]) for j in range(n_ops)])
    lam = np.linalg.eigvalsh(H)
    X = rng.standard_normal((nv, kA, kB))
    ref = _dense_filter(H, X, 5, lam[0], lam[20], lam[-1] + 0.1)
    d = [dev(v, np.float64) for v in (EA, EB, oA, oB, X)]
    torch_cuda().cuda.synchronize()
    ctx.cheb_filter(0, kA, kB, n_ops, nv, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(), coef,
                    d[4].data_ptr(), 5, lam[0], lam[20], lam[-1] + 0.1, True, d[4].data_ptr())
    assert np.abs(host(d[4]) - ref).max() <= 1e-11
    big = [dev(np.zeros(s), np.float32) for s in (128, 128, (3, 128, 128), (3, 128, 128), (2, 128, 128))]
    torch_cuda().cuda.synchronize()
    with pytest.raises(P.RmcError) as e:
        ctx.cheb_filter(1, 128, 128, 3, 2, big[0].data_ptr(), big[1].data_ptr(), big[2].data_ptr(),
                        big[3].data_ptr(), [1.0, 1.0, 1.0], big[4].data_ptr(), 3, -2.0, -1.0, 1.0, True,
                        big[4].data_ptr())
    assert e.value.status == P.RMC_ERR_INVAL
    with pytest.raises(P.RmcError) as e:
        ctx.cheb_filter(0, kA, kB, n_ops, nv, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(),
                        coef, d[4].data_ptr(), 3, 1.0, 0.5, 2.0, False, d[4].data_ptr())
    assert e.value.status == P.RMC_ERR_INVAL


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
