"""The allocation-free Kronecker-form product against the regular entry point.

Some callers cannot allocate device memory once they are running (a plug-in
inside an application that owns the device memory through its own allocator,
or a loop that must not let cudaMalloc / cudaFree synchronise the device).
For them the library has rmc_kron_matvec_noalloc, which keeps its scratch in a
fixed device array instead of allocating.  This test calls it through the C
ABI twice in a row, with different shapes, and checks each result against
rmc_kron_matvec (which allocates its scratch) within the tolerances of the
other Kronecker-product tests.  It lives in a file collected last.
"""
import numpy as np
import pytest

import instances as I
from tests.gpu_util import dev, host, torch_cuda

import paper_2609_02394_b300 as P

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [0, 1])
def test_noalloc_matches_regular_entry_point_twice(dtype):
    torch = torch_cuda()
    npdt = np.float64 if dtype == 0 else np.float32
    tol = 1e-12 if dtype == 0 else 3e-5
    with P.Context(precision="fp64") as ctx:
        for call, (kA, kB, n_ops, nv, ab) in enumerate([(64, 64, 3, 96, (0.37, -1.3, 0.8)),
                                                        (62, 60, 2, 33, (1.0, 0.0, 0.0))]):
            rng = np.random.default_rng(100 * dtype + call)
            EA, EB, oA, oB, coef = I.random_block_inputs(rng, kA, kB, n_ops)
            X = rng.standard_normal((nv, kA, kB))
            Z = rng.standard_normal((nv, kA, kB))
            d = [dev(a, npdt) for a in (EA, EB, oA, oB, X, Z)]
            Y_ref = dev(np.zeros_like(X), npdt)
            Y_new = dev(np.full_like(X, np.nan), npdt)
            alpha, beta, gamma = ab
            torch.cuda.synchronize()
            ctx.kron_matvec(dtype, kA, kB, n_ops, nv, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                            d[3].data_ptr(), coef, d[4].data_ptr(), Y_ref.data_ptr(), d[5].data_ptr(),
                            alpha, beta, gamma)
            torch.cuda.synchronize()
            st = P.kron_matvec_noalloc(torch.cuda.current_stream().cuda_stream, dtype, kA, kB, n_ops, nv,
                                       d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(), coef,
                                       d[4].data_ptr(), Y_new.data_ptr(), d[5].data_ptr(), alpha, beta, gamma)
            assert st == P.RMC_OK
            ref, got = host(Y_ref), host(Y_new)
            scale = max(1.0, np.abs(ref).max())
            assert np.abs(got - ref).max() <= tol * scale, (call, np.abs(got - ref).max() / scale)


def test_noalloc_rejects_requests_beyond_its_scratch():
    torch = torch_cuda()
    kA = kB = 128
    nv, n_ops = 64, 3      # 3 * 128 * 128 * 64 doubles = 25 MB > 16 MiB
    d = [dev(np.zeros(s)) for s in (kA, kB, (n_ops, kA, kA), (n_ops, kB, kB), (nv, kA, kB), (nv, kA, kB))]
    torch.cuda.synchronize()
    st = P.kron_matvec_noalloc(0, 0, kA, kB, n_ops, nv, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                               d[3].data_ptr(), [1.0, 1.0, 1.0], d[4].data_ptr(), d[5].data_ptr())
    assert st == P.RMC_ERR_NOMEM


@pytest.mark.parametrize("dtype", [0, 1])
def test_noalloc_without_coupling_terms(dtype):
    """n_ops = 0: the product is the diagonal part alone, D o X, scaled and
    combined with X and Z; the allocation-free call agrees with the regular
    one on two shapes in a row."""
    torch = torch_cuda()
    npdt = np.float64 if dtype == 0 else np.float32
    tol = 1e-12 if dtype == 0 else 3e-5
    with P.Context(precision="fp64") as ctx:
        for call, (kA, kB, nv) in enumerate([(40, 24, 17), (7, 130, 3)]):
            rng = np.random.default_rng(500 + 10 * dtype + call)
            EA = np.sort(rng.uniform(-3, 3, kA))
            EB = np.sort(rng.uniform(-3, 3, kB))
            X = rng.standard_normal((nv, kA, kB))
            Z = rng.standard_normal((nv, kA, kB))
            d = [dev(a, npdt) for a in (EA, EB, X, Z)]
            Y_ref = dev(np.zeros_like(X), npdt)
            Y_new = dev(np.full_like(X, np.nan), npdt)
            torch.cuda.synchronize()
            ctx.kron_matvec(dtype, kA, kB, 0, nv, d[0].data_ptr(), d[1].data_ptr(), 0, 0, [], d[2].data_ptr(),
                            Y_ref.data_ptr(), d[3].data_ptr(), 0.5, 0.25, -1.0)
            torch.cuda.synchronize()
            st = P.kron_matvec_noalloc(torch.cuda.current_stream().cuda_stream, dtype, kA, kB, 0, nv,
                                       d[0].data_ptr(), d[1].data_ptr(), 0, 0, [], d[2].data_ptr(),
                                       Y_new.data_ptr(), d[3].data_ptr(), 0.5, 0.25, -1.0)
            assert st == P.RMC_OK
            ref, got = host(Y_ref), host(Y_new)
            # the definition, element by element: 0.5 (E_A[a] + E_B[b]) X + 0.25 X - Z
            want = 0.5 * (EA[:, None] + EB[None, :]) * X + 0.25 * X - Z
            scale = max(1.0, np.abs(want).max())
            assert np.abs(ref - want).max() <= tol * scale
            assert np.abs(got - ref).max() <= tol * scale, (call, np.abs(got - ref).max() / scale)
