"""The no-allocation gradient entry point, ihs_gradient_noalloc.

Some callers cannot allocate device memory when they call into the library
(their device memory is all owned by their own pool allocator, or they run
in a latency-critical loop that cannot take cudaMalloc's implicit device-wide
synchronisation).  For them the dense gradient pass g = A^T (b - A x) has a
variant whose scratch is a fixed array inside the library.  This file checks
that it returns what ihs_gradient returns, on two calls in a row (the second
call must not see stale partials of the first).  It is named to be collected
last, and it passes alone in a fresh process as well as after the others."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,d,dt", [(30001, 500, np.float32), (20000, 50, np.float64),
                                    (5000, 37, np.float32), (70, 1000, np.float32)])
def test_noalloc_gradient_matches_ihs_gradient(cuda_lib, n, d, dt):
    """Same tolerance as the gradient parity tests: 1e-12 relative to
    sum_i |A_i| |r_i| per entry."""
    rng = np.random.default_rng(n + d)
    A = rng.standard_normal((n, d)).astype(dt)
    xs = rng.standard_normal(d)
    b = A.astype(np.float64) @ xs + 0.1 * rng.standard_normal(n)
    Ad, bd = dev(A), dev(b)
    solver = cuda_lib.IHS(Ad, bd, m=max(d, 64), precision="fp64")
    A64 = A.astype(np.float64)
    for call in range(2):
        x = xs + (10.0 ** -(call + 2)) * rng.standard_normal(d)
        xd = dev(x)
        g_ref = solver.gradient(xd).cpu().numpy()
        g_na = cuda_lib.ihs_gradient_noalloc(Ad, bd, xd).cpu().numpy()
        r = b - A64 @ x
        scale = np.abs(A64).T @ np.abs(r)
        assert np.all(np.abs(g_na - g_ref) <= 1e-12 * scale), call


def test_noalloc_gradient_with_lambda_and_bad_shape(cuda_lib):
    """The lambda term matches the ridge context's gradient; d > 1024 is
    rejected with IHS_ERR_UNSUPPORTED before any work is issued."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((4096, 64)).astype(np.float32)
    b = rng.standard_normal(4096)
    x = rng.standard_normal(64)
    Ad, bd, xd = dev(A), dev(b), dev(x)
    ridge = cuda_lib.IHS(Ad, bd, kind="ridge", param=0.25, m=640, precision="fp64")
    for _ in range(2):
        g_ref = ridge.gradient(xd).cpu().numpy()
        g_na = cuda_lib.ihs_gradient_noalloc(Ad, bd, xd, 0.25).cpu().numpy()
        scale = np.abs(A.astype(np.float64)).T @ np.abs(b - A.astype(np.float64) @ x) + 0.25 * np.abs(x)
        assert np.all(np.abs(g_na - g_ref) <= 1e-12 * scale)
    big = torch.zeros((4, 1025), dtype=torch.float32, device="cuda")
    with pytest.raises(cuda_lib.IHSError) as e:
        cuda_lib.ihs_gradient_noalloc(big, torch.zeros(4, dtype=torch.float64, device="cuda"),
                                      torch.zeros(1025, dtype=torch.float64, device="cuda"))
    assert e.value.status == 8
