"""The no-allocation gradient entry point, ihs_gradient_noalloc.

Some callers cannot allocate device memory when they call into the library
(their device memory is all owned by their own pool allocator, or they run
in a latency-critical loop that cannot take cudaMalloc's implicit device-wide
synchronisation).  For them the dense gradient pass g = A^T (b - A x) has a
variant whose scratch is a fixed array inside the library.  This file checks
it against the FP64 CPU oracle and against what ihs_gradient returns, on two
calls in a row (the second call must not see stale partials of the first),
including an empty A and one with fewer rows than a warp's minimum share.
It is named to be collected last, and it passes alone in a fresh process as
well as after the others."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_against_oracle(g, A64, b, x, lam):
    """Against the oracle's FP64 loop, per entry j:
        |g_j - g_j(oracle)| <= 1e-12 sum_i |a_ij| |r_i| + 1e-14 sum_i |a_ij| sum_k |a_ik x_k|.
    The first term is the gradient parity tests' bar (the sum over rows in
    float pairs, about 48 bits).  The second covers the residual itself:
    r_i = b_i - sum_k a_ik x_k is formed from terms that cancel, and any
    finite-precision sum of them (the oracle's FP64 one too, at 1e-16) errs
    relative to sum_k |a_ik x_k|, not to |r_i|; float pairs carry 2^-48 per
    operation, and 1e-14 leaves room for the d / 32 + 5 sequential additions
    of a lane's share and the warp's butterfly.  Where |A_i x| is thousands
    of times |r_i| (70 rows, d = 1000) the second term is the binding one."""
    r, go = O.resid_grad(A64, b, x, want_r=True)
    go = go - lam * x
    absA = np.abs(A64)
    scale = absA.T @ np.abs(r) + abs(lam) * np.abs(x)
    cancel = absA.T @ (absA @ np.abs(x))
    assert np.all(np.abs(g - go) <= 1e-12 * scale + 1e-14 * cancel + 1e-300)


@pytest.mark.parametrize("n,d,dt", [(30001, 500, np.float32), (20000, 50, np.float64),
                                    (5000, 37, np.float32), (70, 1000, np.float32),
                                    (3, 20, np.float32), (3, 20, np.float64)])
def test_noalloc_gradient_matches_oracle_and_ihs_gradient(cuda_lib, n, d, dt):
    """Against the oracle and against ihs_gradient, both at the bar of
    check_against_oracle, on two calls in a row."""
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
        check_against_oracle(g_na, A64, b, x, 0.0)
        absA = np.abs(A64)
        scale = absA.T @ np.abs(b - A64 @ x)
        cancel = absA.T @ (absA @ np.abs(x))
        assert np.all(np.abs(g_na - g_ref) <= 1e-12 * scale + 1e-14 * cancel), call


def test_noalloc_gradient_empty_matrix(cuda_lib):
    """n = 0: no rows, so g = -lambda x exactly (twice, after a call that
    filled the scratch with partials of another problem)."""
    rng = np.random.default_rng(5)
    A1 = rng.standard_normal((4096, 33)).astype(np.float32)
    cuda_lib.ihs_gradient_noalloc(dev(A1), dev(rng.standard_normal(4096)),
                                  dev(rng.standard_normal(33)))
    A0 = torch.zeros((0, 33), dtype=torch.float32, device="cuda")
    b0 = torch.zeros(0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        x = rng.standard_normal(33)
        g = cuda_lib.ihs_gradient_noalloc(A0, b0, dev(x), 0.5).cpu().numpy()
        assert np.array_equal(g, -0.5 * x)


def test_noalloc_gradient_with_lambda_and_bad_shape(cuda_lib):
    """The lambda term matches the oracle and the ridge context's gradient;
    d > 1024 is rejected with IHS_ERR_UNSUPPORTED before any work is issued."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((4096, 64)).astype(np.float32)
    b = rng.standard_normal(4096)
    x = rng.standard_normal(64)
    Ad, bd, xd = dev(A), dev(b), dev(x)
    A64 = A.astype(np.float64)
    ridge = cuda_lib.IHS(Ad, bd, kind="ridge", param=0.25, m=640, precision="fp64")
    for _ in range(2):
        g_ref = ridge.gradient(xd).cpu().numpy()
        g_na = cuda_lib.ihs_gradient_noalloc(Ad, bd, xd, 0.25).cpu().numpy()
        check_against_oracle(g_na, A64, b, x, 0.25)
        scale = np.abs(A64).T @ np.abs(b - A64 @ x) + 0.25 * np.abs(x)
        assert np.all(np.abs(g_na - g_ref) <= 1e-12 * scale)
    big = torch.zeros((4, 1025), dtype=torch.float32, device="cuda")
    with pytest.raises(cuda_lib.IHSError) as e:
        cuda_lib.ihs_gradient_noalloc(big, torch.zeros(4, dtype=torch.float64, device="cuda"),
                                      torch.zeros(1025, dtype=torch.float64, device="cuda"))
    assert e.value.status == 8


def test_noalloc_gradient_rejects_mismatched_vectors(cuda_lib):
    """The C entry point cannot see the vectors' types or lengths, so the
    binding refuses a float32 b, a short b, a short x and a b on the CPU
    before it calls into the library (nothing is launched)."""
    A = torch.zeros((100, 8), dtype=torch.float32, device="cuda")
    b = torch.zeros(100, dtype=torch.float64, device="cuda")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        cuda_lib.ihs_gradient_noalloc(A, b.float(), x)
    with pytest.raises(ValueError):
        cuda_lib.ihs_gradient_noalloc(A, b[:99], x)
    with pytest.raises(ValueError):
        cuda_lib.ihs_gradient_noalloc(A, b, x[:7])
    with pytest.raises(TypeError):
        cuda_lib.ihs_gradient_noalloc(A, b.cpu(), x)
    g = cuda_lib.ihs_gradient_noalloc(A, b, x)
    assert torch.count_nonzero(g).item() == 0
