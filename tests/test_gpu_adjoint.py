"""The adjoint of the ridge solve (not in the paper): GPU gradients through
torch.autograd against the oracle's exact dense-solve gradient and against
FP64 central differences (h = 1e-6) computed on the CPU."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dt,prec", [(np.float64, "fp64"), (np.float32, "tf32")])
def test_adjoint_matches_exact_dense_solve(cuda_lib, dt, prec):
    from paper_1910_14166_gb300.autograd import ihs_ridge
    w = synth.make("ridge_dense", n=20000, d=48, m=480)
    A = w["A"].astype(dt)
    lam = w["param"]
    At = dev(A).requires_grad_(True)
    bt = dev(w["b"]).requires_grad_(True)
    x = ihs_ridge(At, bt, lam=lam, m=480, precision=prec, iters=40)
    xt = dev(w["x_target"])
    loss = ((x - xt) ** 2).sum()
    loss.backward()
    A64 = A.astype(np.float64)
    x_o, dLdb_o, dLdA_o = O.ridge_adjoint(A64, w["b"], lam, 2 * (O.x_opt_ols_normal(A64, w["b"], lam) - w["x_target"]))
    assert relerr(x.detach().cpu().numpy(), x_o) < 1e-10
    assert relerr(bt.grad.cpu().numpy(), dLdb_o) < 1e-9
    tol_A = 1e-9 if dt == np.float64 else 1e-6  # FP32 output: one rounding per entry
    assert relerr(At.grad.cpu().numpy(), dLdA_o) < tol_A


def test_adjoint_full_size_against_central_differences(cuda_lib):
    """262144 x 256 FP32, lam = 1e-3, CountSketch m = 2560, L = ||x - x_t||^2.
    GPU dL/db, dL/dA vs (i) the oracle's exact dense-solve gradient and (ii)
    FP64 central differences (relative step h = 1e-6 of the variable's norm)
    along 6 random directions of b and 6 rank-1 directions u w^T of A, all
    within 1e-6 relative."""
    from paper_1910_14166_gb300.autograd import ihs_ridge
    w = synth.make("ridge_dense")
    A, b, lam, xtar = w["A"], w["b"], w["param"], w["x_target"]
    At = dev(A).requires_grad_(True)
    bt = dev(b).requires_grad_(True)
    x = ihs_ridge(At, bt, lam=lam, m=2560, precision="tf32", iters=40)
    loss = ((x - dev(xtar)) ** 2).sum()
    loss.backward()
    gA = At.grad.cpu().numpy().astype(np.float64)
    gb = bt.grad.cpu().numpy()

    A64 = A.astype(np.float64)
    G = A64.T @ A64 + lam * np.eye(A.shape[1])
    Atb = A64.T @ b
    xo = np.linalg.solve(G, Atb)
    _, dLdb_o, dLdA_o = O.ridge_adjoint(A64, b, lam, 2 * (xo - xtar))
    assert relerr(gb, dLdb_o) < 1e-6
    assert relerr(gA, dLdA_o) < 1e-6

    def loss_of(Gm, rhs):
        xx = np.linalg.solve(Gm, rhs)
        return float(np.sum((xx - xtar) ** 2))

    rng = np.random.default_rng(11)
    # central differences with a relative step h = 1e-6 of each variable's norm
    h = 1e-6
    hb = h * np.linalg.norm(b)
    for _ in range(6):
        e = rng.standard_normal(b.size)
        e /= np.linalg.norm(e)
        fd = (loss_of(G, Atb + hb * (A64.T @ e)) - loss_of(G, Atb - hb * (A64.T @ e))) / (2 * hb)
        assert abs(fd - gb @ e) <= 1e-6 * max(abs(fd), np.linalg.norm(gb) * 1e-3)
    hA = h * np.linalg.norm(A64)
    for _ in range(6):
        u = rng.standard_normal(A.shape[0])
        u /= np.linalg.norm(u)
        v = rng.standard_normal(A.shape[1])
        v /= np.linalg.norm(v)
        Au = A64.T @ u  # (A + t u v^T): G(t) = G + t (v Au^T + Au v^T) + t^2 v v^T, rhs(t) = Atb + t v (u.b)
        ub = u @ b
        def at(t):
            Gt = G + t * (np.outer(v, Au) + np.outer(Au, v)) + t * t * np.outer(v, v)
            return loss_of(Gt, Atb + t * v * ub)
        fd = (at(hA) - at(-hA)) / (2 * hA)
        an = u @ gA @ v
        assert abs(fd - an) <= 1e-6 * max(abs(fd), np.linalg.norm(gA) * 1e-3), (fd, an)


def test_sketch_adjoint_gather(cuda_lib):
    """S^T G on the GPU equals the oracle's gather, and <S A, G> = <A, S^T G>."""
    n, d, m, s = 5001, 7, 64, 4
    rng = np.random.default_rng(2)
    G = rng.standard_normal((m, d))
    out = cuda_lib.ihs_sketch_adjoint(5, 3, s, m, n, dev(G)).cpu().numpy()
    bo, so = O.hash_draw(5, 3, s, m, n)
    ref = O.sketch_adjoint(G, n, s, bo, so)
    assert np.abs(out - ref).max() <= 1e-14 * np.abs(ref).max()
    A = rng.standard_normal((n, d))
    SA = O.sketch(A, m, s, bo, so) / np.sqrt(s)
    assert abs((SA * G).sum() - (A * out).sum()) <= 1e-11 * np.abs(SA).sum()
