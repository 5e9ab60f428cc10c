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
    FP64 central differences (relative step h = 1e-6 of the variable's norm),
    all within 1e-6 relative.  The FD probes are chosen so that the
    directional derivative is of the order of the gradient's norm (a random
    direction of a 67-million-entry dL/dA would see only ~1e-4 of it, and the
    relative bar would then measure noise): for b, directions mixing dL/db
    itself with a random part; for A, rank-1 directions u w^T with w mixing
    dL/dA's top right singular vector with a random part and u = dL/dA w
    (normalised), so u^T dL/dA w is near the top singular value."""
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
    h = 1e-6
    hb = h * np.linalg.norm(b)
    gb_dir = gb / np.linalg.norm(gb)
    for k in range(4):
        e = rng.standard_normal(b.size)
        e = gb_dir + (0.5 * k / 3.0) * e / np.linalg.norm(e)
        e /= np.linalg.norm(e)
        # L(b + t e): only A^T b moves, by t A^T e
        fd = (loss_of(G, Atb + hb * (A64.T @ e)) - loss_of(G, Atb - hb * (A64.T @ e))) / (2 * hb)
        an = gb @ e
        assert abs(fd) > 0.5 * np.linalg.norm(gb)
        assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)
    # top right singular vector of dL/dA (rank 2 by construction: r v^T - (A v) x^T)
    _, _, Vt = np.linalg.svd(gA.T @ gA)
    v1 = Vt[0]
    hA = h * np.linalg.norm(A64)
    for k in range(4):
        wv = rng.standard_normal(A.shape[1])
        wv = v1 + (0.5 * k / 3.0) * wv / np.linalg.norm(wv)
        wv /= np.linalg.norm(wv)
        u = gA @ wv
        u /= np.linalg.norm(u)
        Au = A64.T @ u  # (A + t u w^T): G(t) = G + t (w Au^T + Au w^T) + t^2 w w^T
        ub = u @ b       # rhs(t) = A^T b + t w (u.b)

        def at(t):
            Gt = G + t * (np.outer(wv, Au) + np.outer(Au, wv)) + t * t * np.outer(wv, wv)
            return loss_of(Gt, Atb + t * wv * ub)
        fd = (at(hA) - at(-hA)) / (2 * hA)
        an = u @ gA @ wv
        assert abs(fd) > 0.5 * np.linalg.norm(gA) / np.sqrt(2.0)
        assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


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
