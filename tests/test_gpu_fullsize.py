"""Parity at the full workload sizes, in the launch configuration the
benchmark uses (ihs_solve, default options): hashes bit-exact on every row,
SA and the gradient against the FP64 oracle, and convergence of the iterate
to the oracle's x_OPT within 1e-10 in the A-seminorm.  (The 20000 x 50 OLS
workload is covered iteration by iteration in test_gpu_parity.py and the
262144 x 256 ridge workload in test_gpu_adjoint.py.)"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_full_lasso_csr_fp64_every_iteration(cuda_lib):
    """CSR 1,000,000 x 200, 2 nnz/row, FP64, SJLT s = 4, m = 2000, l1 ball
    R = ||x*||_1 / 2, 15 iterations: every GPU iterate within 1e-11 of the
    oracle's; the last within 1e-10 of x_OPT."""
    w = synth.make("lasso_csr_fp64")
    C = O.CSR(w["n"], w["d"], w["rowptr"], w["col"], w["val"])
    R = w["param"]
    xs = O.ihs(C, w["b"], O.L1_BALL, R, w["m"], w["s"], 0, w["iters"])
    G = C.gram()
    xo = O.x_opt_l1(C, w["b"], R)
    nrm = np.sqrt(xo @ G @ xo)
    sv = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]), kind="l1",
                      param=R, m=w["m"], s=w["s"], seed=0, precision="fp64", shape=(w["n"], w["d"]))
    x = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
    for t in range(w["iters"]):
        sv.solve(x, t0=t, iters=1)
        e = x.cpu().numpy() - xs[t + 1]
        assert np.sqrt(max(e @ G @ e, 0.0)) / nrm <= 1e-11, t
    assert O.err_A(x.cpu().numpy(), xo, G) <= 1e-10


def test_full_ols_dense_ar1(cuda_lib):
    """Dense 1,048,576 x 500 FP32 AR(1), CountSketch m = 5000, mixed TF32:
    the draw is bit-exact on all rows, SA agrees with the FP64 oracle to FP32
    accumulation accuracy, the FP64-class gradient to 1e-12 of sum |A_i||r_i|,
    and 25 iterations reach 1e-10 of x_OPT."""
    w = synth.make("ols_dense_ar1")
    n, d, m = w["n"], w["d"], w["m"]
    A, b = dev(w["A"]), dev(w["b"])
    bg, sg = cuda_lib.ihs_hash(0, 0, 1, m, n)
    bo, so = O.hash_draw(0, 0, 1, m, n)
    assert np.array_equal(bg.cpu().numpy(), bo) and np.array_equal(sg.cpu().numpy(), so)
    del bg, sg
    A64 = w["A"].astype(np.float64)
    sv = cuda_lib.IHS(A, b, m=m, s=1, seed=0, precision="tf32")
    sv.sketch(0)
    SA, H, _ = sv.get_sketch()
    SAo = O.sketch(A64, m, 1, bo, so)
    assert np.abs(SA.cpu().numpy() - SAo).max() <= 1e-5 * np.abs(SAo).max()
    x = w["x_star"]
    g = sv.gradient(dev(x)).cpu().numpy()
    r, go = O.resid_grad(A64, w["b"], x, want_r=True)
    scale = np.abs(A64).T @ np.abs(r)
    assert np.all(np.abs(g - go) <= 1e-12 * scale)
    xopt = O.x_opt_ols_normal(A64, w["b"])
    G = A64.T @ A64
    xg, rep = sv.solve(iters=25)
    assert rep.status == 0
    assert O.err_A(xg.cpu().numpy(), xopt, G) <= 1e-10


def test_full_lasso_csr_zipf(cuda_lib):
    """CSR 10,000,000 x 1000, 5 nnz/row with Zipf(1.1) columns, FP32, SJLT
    s = 8, m = 10000, mixed TF32, 20 iterations: bit-exact draw, SA and the
    gradient against the oracle, 1e-10 of x_OPT."""
    w = synth.make("lasso_csr_zipf")
    n, d, m, s = w["n"], w["d"], w["m"], w["s"]
    R = w["param"]
    bg, sg = cuda_lib.ihs_hash(0, 0, s, m, n)
    bo, so = O.hash_draw(0, 0, s, m, n)
    assert np.array_equal(bg.cpu().numpy(), bo) and np.array_equal(sg.cpu().numpy(), so)
    del bg, sg
    C = O.CSR(n, d, w["rowptr"], w["col"], w["val"].astype(np.float64))
    sv = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]), kind="l1",
                      param=R, m=m, s=s, seed=0, precision="tf32", shape=(n, d))
    sv.sketch(0)
    SA, _, _ = sv.get_sketch()
    SAo = O.sketch(C, m, s, bo, so)
    assert np.abs(SA.cpu().numpy() - SAo).max() <= 1e-5 * np.abs(SAo).max()
    x = w["x_star"]
    g = sv.gradient(dev(x)).cpu().numpy()
    r, go = O.resid_grad(C, w["b"], x, want_r=True)
    rows = np.repeat(np.arange(n), np.diff(C.rowptr))
    scale = np.zeros(d)
    np.add.at(scale, C.col, np.abs(C.val) * np.abs(r[rows]))
    assert np.all(np.abs(g - go) <= 1e-12 * scale)
    G = C.gram()
    xo = O.l1_ball_qp(G, C.rmatvec(w["b"]), np.zeros(d), R)
    xg, rep = sv.solve(iters=w["iters"])
    assert rep.status == 0
    assert O.err_A(xg.cpu().numpy(), xo, G) <= 1e-10
    assert np.abs(xg.cpu().numpy()).sum() <= R * (1 + 1e-12)
