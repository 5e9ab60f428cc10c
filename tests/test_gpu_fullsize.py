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


U24 = 2.0 ** -24  # unit roundoff of FP32
U_TF32 = 2.0 ** -11  # relative rounding of an FP32 value to TF32


def check_sa_fp32(SA, A64, absA64, m, s, bucket, sign):
    """SA accumulated in FP32 against the FP64 oracle, entry by entry: a sum
    of the L exact terms +-A_ij of a bucket, added in any order with L - 1
    FP32 roundings, is within gamma_{L-1} = (L-1)u/(1-(L-1)u) of the exact
    sum times sum |A_ij| (u = 2^-24; Higham, Accuracy and Stability, Sec. 4.2).
    The oracle's own FP64 error is below 1e-15 of that sum."""
    SAo = O.sketch(A64, m, s, bucket, sign)
    absS = O.sketch(absA64, m, s, bucket, np.ones_like(sign))
    L = np.maximum(np.bincount(bucket.ravel(), minlength=m).astype(np.float64) - 1.0, 0.0)
    gam = L * U24 / (1.0 - L * U24)
    err = np.abs(np.asarray(SA, np.float64) - SAo)
    bound = (gam[:, None] + 1e-15) * absS
    assert np.all(err <= bound), float((err / np.maximum(bound, 1e-300)).max())
    return SAo


def check_hessian_tf32(H, SA, scale):
    """The tensor-core Gram of the FP32 SA with TF32 inputs: each product
    carries at most 2 u_tf32 (+ u_tf32^2) from rounding its two inputs, and
    the FP32 accumulation over at most m terms adds at most m 2^-24 <= 2^-11.5
    at m = 5000, so |H - scale SA^T SA| <= 4 u_tf32 scale |SA|^T |SA| entrywise,
    with SA^T SA formed from the GPU's own SA by the oracle's FP64 loop."""
    SA64 = np.asarray(SA, np.float64)
    Ho = O.gram(SA64, scale)
    absG = O.gram(np.abs(SA64), scale)
    assert np.all(np.abs(np.asarray(H) - Ho) <= 4 * U_TF32 * absG)


@pytest.fixture(scope="module")
def ar1():
    """The 1,048,576 x 500 FP32 AR(1) OLS workload, with A promoted to FP64."""
    w = synth.make("ols_dense_ar1")
    w["A64"] = w["A"].astype(np.float64)
    w["absA64"] = np.abs(w["A64"])
    return w


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


def test_full_ols_dense_ar1(cuda_lib, ar1):
    """Dense 1,048,576 x 500 FP32 AR(1), CountSketch m = 5000, mixed TF32:
    the draw is bit-exact on all rows, the sketch-only pass's SA agrees with
    the FP64 oracle within the FP32 summation bound, the two-pass gradient
    to 1e-12 of sum |A_i||r_i|, and 25 iterations reach 1e-10 of x_OPT."""
    w = ar1
    n, d, m = w["n"], w["d"], w["m"]
    A, b = dev(w["A"]), dev(w["b"])
    bg, sg = cuda_lib.ihs_hash(0, 0, 1, m, n)
    bo, so = O.hash_draw(0, 0, 1, m, n)
    assert np.array_equal(bg.cpu().numpy(), bo) and np.array_equal(sg.cpu().numpy(), so)
    del bg, sg
    A64 = w["A64"]
    sv = cuda_lib.IHS(A, b, m=m, s=1, seed=0, precision="tf32")
    sv.sketch(0)
    SA, H, scale = sv.get_sketch()
    check_sa_fp32(SA.cpu().numpy(), A64, w["absA64"], m, 1, bo, so)
    check_hessian_tf32(H.cpu().numpy(), SA.cpu().numpy(), scale)
    x = w["x_star"]
    g = sv.gradient(dev(x)).cpu().numpy()
    r, go = O.resid_grad(A64, w["b"], x, want_r=True)
    scale_g = np.abs(A64).T @ np.abs(r)
    assert np.all(np.abs(g - go) <= 1e-12 * scale_g)
    xopt = O.x_opt_ols_normal(A64, w["b"])
    G = A64.T @ A64
    xg, rep = sv.solve(iters=25)
    assert rep.status == 0
    assert O.err_A(xg.cpu().numpy(), xopt, G) <= 1e-10


def test_full_lookahead_pipeline_sketches(cuda_lib, ar1):
    """The benchmark's launch configuration (default options: the look-ahead
    fused pipeline, the pass of iteration t forming the gradient at x^t and
    SA of counter t + 1, on 288 CTAs beside the factor).  After solve(iters=k)
    the context holds the sketch of the last iteration, counter k - 1: for
    k = 1 the sketch-only pass's, for k = 2 and 25 the fused pass's, formed
    with the full-size row-chunk plan (buckets split over chunks, the fix-up
    of straddling buckets, the counter one ahead).  Each SA is compared with
    the FP64 oracle's sketch of that counter entry by entry within the FP32
    summation bound, and its Hessian with the Gram of that SA."""
    w = ar1
    n, d, m = w["n"], w["d"], w["m"]
    sv = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), m=m, s=1, seed=0, precision="tf32")
    for k in (1, 2, 25):
        x = torch.zeros(d, dtype=torch.float64, device="cuda")
        _, rep = sv.solve(x, iters=k)
        assert rep.status == 0
        SA, H, scale = sv.get_sketch()
        SA = SA.cpu().numpy()
        bo, so = O.hash_draw(0, k - 1, 1, m, n)
        check_sa_fp32(SA, w["A64"], w["absA64"], m, 1, bo, so)
        check_hessian_tf32(H.cpu().numpy(), SA, scale)


def test_full_fused_pass_sketch_and_gradient(cuda_lib, ar1):
    """One fused pass (ihs_sketch_gradient: the solve's kernel and row-chunk
    plan) at full size: SA of counter 7 within the FP32 summation bound of
    the oracle's, the FP64-class gradient at x = x* + noise within 1e-12 of
    sum |A_i||r_i| of the oracle's (Eq. 2's linear term), and the Hessian of
    that SA; then a second pass at another x and counter (no stale state)."""
    w = ar1
    n, d, m = w["n"], w["d"], w["m"]
    A64 = w["A64"]
    sv = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), m=m, s=1, seed=0, precision="tf32")
    rng = np.random.default_rng(17)
    for t, eps in ((7, 1e-3), (8, 1e-7)):
        x = w["x_star"] + eps * rng.standard_normal(d)
        g = sv.sketch_gradient(t, dev(x)).cpu().numpy()
        SA, H, scale = sv.get_sketch()
        SA = SA.cpu().numpy()
        bo, so = O.hash_draw(0, t, 1, m, n)
        check_sa_fp32(SA, A64, w["absA64"], m, 1, bo, so)
        check_hessian_tf32(H.cpu().numpy(), SA, scale)
        r, go = O.resid_grad(A64, w["b"], x, want_r=True)
        scale_g = w["absA64"].T @ np.abs(r)
        assert np.all(np.abs(g - go) <= 1e-12 * scale_g), t


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
