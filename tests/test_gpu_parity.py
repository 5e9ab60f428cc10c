"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, on
the same seeded inputs.  Tolerances are stated per test with their origin."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# ------------------------------------------------------------------ hash ---
@pytest.mark.parametrize("seed,t,s,m,n", [(0, 0, 1, 500, 20000), (7, 3, 4, 2000, 100003),
                                          (2**63 + 5, 11, 8, 10000, 4097), (1, 0, 2, 2, 33),
                                          (5, 2, 1, 1, 1000), (9, 1, 64, 128, 77)])
def test_hash_bit_exact(cuda_lib, seed, t, s, m, n):
    """Bucket and sign draws equal the oracle's bit for bit (Sec. 2 draw,
    SplitMix64 keyed by seed, t, block, row)."""
    bg, sg = cuda_lib.ihs_hash(seed, t, s, m, n)
    bo, so = O.hash_draw(seed, t, s, m, n)
    assert np.array_equal(bg.cpu().numpy(), bo)
    assert np.array_equal(sg.cpu().numpy(), so)


# ---------------------------------------------------------------- sketch ---
DENSE_CASES = [
    # (n, d, m, s, dtype, precision)
    (20000, 50, 500, 1, np.float64, "fp64"),     # the 20000 x 50 OLS workload
    (5003, 37, 64, 1, np.float64, "fp64"),       # odd d (scalar path), ragged n
    (777, 13, 1000, 1, np.float64, "fp64"),      # m > n: many empty buckets
    (3000, 9, 9, 1, np.float64, "fp64"),         # few, large buckets straddling chunks
    (4000, 16, 64, 4, np.float64, "fp64"),       # dense SJLT
    (20011, 500, 5000, 1, np.float32, "fp64"),   # FP32 data, FP64 accumulation
    (20011, 500, 5000, 1, np.float32, "tf32"),   # mixed form
    (9000, 256, 2560, 1, np.float32, "bf16"),
    (4099, 130, 1300, 1, np.float32, "tf32"),    # d not a multiple of 4 groups per lane
]


@pytest.mark.parametrize("n,d,m,s,dt,prec", DENSE_CASES)
def test_sketch_dense(cuda_lib, n, d, m, s, dt, prec):
    """SA = S A: FP64 accumulation is bit-identical to the oracle's ascending-row
    loop (<= 1e-12 relative bar); FP32 accumulation within 1e-5 relative to the
    largest |SA| (about 2^-24 per add over ~n/m adds)."""
    rng = np.random.default_rng(n + d)
    A = rng.standard_normal((n, d)).astype(dt)
    b = rng.standard_normal(n)
    solver = cuda_lib.IHS(dev(A), dev(b), m=m, s=s, seed=3, precision=prec)
    solver.sketch(5)
    SA, H, scale = solver.get_sketch()
    bo, so = O.hash_draw(3, 5, s, m, n)
    SAo = O.sketch(A.astype(np.float64), m, s, bo, so)
    if prec == "fp64":
        assert np.array_equal(SA.cpu().numpy(), SAo)
    else:
        assert rel(SA.cpu().numpy(), SAo) < 1e-5
    Ho = O.gram(SAo, 1.0 / s)
    if prec == "fp64":
        assert rel(H.cpu().numpy(), Ho) < 1e-13
    else:
        # TF32 inputs carry 2^-11 relative rounding, BF16 2^-8; the Gram entry
        # error is bounded by about 2u * sum |SA_ri||SA_rj| <= 2u * max diag.
        u = 2.0 ** -11 if prec == "tf32" else 2.0 ** -8
        err = np.abs(H.cpu().numpy() - Ho).max()
        assert err <= 4 * u * np.abs(np.diag(Ho)).max()


@pytest.mark.parametrize("dt,prec,s,n,d,m", [
    (np.float64, "fp64", 4, 30011, 40, 400), (np.float32, "tf32", 8, 30011, 40, 400),
    (np.float64, "fp64", 1, 30011, 40, 400), (np.float64, "fp64", 2, 30011, 40, 400),
    (np.float64, "fp64", 3, 30011, 40, 402), (np.float64, "fp64", 8, 100003, 8, 800),
    (np.float32, "tf32", 1, 30011, 40, 40000), (np.float64, "fp64", 8, 30011, 40, 10000),
    (np.float32, "tf32", 2, 30011, 40, 80000)])
def test_sketch_csr(cuda_lib, dt, prec, s, n, d, m):
    """CSR sketch through the column copy; FP64 exact vs the oracle's
    ascending-row order.  Cases cover s = 1, 2, 3, 4, 8, columns split into
    several items (100003 rows over 8 columns: partial columns merged in
    item order, so a bucket's sum is associated by item and agrees with the
    oracle's entry-by-entry sum to rounding), m/s = 40000 buckets (one
    warp's accumulator fills the shared memory of its CTA; with s = 2 this
    is the one-warp-per-block kernel taking its half of the pair draw), and
    FP64 with 1250 buckets a block (the one-CTA-per-chunk kernel with byte
    tags, bit for bit)."""
    rowptr, col, val = synth.csr_uniform(n, d, 3, 1, dt)
    b = np.random.default_rng(0).standard_normal(n)
    solver = cuda_lib.IHS((dev(rowptr), dev(col), dev(val)), dev(b), m=m, s=s, seed=9,
                          precision=prec, shape=(n, d))
    solver.sketch(2)
    SA, H, _ = solver.get_sketch()
    bo, so = O.hash_draw(9, 2, s, m, n)
    C = O.CSR(n, d, rowptr, col, val.astype(np.float64))
    SAo = O.sketch(C, m, s, bo, so)
    split = n * 3 / d > 16384
    if prec == "fp64" and not split:
        assert np.array_equal(SA.cpu().numpy(), SAo)
    elif prec == "fp64":
        assert rel(SA.cpu().numpy(), SAo) < 1e-13
    else:
        assert rel(SA.cpu().numpy(), SAo) < 1e-5


def test_sketch_csr_fp32_repeats_bit_for_bit(cuda_lib):
    """With FP32 accumulators the CSC sketch adds the lanes of a batch with
    shared-memory atomic adds, so lanes that share a bucket add in the order
    the hardware serialises them, not in lane order.  The accumulator is
    private to one warp and batches add in entry order, so the same sketch
    must give the same bits again: in one context, in a second context, and
    after other sketches.  100 buckets a block make collisions in most
    batches.  The values stay within the FP32 bar of the oracle's sum."""
    n, d, m, s = 200003, 16, 800, 8
    rowptr, col, val = synth.csr_uniform(n, d, 5, 3, np.float32)
    b = np.random.default_rng(1).standard_normal(n)
    args = ((dev(rowptr), dev(col), dev(val)), dev(b))
    kw = dict(m=m, s=s, seed=4, precision="tf32", shape=(n, d))
    one, two = cuda_lib.IHS(*args, **kw), cuda_lib.IHS(*args, **kw)
    one.sketch(7)
    SA1 = one.get_sketch()[0].clone()
    one.sketch(8)
    one.sketch(7)
    two.sketch(7)
    assert torch.equal(one.get_sketch()[0], SA1)
    assert torch.equal(two.get_sketch()[0], SA1)
    bo, so = O.hash_draw(4, 7, s, m, n)
    SAo = O.sketch(O.CSR(n, d, rowptr, col, val.astype(np.float64)), m, s, bo, so)
    # FP32 sums of at most L terms: |err| <= gamma_L sum |terms|, L the
    # longest column chunk (16384 entries) plus the merge of a column's chunks
    absS = O.sketch(O.CSR(n, d, rowptr, col, np.abs(val.astype(np.float64))), m, s, bo,
                    np.ones_like(so))
    L = 16384 + n * 5 // d // 16384 + 1
    u = 2.0 ** -24
    assert np.all(np.abs(SA1.cpu().numpy() - SAo) <= (L * u / (1 - L * u)) * absS + 1e-30)


# -------------------------------------------------------------- gradient ---
@pytest.mark.parametrize("n,d,dt", [(20000, 50, np.float64), (30001, 500, np.float32),
                                    (5000, 37, np.float32), (7000, 1000, np.float32),
                                    (3001, 3, np.float64)])
def test_gradient_dense(cuda_lib, n, d, dt):
    """g = A^T (b - A x): FP64 data in FP64; FP32 data in double-float
    (about 2^-48 per operation).  Bar: 1e-12 relative to sum_i |A_i| |r_i|."""
    rng = np.random.default_rng(d)
    A = rng.standard_normal((n, d)).astype(dt)
    xs = rng.standard_normal(d)
    b = A.astype(np.float64) @ xs + 0.1 * rng.standard_normal(n)
    x = xs + 1e-3 * rng.standard_normal(d)
    solver = cuda_lib.IHS(dev(A), dev(b), m=max(d, 64), precision="fp64")
    r, g = solver.gradient(dev(x), want_r=True)
    ro, go = O.resid_grad(A.astype(np.float64), b, x, want_r=True)
    scale = np.abs(A.astype(np.float64)).T @ np.abs(ro)
    assert np.all(np.abs(g.cpu().numpy() - go) <= 1e-12 * scale)
    assert np.abs(r.cpu().numpy() - ro).max() <= 1e-12 * np.abs(b).max()


def test_gradient_csr(cuda_lib):
    n, d = 50000, 60
    for dt in (np.float64, np.float32):
        rowptr, col, val = synth.csr_uniform(n, d, 4, 2, dt)
        rng = np.random.default_rng(1)
        b = rng.standard_normal(n)
        x = rng.standard_normal(d)
        solver = cuda_lib.IHS((dev(rowptr), dev(col), dev(val)), dev(b), m=120, precision="fp64",
                              shape=(n, d))
        g = solver.gradient(dev(x)).cpu().numpy()
        C = O.CSR(n, d, rowptr, col, val.astype(np.float64))
        ro, go = O.resid_grad(C, b, x, want_r=True)
        scale = np.abs(C.todense()).T @ np.abs(ro)
        assert np.all(np.abs(g - go) <= 1e-12 * scale)


# ------------------------------------------- one pass: sketch + gradient ---
@pytest.mark.parametrize("n,d,m,prec", [(70001, 500, 5000, "tf32"), (20011, 132, 1320, "bf16"),
                                        (3001, 4, 40, "tf32"), (5003, 36, 64, "fp64")])
def test_sketch_gradient_one_pass(cuda_lib, n, d, m, prec):
    """ihs_sketch_gradient: SA of counter 4 and g at x from one read of A (the
    fused pass for FP32 data in the mixed forms; the sketch chain and the
    gradient pass for the plain form).  SA: within the FP32 summation bound
    gamma_{L-1} sum |A_ij| per bucket of L rows (bit-identical to the oracle in
    FP64); g: within 1e-12 of sum_i |A_i||r_i|; H: the Gram of that SA."""
    rng = np.random.default_rng(n + m)
    A = rng.standard_normal((n, d)).astype(np.float32 if prec != "fp64" else np.float64)
    A64 = A.astype(np.float64)
    xs = rng.standard_normal(d)
    b = A64 @ xs + 0.1 * rng.standard_normal(n)
    sv = cuda_lib.IHS(dev(A), dev(b), m=m, s=1, seed=2, precision=prec)
    for t in (4, 5):
        x = xs + 1e-3 * rng.standard_normal(d)
        g = sv.sketch_gradient(t, dev(x)).cpu().numpy()
        SA, H, scale = sv.get_sketch()
        SA = SA.cpu().numpy()
        bo, so = O.hash_draw(2, t, 1, m, n)
        SAo = O.sketch(A64, m, 1, bo, so)
        if prec == "fp64":
            assert np.array_equal(SA, SAo)
            assert rel(H.cpu().numpy(), O.gram(SAo, 1.0)) < 1e-13
        else:
            absS = O.sketch(np.abs(A64), m, 1, bo, np.ones_like(so))
            L = np.maximum(np.bincount(bo.ravel(), minlength=m) - 1.0, 0.0)
            gam = L * 2.0 ** -24 / (1.0 - L * 2.0 ** -24)
            assert np.all(np.abs(SA - SAo) <= (gam[:, None] + 1e-15) * absS)
            u = 2.0 ** -11 if prec == "tf32" else 2.0 ** -8
            SA64 = SA.astype(np.float64)
            assert np.all(np.abs(H.cpu().numpy() - O.gram(SA64, scale))
                          <= 4 * u * O.gram(np.abs(SA64), scale))
        r, go = O.resid_grad(A64, b, x, want_r=True)
        assert np.all(np.abs(g - go) <= 1e-12 * (np.abs(A64).T @ np.abs(r))), t


# ------------------------------------------------------------ full solve ---
def test_ihs_ols_plain_matches_oracle_every_iteration(cuda_lib):
    """20000 x 50 OLS, CountSketch m = 500, 10 iterations, seed 0: every GPU
    iterate within 1e-12 of the oracle's in the A-seminorm relative to x_OPT."""
    w = synth.make("ols_dense_fp64")
    A, b = w["A"], w["b"]
    G = A.T @ A
    xo = O.x_opt_ols_qr(A, b)
    xs = O.ihs(A, b, O.OLS, 0.0, 500, 1, 0, 10)
    solver = cuda_lib.IHS(dev(A), dev(b), m=500, s=1, seed=0, precision="fp64")
    x = torch.zeros(50, dtype=torch.float64, device="cuda")
    nrm = np.sqrt(xo @ G @ xo)
    for t in range(10):
        solver.sketch(t)
        solver.step(x)
        e = x.cpu().numpy() - xs[t + 1]
        assert np.sqrt(e @ G @ e) / nrm <= 1e-12, t
    solver.sync()


def test_ihs_ols_mixed_reaches_1e10(cuda_lib):
    """Mixed form (FP32 data, TF32 Gram, FP32 factor, FP64-class gradient)
    reaches ||x - x_OPT||_A / ||x_OPT||_A <= 1e-10 on an AR(1) design."""
    w = synth.make("ols_dense_ar1", n=65536, d=128, m=1280)
    A64 = w["A"].astype(np.float64)
    xo = O.x_opt_ols_normal(A64, w["b"])
    G = A64.T @ A64
    for prec in ("tf32", "bf16"):
        solver = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), m=1280, s=1, seed=0, precision=prec)
        x, rep = solver.solve(iters=40)
        assert O.err_A(x.cpu().numpy(), xo, G) <= 1e-10, prec


def test_resume_reproduces_run(cuda_lib):
    """Counter-based sketches: 10 iterations equal 4 + 6 resumed at t0 = 4."""
    w = synth.make("ols_dense_fp64", n=5000, d=20, m=200)
    A, b = dev(w["A"]), dev(w["b"])
    s1 = cuda_lib.IHS(A, b, m=200, seed=4)
    x1, _ = s1.solve(iters=10)
    s2 = cuda_lib.IHS(A, b, m=200, seed=4)
    x2, _ = s2.solve(iters=4)
    x2, _ = s2.solve(x2, t0=4, iters=6)
    assert torch.equal(x1, x2)


def test_invalid_arguments_are_rejected(cuda_lib):
    A = torch.zeros((100, 10), dtype=torch.float64, device="cuda")
    b = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(cuda_lib.IHSError) as e:
        cuda_lib.IHS(A, b, m=12, s=5)  # m % s != 0
    assert e.value.status == 1
    with pytest.raises(cuda_lib.IHSError):
        cuda_lib.IHS(A, b, m=5)  # m < d
    with pytest.raises(cuda_lib.IHSError):
        cuda_lib.ihs_hash(0, 0, 3, 10, 5)


def test_binding_rejects_mismatched_tensors(cuda_lib):
    """The C ABI sees bare pointers, so the binding checks every tensor's
    dtype, length and device before it calls into the library: a short or
    float32 b, a CSR triple with a short rowptr or int64 columns, an x of the
    wrong type or length, a Gram of the wrong shape and an S^T G operand
    without m rows are refused with nothing launched for them."""
    n, d, m = 200, 8, 40
    rng = np.random.default_rng(12)
    A = dev(rng.standard_normal((n, d)))
    b = dev(rng.standard_normal(n))
    with pytest.raises(ValueError):
        cuda_lib.IHS(A, b[:-1], m=m)
    with pytest.raises(TypeError):
        cuda_lib.IHS(A, b.float(), m=m)
    rowptr, col, val = synth.csr_uniform(n, d, 3, 1)
    csr = (dev(rowptr), dev(col), dev(val))
    with pytest.raises(ValueError):
        cuda_lib.IHS((csr[0][:-1], csr[1], csr[2]), b, m=m, shape=(n, d))
    with pytest.raises(TypeError):
        cuda_lib.IHS((csr[0], csr[1].long(), csr[2]), b, m=m, shape=(n, d))
    with pytest.raises(ValueError):
        cuda_lib.IHS((csr[0], csr[1][:-1], csr[2]), b, m=m, shape=(n, d))
    sv = cuda_lib.IHS(A, b, m=m)
    x = torch.zeros(d, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        sv.solve(x.float(), iters=1)
    with pytest.raises(ValueError):
        sv.solve(torch.zeros(d + 1, dtype=torch.float64, device="cuda"), iters=1)
    with pytest.raises(ValueError):
        sv.gradient(x[:-1])
    with pytest.raises(ValueError):
        sv.step(x[:-1])
    with pytest.raises(ValueError):
        sv.sketch_error(0, torch.zeros((d, d + 1), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        cuda_lib.ihs_sketch_adjoint(0, 0, 1, m, n,
                                    torch.zeros((m - 1, d), dtype=torch.float64, device="cuda"))
    # the context still works after the refusals
    x, rep = sv.solve(x, iters=3)
    assert rep.status == 0 and torch.isfinite(x).all().item()
    sv.close()


def test_not_spd_is_reported(cuda_lib):
    """A rank-deficient sketch (m >= d but zero columns in A) makes the
    Hessian singular; the factor reports it through the status word."""
    A = torch.zeros((1000, 8), dtype=torch.float64, device="cuda")
    A[:, :4] = torch.randn(1000, 4, dtype=torch.float64, device="cuda")
    b = torch.randn(1000, dtype=torch.float64, device="cuda")
    solver = cuda_lib.IHS(A, b, m=64)
    with pytest.raises(cuda_lib.IHSError) as e:
        solver.solve(iters=1)
    assert e.value.status == 4


# ------------------------------------------------------------------ LASSO ---
def _csr_problem(name, n, d, m, seed=0):
    w = synth.make(name, n=n, d=d, m=m, seed=seed)
    C = O.CSR(w["n"], w["d"], w["rowptr"], w["col"], w["val"].astype(np.float64))
    return w, C


@pytest.mark.parametrize("n,d,m", [(40000, 60, 600), (120000, 600, 3000)])
def test_l1_qp_step_matches_oracle_qp(cuda_lib, n, d, m):
    """One l1-ball step of Eq. 2 on the GPU equals the oracle's exact QP on the
    same H and g (from the same sketch): the QP solution is unique.  At
    d = 600 the step runs as a thread-block cluster whose helper CTAs form
    the FP32 products of the power iteration and FISTA."""
    w, C = _csr_problem("lasso_csr_fp64", n, d, m)
    R = w["param"]
    solver = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]), kind="l1",
                          param=R, m=m, s=4, seed=0, precision="fp64", shape=(w["n"], w["d"]))
    x = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
    xo = np.zeros(w["d"])
    for t in range(4):
        solver.sketch(t)
        SA, H, _ = solver.get_sketch()
        g = solver.gradient(x).cpu().numpy()
        solver.step(x)
        solver.sync()
        Hn = H.cpu().numpy()
        xq = O.l1_ball_qp(Hn, g, x_prev := xo.copy(), R)
        xo = xq
        assert rel(x.cpu().numpy(), xq) < 1e-11, t
        x.copy_(dev(xq))


def test_ihs_lasso_plain_matches_oracle_every_iteration(cuda_lib):
    """LASSO over the l1 ball (R = ||x*||_1 / 2), CSR FP64 data, SJLT s = 4:
    every GPU iterate within 1e-11 of the oracle's (A-seminorm, relative to
    x_OPT), and the final error below 1e-10 after 25 iterations."""
    w, C = _csr_problem("lasso_csr_fp64", 100000, 200, 2000)
    R = w["param"]
    G = C.gram()
    xo = O.x_opt_l1(C, w["b"], R)
    xs = O.ihs(C, w["b"], O.L1_BALL, R, 2000, 4, 0, 25)
    solver = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]), kind="l1",
                          param=R, m=2000, s=4, seed=0, precision="fp64", shape=(w["n"], w["d"]))
    x = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
    nrm = np.sqrt(xo @ G @ xo)
    for t in range(25):
        solver.sketch(t)
        solver.step(x)
        e = x.cpu().numpy() - xs[t + 1]
        assert np.sqrt(max(e @ G @ e, 0)) / nrm <= 1e-11, t
    solver.sync()
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


def test_ihs_lasso_mixed_reaches_1e10(cuda_lib):
    """Mixed form on Zipf-column CSR FP32 data with SJLT s = 8 reaches 1e-10."""
    w, C = _csr_problem("lasso_csr_zipf", 200000, 100, 1000)
    R = w["param"]
    G = C.gram()
    xo = O.x_opt_l1(C, w["b"], R)
    solver = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]), kind="l1",
                          param=R, m=1000, s=8, seed=0, precision="tf32", shape=(w["n"], w["d"]))
    x, rep = solver.solve(iters=30)
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


@pytest.mark.parametrize("kind", ["ols_dense", "l1_csr"])
def test_mixed_fp64_factor(cuda_lib, kind):
    """IHS_FLAG_FP64_FACTOR: the mixed form with the TF32 sketched Hessian
    factored and applied in FP64 (as in the plain form) reaches 1e-10 in the
    same iteration budget as with the FP32 factor; after the first step (the
    same sketch, the same TF32 Hessian) the two iterates agree to FP32
    accuracy, the only difference being the factor's precision."""
    if kind == "ols_dense":
        w = synth.make("ols_dense_ar1", n=65536, d=128, m=1280)
        A64 = w["A"].astype(np.float64)
        xo = O.x_opt_ols_normal(A64, w["b"])
        G = A64.T @ A64
        args = (dev(w["A"]), dev(w["b"]))
        kw = dict(m=1280, precision="tf32")
        iters = 40
    else:
        w, C = _csr_problem("lasso_csr_zipf", 200000, 100, 1000)
        G = C.gram()
        xo = O.x_opt_l1(C, w["b"], w["param"])
        args = ((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]))
        kw = dict(kind="l1", param=w["param"], m=1000, s=8, precision="tf32",
                  shape=(w["n"], w["d"]))
        iters = 30
    f64 = cuda_lib.IHS(*args, fp64_factor=True, **kw)
    f32 = cuda_lib.IHS(*args, **kw)
    x1, r1 = f64.solve(iters=1)
    x2, r2 = f32.solve(iters=1)
    assert r1.status == 0 and r2.status == 0
    e = (x1 - x2).cpu().numpy()
    assert np.sqrt(e @ G @ e) / np.sqrt(xo @ G @ xo) < 1e-5
    x1, _ = f64.solve(x1, t0=1, iters=iters - 1)
    x2, _ = f32.solve(x2, t0=1, iters=iters - 1)
    assert O.err_A(x1.cpu().numpy(), xo, G) < 1e-10
    assert O.err_A(x2.cpu().numpy(), xo, G) < 1e-10


def test_ihs_ridge_plain_and_mixed(cuda_lib):
    w = synth.make("ridge_dense", n=32768, d=64, m=640)
    A64 = w["A"].astype(np.float64)
    xo = O.x_opt_ols_normal(A64, w["b"], lam=w["param"])
    xs = O.ihs(A64, w["b"], O.RIDGE, w["param"], 640, 1, 0, 8)
    G = A64.T @ A64
    s1 = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), kind="ridge", param=w["param"], m=640,
                      precision="fp64")
    x1, _ = s1.solve(iters=8)
    e = x1.cpu().numpy() - xs[-1]
    assert np.sqrt(e @ G @ e) / np.sqrt(xo @ G @ xo) < 1e-12
    s2 = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), kind="ridge", param=w["param"], m=640,
                      precision="tf32")
    x2, _ = s2.solve(iters=35)
    assert O.err_A(x2.cpu().numpy(), xo, G) < 1e-10


def test_profile_counts_stages(cuda_lib):
    w = synth.make("ols_dense_fp64", n=5000, d=20, m=200)
    s1 = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), m=200)
    s1.profile(True)
    s1.solve(iters=3)
    ms, cnt, launches = s1.profile_read()
    assert cnt["sketch"] == 3 and cnt["grad"] == 3 and cnt["step"] == 3
    assert all(v >= 0 for v in ms.values()) and launches > 0


def test_fused_pass_agrees_with_two_passes(cuda_lib):
    """The single fused pass (SA and gradient from one read of A) gives the
    same SA bit for bit and iterates within 1e-12 of the two-pass path, and
    both reach 1e-10 against x_OPT."""
    w = synth.make("ols_dense_ar1", n=50021, d=96, m=960)
    A64 = w["A"].astype(np.float64)
    xo = O.x_opt_ols_normal(A64, w["b"])
    G = A64.T @ A64
    A, b = dev(w["A"]), dev(w["b"])
    fu = cuda_lib.IHS(A, b, m=960, precision="tf32", fuse=True)
    tw = cuda_lib.IHS(A, b, m=960, precision="tf32", fuse=False)
    x1, _ = fu.solve(iters=3)
    x2, _ = tw.solve(iters=3)
    S1, H1, _ = fu.get_sketch()
    S2, H2, _ = tw.get_sketch()
    assert torch.equal(S1, S2) and torch.equal(H1, H2)
    e = (x1 - x2).cpu().numpy()
    assert np.sqrt(e @ G @ e) / np.sqrt(xo @ G @ xo) < 1e-12
    x1, _ = fu.solve(x1, t0=3, iters=30)
    x2, _ = tw.solve(x2, t0=3, iters=30)
    assert O.err_A(x1.cpu().numpy(), xo, G) < 1e-10 and O.err_A(x2.cpu().numpy(), xo, G) < 1e-10


@pytest.mark.parametrize("kind,iters,serial,fp64fac", [
    ("ols", 1, False, False), ("ols", 2, False, False), ("ols", 3, False, False),
    ("ols", 7, False, False), ("ols", 4, True, False), ("ridge", 5, False, False),
    ("l1", 5, False, False), ("l2", 4, False, False),
    ("ols", 1, False, True), ("ols", 2, False, True), ("ols", 3, False, True),
    ("ols", 4, False, True), ("ols", 7, False, True), ("ols", 5, True, True),
    ("ridge", 4, False, True), ("l1", 6, False, True)])
def test_lookahead_matches_in_order_fused(cuda_lib, kind, iters, serial, fp64fac):
    """The look-ahead fused pipeline (SA of iteration t+1 formed in the pass of
    iteration t, its factor beside the next pass; t+2 with the FP64 factor,
    three factors in rotation) takes the same sketches as the in-order fused
    pipeline: the iterates agree to rounding, for 1 to 7 iterations (every
    branch of the sort schedule at both depths), serial or overlapped, and a
    second solve continues to 1e-10.  At this size (fewer than 32 rows per
    warp slot) both pipelines split the rows into the same chunks, so the
    sketch and Hessian left behind (the last iteration's) are identical bit
    for bit and the iterates differ only by the gradient's summation order."""
    # 60001 rows: fewer row pairs than warp slots in every pipeline's plan
    # (the FP64-factor pipeline leaves 32 CTA slots to the factor)
    w = synth.make("ols_dense_ar1", n=60001, d=120, m=1200)
    A64 = w["A"].astype(np.float64)
    A, b = dev(w["A"]), dev(w["b"])
    xo = O.x_opt_ols_normal(A64, w["b"])
    G = A64.T @ A64
    kw = dict(m=1200, precision="tf32", seed=11, serial=serial, fp64_factor=fp64fac)
    if kind == "ridge":
        kw.update(kind="ridge", param=3.0)
    elif kind == "l1":
        kw.update(kind="l1", param=0.5 * float(np.abs(xo).sum()))
    elif kind == "l2":
        kw.update(kind="l2", param=0.5 * float(np.linalg.norm(xo)))
    la = cuda_lib.IHS(A, b, lookahead=True, **kw)
    io = cuda_lib.IHS(A, b, lookahead=False, **kw)
    x1, r1 = la.solve(iters=iters)
    x2, r2 = io.solve(iters=iters)
    assert r1.status == 0 and r2.status == 0
    S1, H1, _ = la.get_sketch()
    S2, H2, _ = io.get_sketch()
    assert torch.equal(S1, S2) and torch.equal(H1, H2)
    e = (x1 - x2).cpu().numpy()
    scale = np.sqrt(max(xo @ G @ xo, 1e-300))
    assert np.sqrt(e @ G @ e) / scale < 1e-11
    if kind == "ols" and not serial:
        x1, _ = la.solve(x1, t0=iters, iters=30)
        x2, _ = io.solve(x2, t0=iters, iters=30)
        assert O.err_A(x1.cpu().numpy(), xo, G) < 1e-10
        assert O.err_A(x2.cpu().numpy(), xo, G) < 1e-10


@pytest.mark.parametrize("kind", ["dense_fp64", "dense_tf32", "csr_fp64", "dense_fp64_d700", "ridge_bf16"])
def test_cluster_factor_matches_grid_factor(cuda_lib, kind):
    """The 16-CTA cluster factor and the cooperative grid factor carry out the
    same tile operations in the same order: the iterates they produce are
    identical bit for bit (FP64 and FP32 factors, d from 50 to 700)."""
    if kind == "csr_fp64":
        w = synth.make("lasso_csr_fp64", n=60000, d=200, m=2000)
        args = ((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]))
        kw = dict(kind="l1", param=w["param"], m=2000, s=4, precision="fp64", shape=(w["n"], w["d"]))
    elif kind == "dense_fp64":
        w = synth.make("ols_dense_fp64")
        args = (dev(w["A"]), dev(w["b"]))
        kw = dict(m=500, precision="fp64")
    elif kind == "dense_fp64_d700":
        w = synth.make("ols_dense_fp64", n=9000, d=700, m=7000)
        args = (dev(w["A"]), dev(w["b"]))
        kw = dict(m=7000, precision="fp64")
    elif kind == "ridge_bf16":
        w = synth.make("ridge_dense", n=40000, d=256, m=2560)
        args = (dev(w["A"]), dev(w["b"]))
        kw = dict(kind="ridge", param=w["param"], m=2560, precision="bf16")
    else:
        w = synth.make("ols_dense_ar1", n=60000, d=500, m=5000)
        args = (dev(w["A"]), dev(w["b"]))
        kw = dict(m=5000, precision="tf32")
    a = cuda_lib.IHS(*args, seed=3, cluster=True, **kw)
    b = cuda_lib.IHS(*args, seed=3, cluster=False, **kw)
    xa, ra = a.solve(iters=4)
    xb, rb = b.solve(iters=4)
    assert ra.status == 0 and rb.status == 0
    assert torch.equal(xa, xb)


@pytest.mark.parametrize("kind,s", [("dense64", 1), ("dense32", 4), ("csr64", 4), ("csr32", 8)])
def test_sketch_error_matches_oracle(cuda_lib, kind, s):
    """Sketch-quality experiment (App. B): the exact Gram A^T A and the
    empirical error ||A^T S^T S A - A^T A||_F / ||A^T A||_F of the sketches of
    counters t = 0..3 agree with the oracle's (FP64 sketch and Gram)."""
    if kind.startswith("dense"):
        w = synth.make("ols_dense_fp64", n=6000, d=40, m=400)
        Ah = w["A"] if kind == "dense64" else w["A"].astype(np.float32)
        args = (dev(Ah), dev(w["b"]))
        Ao = Ah.astype(np.float64)
        kw = dict(m=400, s=s, precision="fp64")
    else:
        w = synth.make("lasso_csr_fp64", n=30000, d=60, m=600)
        val = w["val"] if kind == "csr64" else w["val"].astype(np.float32)
        args = ((dev(w["rowptr"]), dev(w["col"]), dev(val)), dev(w["b"]))
        Ao = O.CSR(w["n"], w["d"], w["rowptr"], w["col"], val.astype(np.float64))
        kw = dict(m=600, s=s, precision="fp64", shape=(w["n"], w["d"]))
    sv = cuda_lib.IHS(*args, seed=9, **kw)
    G = sv.exact_gram()
    Go = O.ata(Ao)
    assert np.abs(G.cpu().numpy() - Go).max() <= 1e-12 * np.abs(Go).max()
    for t in range(4):
        e = sv.sketch_error(t, G)
        eo = O.sketch_error(Ao, kw["m"], s, 9, t)
        assert abs(e - eo) <= 1e-10 * eo, (t, e, eo)


def _pen_lambda(C, b, frac):
    return frac * float(np.abs(C.rmatvec(b)).max())


def test_l1_penalty_step_matches_oracle_qp(cuda_lib):
    """One penalised-LASSO step (argmin 1/2 ||S A (x - x^t)||^2 - g^T (x - x^t)
    + lambda ||x||_1) on the GPU equals the oracle's exact solution on the same
    H and g; the solution is unique."""
    w, C = _csr_problem("lasso_csr_fp64", 40000, 60, 600)
    lam = _pen_lambda(C, w["b"], 0.05)
    solver = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]),
                          kind="l1pen", param=lam, m=600, s=4, seed=0, precision="fp64",
                          shape=(w["n"], w["d"]))
    x = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
    xo = np.zeros(w["d"])
    for t in range(4):
        solver.sketch(t)
        SA, H, _ = solver.get_sketch()
        g = solver.gradient(x).cpu().numpy()
        solver.step(x)
        solver.sync()
        xq = O.l1_penalty_qp(H.cpu().numpy(), g, xo.copy(), lam)
        assert 0 < np.count_nonzero(xq) < w["d"]
        xo = xq
        assert rel(x.cpu().numpy(), xq) < 1e-11, t
        x.copy_(dev(xq))


def test_ihs_lasso_penalty_plain_matches_oracle_every_iteration(cuda_lib):
    """Penalised LASSO, CSR FP64 data, SJLT s = 4: every GPU iterate within
    1e-11 of the oracle's (A-seminorm, relative to x_OPT), and 1e-10 of x_OPT
    after 25 iterations."""
    w, C = _csr_problem("lasso_csr_fp64", 100000, 200, 2000)
    lam = _pen_lambda(C, w["b"], 0.02)
    G = C.gram()
    xo = O.x_opt_l1_penalty(C, w["b"], lam)
    assert 0 < np.count_nonzero(xo) < w["d"]
    xs = O.ihs(C, w["b"], O.L1_PENALTY, lam, 2000, 4, 0, 25)
    solver = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]),
                          kind="l1pen", param=lam, m=2000, s=4, seed=0, precision="fp64",
                          shape=(w["n"], w["d"]))
    x = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
    nrm = np.sqrt(xo @ G @ xo)
    for t in range(25):
        solver.sketch(t)
        solver.step(x)
        e = x.cpu().numpy() - xs[t + 1]
        assert np.sqrt(max(e @ G @ e, 0)) / nrm <= 1e-11, t
    solver.sync()
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


def test_ihs_lasso_penalty_mixed_lambda5(cuda_lib):
    """The experiments' setting, lambda = 5, mixed form on Zipf-column CSR FP32
    data (SJLT s = 8): 1e-10 of x_OPT."""
    w, C = _csr_problem("lasso_csr_zipf", 200000, 100, 1000)
    G = C.gram()
    xo = O.x_opt_l1_penalty(C, w["b"], 5.0)
    solver = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]),
                          kind="l1pen", param=5.0, m=1000, s=8, seed=0, precision="tf32",
                          shape=(w["n"], w["d"]))
    x, rep = solver.solve(iters=30)
    assert rep.status == 0
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


def test_l1_penalty_zero_solution(cuda_lib):
    """lambda >= ||A^T b||_inf: x_OPT = 0, reached exactly in one step."""
    w, C = _csr_problem("lasso_csr_fp64", 20000, 30, 300)
    lam = _pen_lambda(C, w["b"], 1.01)
    solver = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]),
                          kind="l1pen", param=lam, m=300, s=1, seed=0, precision="fp64",
                          shape=(w["n"], w["d"]))
    x, rep = solver.solve(iters=2)
    assert rep.status == 0
    assert torch.count_nonzero(x).item() == 0


@pytest.mark.parametrize("precision", ["fp64", "tf32"])
def test_ihs_lasso_penalty_large_support(cuda_lib, precision):
    """lambda = 5 on 100,000 x 200 CSR data: the solution keeps most indices
    (the active-set pass over the small zero set handles these faces).
    Plain form: every iterate within 1e-11 of the oracle's for 28 iterations;
    both forms reach 1e-10 of x_OPT (the rate here is about 0.35 per step)."""
    w, C = _csr_problem("lasso_csr_fp64", 100000, 200, 2000)
    val = w["val"] if precision == "fp64" else w["val"].astype(np.float32)
    # the mixed form solves the problem of the FP32-rounded data, promoted exactly
    C = O.CSR(w["n"], w["d"], w["rowptr"], w["col"], val.astype(np.float64))
    lam = 5.0
    G = C.gram()
    xo = O.x_opt_l1_penalty(C, w["b"], lam)
    assert 0.8 * w["d"] < np.count_nonzero(xo) < w["d"]
    solver = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(val)), dev(w["b"]),
                          kind="l1pen", param=lam, m=2000, s=4, seed=0, precision=precision,
                          shape=(w["n"], w["d"]))
    if precision == "fp64":
        xs = O.ihs(C, w["b"], O.L1_PENALTY, lam, 2000, 4, 0, 28)
        x = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
        nrm = np.sqrt(xo @ G @ xo)
        for t in range(28):
            solver.sketch(t)
            solver.step(x)
            e = x.cpu().numpy() - xs[t + 1]
            assert np.sqrt(max(e @ G @ e, 0)) / nrm <= 1e-11, t
        solver.sync()
    else:
        x, rep = solver.solve(iters=30)
        assert rep.status == 0
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


@pytest.mark.parametrize("n,d,m", [(1, 3, 4), (4096, 40, 400), (5000, 33, 300), (100000, 64, 640)])
def test_srht_sketch_matches_oracle(cuda_lib, n, d, m):
    """SRHT (Sec. 2, S = m^{-1/2} P H D): the draw and the raw P H D A equal the
    oracle's -- bit for bit in FP64 (the transform runs the stages in the
    definition's order), to FP32 accumulation in the mixed form; the Gram
    scale is 1/m.  Sizes cover n = 1, a power of two, zero padding, several
    passes of the transform and d not a multiple of 32."""
    rng = np.random.default_rng(n + d)
    A = rng.standard_normal((n, d))
    b = rng.standard_normal(n)
    rows, sign = O.srht_draw(4, 2, m, n)
    want = O.srht_sketch_fast(A, m, rows, sign)
    if n * m * d <= 4e8:
        assert np.allclose(want, O.srht_sketch(A, m, rows, sign), rtol=0, atol=1e-10 * np.abs(want).max())
    sv = cuda_lib.IHS(dev(A), dev(b), m=m, seed=4, precision="fp64", sketch="srht")
    sv.sketch(2)
    SA, H, scale = sv.get_sketch()
    assert scale == 1.0 / m
    assert np.array_equal(SA.cpu().numpy(), want)
    Hn = H.cpu().numpy()
    Ho = O.gram(want, 1.0 / m)
    assert np.abs(Hn - Ho).max() <= 1e-12 * np.abs(Ho).max()
    A32 = A.astype(np.float32)
    want32 = O.srht_sketch_fast(A32.astype(np.float64), m, rows, sign)
    sv32 = cuda_lib.IHS(dev(A32), dev(b), m=m, seed=4, precision="tf32", sketch="srht")
    sv32.sketch(2)
    SA32, _, _ = sv32.get_sketch()
    tol = 1e-6 * np.sqrt(O.srht_n2(n)) * np.abs(A32).max() * 4
    assert np.abs(SA32.cpu().numpy() - want32).max() <= tol


def test_ihs_srht_plain_matches_oracle_every_iteration(cuda_lib):
    """IHS with the SRHT on the 20000 x 50 FP64 OLS workload (m = 500): every
    GPU iterate within 1e-12 of the oracle's; 25 iterations reach 1e-10."""
    w = synth.make("ols_dense_fp64")
    A, b = w["A"], w["b"]
    xo = O.x_opt_ols_qr(A, b)
    G = A.T @ A
    xs = O.ihs(A, b, O.OLS, 0.0, 500, 1, 0, 25, sketch_kind="srht")
    sv = cuda_lib.IHS(dev(A), dev(b), m=500, seed=0, precision="fp64", sketch="srht")
    x = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
    nrm = np.sqrt(xo @ G @ xo)
    for t in range(25):
        sv.solve(x, t0=t, iters=1)
        e = x.cpu().numpy() - xs[t + 1]
        assert np.sqrt(max(e @ G @ e, 0.0)) / nrm <= 1e-12, t
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


def test_ihs_srht_mixed_reaches_1e10(cuda_lib):
    """Mixed form with the SRHT on AR(1) FP32 data reaches 1e-10 of x_OPT."""
    w = synth.make("ols_dense_ar1", n=100000, d=96, m=960)
    A64 = w["A"].astype(np.float64)
    xo = O.x_opt_ols_normal(A64, w["b"])
    G = A64.T @ A64
    sv = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), m=960, seed=0, precision="tf32", sketch="srht")
    x, rep = sv.solve(iters=30)
    assert rep.status == 0
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


def test_srht_rejects_sparse_and_sjlt(cuda_lib):
    w = synth.make("lasso_csr_fp64", n=1000, d=10, m=100)
    with pytest.raises(cuda_lib.IHSError) as e:
        cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]), m=100,
                     shape=(w["n"], w["d"]), sketch="srht")
    assert e.value.status == 8
    A = np.random.default_rng(0).standard_normal((100, 5))
    with pytest.raises(cuda_lib.IHSError) as e:
        cuda_lib.IHS(dev(A), dev(A[:, 0].copy()), m=40, s=4, sketch="srht")
    assert e.value.status == 1


@pytest.mark.parametrize("n,d,m", [(3000, 40, 200), (700000, 8, 200)])
def test_gauss_sketch_matches_oracle(cuda_lib, n, d, m):
    """Gaussian sketch (Sec. 2, S = G / sqrt(m)): the raw G A equals the
    oracle's to FP64 rounding in the plain form and to TF32 input rounding in
    the mixed form; the Gram scale is 1/m.  The second size spans several
    generated column chunks of G and a ragged last chunk."""
    rng = np.random.default_rng(n + d)
    A = rng.standard_normal((n, d))
    b = rng.standard_normal(n)
    want = O.gauss_sketch(A, m, 6, 1)
    sv = cuda_lib.IHS(dev(A), dev(b), m=m, seed=6, precision="fp64", sketch="gaussian")
    sv.sketch(1)
    SA, H, scale = sv.get_sketch()
    assert scale == 1.0 / m
    assert np.abs(SA.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()
    A32 = A.astype(np.float32)
    want32 = O.gauss_sketch(A32.astype(np.float64), m, 6, 1)
    sv32 = cuda_lib.IHS(dev(A32), dev(b), m=m, seed=6, precision="tf32", sketch="gaussian")
    sv32.sketch(1)
    SA32, _, _ = sv32.get_sketch()
    err = np.linalg.norm(SA32.cpu().numpy() - want32) / np.linalg.norm(want32)
    assert err < 2e-3


def test_ihs_gaussian_plain_matches_oracle_every_iteration(cuda_lib):
    """IHS with the Gaussian sketch on the 20000 x 50 FP64 OLS workload: every
    GPU iterate within 1e-12 of the oracle's."""
    w = synth.make("ols_dense_fp64")
    A, b = w["A"], w["b"]
    xo = O.x_opt_ols_qr(A, b)
    G = A.T @ A
    xs = O.ihs(A, b, O.OLS, 0.0, 500, 1, 0, 10, sketch_kind="gaussian")
    sv = cuda_lib.IHS(dev(A), dev(b), m=500, seed=0, precision="fp64", sketch="gaussian")
    x = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
    nrm = np.sqrt(xo @ G @ xo)
    for t in range(10):
        sv.solve(x, t0=t, iters=1)
        e = x.cpu().numpy() - xs[t + 1]
        assert np.sqrt(max(e @ G @ e, 0.0)) / nrm <= 1e-12, t


def test_ihs_gaussian_mixed_reaches_1e10(cuda_lib):
    """Mixed form with the Gaussian sketch (TF32 GEMM) reaches 1e-10."""
    w = synth.make("ols_dense_ar1", n=100000, d=96, m=960)
    A64 = w["A"].astype(np.float64)
    xo = O.x_opt_ols_normal(A64, w["b"])
    G = A64.T @ A64
    sv = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), m=960, seed=0, precision="tf32", sketch="gaussian")
    x, rep = sv.solve(iters=30)
    assert rep.status == 0
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


def test_ihs_l2_ball_plain_matches_oracle_every_iteration(cuda_lib):
    """p = 2 ball (R = ||x_OLS|| / 2, the constraint active), 20000 x 50 FP64
    OLS data: every GPU iterate within 1e-11 of the oracle's (whose subproblem
    solver is the secular equation on H's eigenbasis, a different route),
    1e-10 of x_OPT after 30 iterations."""
    w = synth.make("ols_dense_fp64")
    A, b = w["A"], w["b"]
    R = 0.5 * np.linalg.norm(O.x_opt_ols_qr(A, b))
    xo = O.x_opt_l2(A, b, R)
    G = A.T @ A
    xs = O.ihs(A, b, O.L2_BALL, R, 500, 1, 0, 30)
    sv = cuda_lib.IHS(dev(A), dev(b), kind="l2", param=R, m=500, seed=0, precision="fp64")
    x = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
    nrm = np.sqrt(xo @ G @ xo)
    for t in range(30):
        sv.solve(x, t0=t, iters=1)
        e = x.cpu().numpy() - xs[t + 1]
        assert np.sqrt(max(e @ G @ e, 0.0)) / nrm <= 1e-11, t
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10
    assert np.linalg.norm(x.cpu().numpy()) <= R * (1 + 1e-12)


@pytest.mark.parametrize("frac", [0.3, 2.0])
def test_ihs_l2_ball_mixed_reaches_1e10(cuda_lib, frac):
    """Mixed form (FP32 factor of H + mu I, FP64-refined solves) on AR(1) FP32
    data reaches 1e-10 of x_OPT, with the ball active (0.3) and inactive (2.0)."""
    w = synth.make("ols_dense_ar1", n=100000, d=96, m=960)
    A64 = w["A"].astype(np.float64)
    R = frac * np.linalg.norm(O.x_opt_ols_normal(A64, w["b"]))
    xo = O.x_opt_l2(A64, w["b"], R)
    G = A64.T @ A64
    sv = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), kind="l2", param=R, m=960, seed=0,
                      precision="tf32")
    x, rep = sv.solve(iters=30)
    assert rep.status == 0
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


def test_ihs_l2_ball_csr(cuda_lib):
    """p = 2 ball over CSR data with an SJLT (s = 4), plain form: 1e-10 of x_OPT."""
    w, C = _csr_problem("lasso_csr_fp64", 100000, 200, 2000)
    xols = O.x_opt_ols_normal(C, w["b"])
    R = 0.4 * np.linalg.norm(xols)
    G = C.gram()
    xo = O.l2_ball_qp(G, C.rmatvec(w["b"]), np.zeros(w["d"]), R)
    sv = cuda_lib.IHS((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]), kind="l2",
                      param=R, m=2000, s=4, seed=0, precision="fp64", shape=(w["n"], w["d"]))
    x, rep = sv.solve(iters=30)
    assert rep.status == 0
    assert O.err_A(x.cpu().numpy(), xo, G) < 1e-10


def test_contexts_reuse_pool_memory_and_trim(cuda_lib):
    """Workspaces come from the library's pool: creating and destroying
    contexts in a loop gives the same results each time, and trimming the
    pool between them changes nothing but the cached memory."""
    w = synth.make("ols_dense_fp64", n=5000, d=30, m=300)
    A, b = dev(w["A"]), dev(w["b"])
    xs = []
    for k in range(4):
        sv = cuda_lib.IHS(A, b, m=300, seed=2, precision="fp64")
        x, rep = sv.solve(iters=5)
        assert rep.status == 0
        xs.append(x.cpu().numpy())
        sv.close()
        if k == 1:
            cuda_lib.trim_memory()
    for x in xs[1:]:
        assert np.array_equal(x, xs[0])


@pytest.mark.parametrize("kind", ["l1", "l1pen"])
def test_l1_contexts_after_poisoned_pool_memory(cuda_lib, kind):
    """The l1-ball and penalised steps read no workspace before writing it:
    after contexts of the same shape whose data hold NaN (so every workspace
    they touched, in the library's pool and in shared memory, is left full of
    NaN) are destroyed, a fresh context on clean data repeats the iterates of
    a context created on a trimmed pool bit for bit.  (The penalised face
    solve once read its border direction, which only the ball form writes,
    multiplied by zero: 0 * NaN poisoned the step.)"""
    w, C = _csr_problem("lasso_csr_fp64", 60000, 120, 1200)
    param = w["param"] if kind == "l1" else _pen_lambda(C, w["b"], 0.02)
    rp, col, b = dev(w["rowptr"]), dev(w["col"]), dev(w["b"])
    val = dev(w["val"])

    def run(values, iters=8, **kw):
        sv = cuda_lib.IHS((rp, col, values), b, kind=kind, param=param, m=1200, s=4, seed=0,
                          precision="fp64", shape=(w["n"], w["d"]), **kw)
        try:
            x, rep = sv.solve(iters=iters)
            out = (x.cpu().numpy(), rep.status)
        except cuda_lib.IHSError as e:
            out = (None, e.status)
        sv.close()
        return out

    cuda_lib.trim_memory()
    x_fresh, st = run(val)
    assert st == 0
    bad = val.clone()
    bad[::7] = float("nan")
    for k in ("l1", "l1pen"):
        sv = cuda_lib.IHS((rp, col, bad), b, kind=k, param=param, m=1200, s=4, seed=0,
                          precision="fp64", shape=(w["n"], w["d"]), qp_max_iter=300)
        with pytest.raises(cuda_lib.IHSError):
            sv.solve(iters=2)
        sv.close()
    x_again, st = run(val)
    assert st == 0
    assert np.array_equal(x_again, x_fresh)


def test_pivot_rsqrt_matches_cuda_rsqrt(cuda_lib):
    """The FP64 factor takes its pivots' reciprocal square roots by two
    Newton-Raphson steps from an FP32 seed.  Against CUDA's rsqrt and a
    long-double evaluation, on 200,000 values over exponents 2^-300..2^300
    (outside FP32's range the routine falls back to rsqrt), powers of two,
    and the ends of FP32's exponent range: within 2 ulp of both."""
    rng = np.random.default_rng(11)
    p = np.ldexp(1.0 + rng.random(200000), rng.integers(-300, 300, size=200000))
    edge = [1.0, 2.0, 4.0, 0.5, 3.0, 2.0 ** -126, 2.0 ** -125 * 1.5, 2.0 ** 127,
            2.0 ** 127 * 1.9999999, 2.0 ** 128, 2.0 ** -127, 1e-310, 1.7e308]
    p = np.concatenate([p, np.array(edge), 2.0 ** np.arange(-200, 200, dtype=np.float64)])
    out, ref = cuda_lib.selftest_rsqrt(torch.from_numpy(p).cuda())
    out, ref = out.cpu().numpy(), ref.cpu().numpy()
    ulp = np.spacing(np.abs(ref))
    assert np.all(np.abs(out - ref) <= 2 * ulp)
    exact = (1 / np.sqrt(p.astype(np.longdouble))).astype(np.longdouble)
    err = np.abs(out.astype(np.longdouble) - exact) / np.spacing(np.abs(exact).astype(np.float64))
    assert float(err.max()) <= 2.0


def test_bounded_wait_gives_up_and_the_context_stays_usable(cuda_lib):
    """Failure detection on the GPU without a fault: a grid barrier that can
    never complete (two CTAs waiting for three) gives up after its poll limit
    and reports IHS_ERR_TIMEOUT through the device status word; the GPU stays
    usable, and a solve afterwards matches the oracle."""
    assert cuda_lib.selftest_wait() == 7  # IHS_ERR_TIMEOUT
    assert cuda_lib.selftest_wait() == 7
    w = synth.make("ols_dense_fp64", n=5000, d=20, m=200)
    xs = O.ihs(w["A"], w["b"], O.OLS, 0.0, 200, 1, 0, 3)
    solver = cuda_lib.IHS(dev(w["A"]), dev(w["b"]), m=200, s=1, seed=0, precision="fp64")
    x, rep = solver.solve(iters=3)
    assert rep.status == 0
    assert np.abs(x.cpu().numpy() - xs[-1]).max() <= 1e-12 * np.abs(xs[-1]).max()


def test_graph_not_used_for_l2_ball_and_l1_penalty(cuda_lib):
    """The p = 2 ball (its step reads scalars on the host) and the l1 penalty
    (its one-CTA step kernels need to be issued ahead of the sketch chain)
    run on the streams even for a small A; the ball and OLS forms of the same
    data replay graphs."""
    w, C = _csr_problem("lasso_csr_fp64", 30000, 60, 600)
    args = ((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]))
    base = dict(m=600, s=4, precision="fp64", shape=(w["n"], w["d"]))
    for kind, param, graph in (("l1pen", 1.0, 0), ("l2", 0.5, 0), ("l1", w["param"], 1)):
        sv = cuda_lib.IHS(*args, kind=kind, param=param, **base)
        for _ in range(2):
            _, rep = sv.solve(iters=3)
            assert rep.status == 0 and rep.graph == graph, (kind, rep.graph)


@pytest.mark.parametrize("case", ["ols_fp64", "l1_csr_fp64", "ols_tf32_lookahead", "ridge_fp64"])
def test_graph_solve_matches_stream_solve(cuda_lib, case):
    """Launch-bound contexts (A up to 128 MB) replay ihs_solve as a CUDA
    graph, captured on the first call with a given (t0, iters).  The graph
    holds the same kernels in the same order as the streams, so the iterates
    equal those of a context with graphs off bit for bit.  This holds on the
    capture, on a replay with another iterate buffer, and across a resume
    (4 + 6 iterations against 10)."""
    if case == "l1_csr_fp64":
        w, C = _csr_problem("lasso_csr_fp64", 60000, 120, 1200)
        args = ((dev(w["rowptr"]), dev(w["col"]), dev(w["val"])), dev(w["b"]))
        kw = dict(kind="l1", param=w["param"], m=1200, s=4, precision="fp64",
                  shape=(w["n"], w["d"]))
        d = w["d"]
    else:
        name = "ridge_dense" if case == "ridge_fp64" else "ols_dense_fp64"
        w = synth.make(name, n=20000, d=48, m=480)
        A = w["A"].astype(np.float32 if case == "ols_tf32_lookahead" else np.float64)
        args = (dev(A), dev(w["b"]))
        kw = dict(m=480, precision="tf32" if case == "ols_tf32_lookahead" else "fp64")
        if case == "ridge_fp64":
            kw.update(kind="ridge", param=w["param"])
        d = 48
    gr = cuda_lib.IHS(*args, **kw)
    st = cuda_lib.IHS(*args, graph=False, **kw)
    x_s, r_s = st.solve(iters=10)
    assert r_s.graph == 0
    for trial in range(2):  # capture, then replay into a fresh buffer
        x_g = torch.zeros(d, dtype=torch.float64, device="cuda")
        _, r_g = gr.solve(x_g, iters=10)
        assert r_g.status == 0 and r_g.graph == 1, trial
        assert torch.equal(x_g, x_s), trial
    x4, r4 = gr.solve(iters=4)
    x10, r10 = gr.solve(x4, t0=4, iters=6)
    assert r4.graph == 1 and r10.graph == 1
    if case == "ols_tf32_lookahead":
        # the look-ahead pipeline's last pass of a solve walks another sort's
        # row order, so a resumed run agrees to the gradient's rounding
        assert float((x10 - x_s).abs().max()) <= 1e-11 * float(x_s.abs().max())
    else:
        assert torch.equal(x10, x_s)
    S1, H1, _ = gr.get_sketch()
    S2, H2, _ = st.get_sketch()
    assert torch.equal(S1, S2) and torch.equal(H1, H2)
