"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics (no GPU).  Each test names what it pins and the passage it
follows."""
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- hash ----
def test_splitmix64_published_outputs():
    """The sketch's generator is SplitMix64 from its published definition."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if l[0] != "#"]
    assert len(rows) == 8
    for st, j, v in rows:
        assert O.sm64_at(int(st), int(j)) == int(v)


@pytest.mark.parametrize("m,s", [(40, 1), (40, 4), (7, 7), (1, 1)])
def test_hash_shape_ranges(m, s):
    """Sec. 2: block k of an SJLT is a CountSketch of m/s rows, stacked row-wise."""
    n = 1000
    bucket, sign = O.hash_draw(3, 2, s, m, n)
    mb = m // s
    for k in range(s):
        assert bucket[k].min() >= k * mb and bucket[k].max() < (k + 1) * mb
    assert set(np.unique(sign)) <= {-1, 1}


def test_hash_rejects_bad_shape():
    """SJLT needs m/s integral (Sec. 2)."""
    with pytest.raises(ValueError):
        O.hash_draw(0, 0, 3, 10, 5)


def test_hash_uniform_and_balanced():
    """Sec. 2: h(i) uniform over the m rows, signs +-1 with probability 1/2.
    Chi-square over 64 buckets for 2^18 draws; sign fraction within 5 sigma."""
    n, m = 1 << 18, 64
    bucket, sign = O.hash_draw(11, 0, 1, m, n)
    cnt = np.bincount(bucket[0], minlength=m)
    e = n / m
    chi2 = ((cnt - e) ** 2 / e).sum()
    assert chi2 < 63 + 6 * np.sqrt(2 * 63)  # mean 63, sd sqrt(126)
    frac = (sign == 1).mean()
    assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(n)


def test_hash_independent_across_iterations_and_blocks():
    """A fresh sketch every iteration (App. A, iteration costs) and
    independent blocks for the SJLT: draws for different (t, k) agree on about
    1/mb of the rows, as independent uniform draws would."""
    n, m, s = 20000, 80, 4
    b0, _ = O.hash_draw(5, 0, s, m, n)
    b1, _ = O.hash_draw(5, 1, s, m, n)
    mb = m // s
    same_t = ((b0 % mb) == (b1 % mb)).mean()
    same_k = ((b0[0] % mb) == (b0[1] % mb)).mean()
    for v in (same_t, same_k):
        assert abs(v - 1 / mb) < 6 * np.sqrt(1 / mb / n)


def _pair_draws_independent(b, sg, mb):
    """For every block pair (2p, 2p + 1) of a draw over n rows: the buckets
    agree on 1/mb of the rows within 6 sigma, and no sign is correlated with
    the other sign or with either bucket's upper half (6 / sqrt(n))."""
    s, n = b.shape
    tol = 6 / np.sqrt(n)
    for p in range(s // 2):
        k0, k1 = 2 * p, 2 * p + 1
        u0, u1 = b[k0] - k0 * mb, b[k1] - k1 * mb
        if abs((u0 == u1).mean() - 1 / mb) >= 6 * np.sqrt(1 / mb / n):
            return False
        s0, s1 = sg[k0].astype(float), sg[k1].astype(float)
        h0, h1 = np.where(u0 >= mb // 2, 1.0, -1.0), np.where(u1 >= mb // 2, 1.0, -1.0)
        for a, c in ((s0, s1), (s0, h0), (s0, h1), (s1, h0), (s1, h1)):
            if abs(np.mean(a * c) - np.mean(a) * np.mean(c)) >= tol:
                return False
    return True


def test_hash_block_pair_halves_independent():
    """Blocks 2p and 2p + 1 of a row take the high and low halves of one
    SplitMix64 output (bucket by multiply-shift of the half, sign from bit 0
    of the other half; the paper names no generator).  They must still behave
    as independent draws: the two buckets agree on about 1/mb of the rows, and
    no sign is correlated with the other sign or with either bucket's upper
    half (a sign taken from the same bits as a bucket, or two blocks taken
    from one half, fails this)."""
    n, m, s = 40000, 96, 6
    mb = m // s
    b, sg = O.hash_draw(3, 1, s, m, n)
    assert _pair_draws_independent(b, sg, mb)
    # s = 1 keeps the high half and bit 0: the same draw as block 0 of any s
    b1, sg1 = O.hash_draw(3, 1, 1, mb, n)
    assert np.array_equal(b1[0], b[0]) and np.array_equal(sg1[0], sg[0])


def test_countsketch_rows_orthogonal_lemma():
    """Lemma (orthogonal rows): S S^T is diagonal with (S S^T)_ii = N_i, the
    number of nonzeros in row i; for CountSketch sum_i N_i = n."""
    n, m = 300, 16
    bucket, sign = O.hash_draw(1, 0, 1, m, n)
    S = O.sketch_matrix(m, 1, bucket, sign)
    SS = S @ S.T
    assert np.array_equal(SS, np.diag(np.diag(SS)))
    assert np.array_equal(np.diag(SS), np.bincount(bucket[0], minlength=m).astype(float))
    assert np.diag(SS).sum() == n


def test_expected_SST_and_STS():
    """Lemmas of App. A: E[S S^T] = (n/m) I_m and E[S^T S] = I_n; for an SJLT
    normalised by its s nonzeros per column, diag(S^T S) = 1 on every draw."""
    n, m, trials = 48, 8, 4000
    acc_sst = np.zeros((m, m))
    acc_sts = np.zeros((n, n))
    for s in (1, 4):
        acc_sst[:] = 0
        acc_sts[:] = 0
        for t in range(trials):
            bucket, sign = O.hash_draw(2024, t, s, m, n)
            S = O.sketch_matrix(m, s, bucket, sign)
            STS = S.T @ S
            assert np.array_equal(np.diag(STS), np.ones(n))  # exact: s * (1/sqrt(s))^2 = 1 for s = 1, 4
            acc_sts += STS
            acc_sst += S @ S.T
        mean_sts = acc_sts / trials
        off = mean_sts[~np.eye(n, dtype=bool)]
        # off-diagonal entries: each draw contributes +-1/s w.p. 1/mb per block -> sd <= 1/sqrt(trials*mb)
        assert np.abs(off).max() < 6 / np.sqrt(trials * (m // s))
        assert abs(off.mean()) < 4 / np.sqrt(trials * (m // s) * off.size)
        mean_sst = acc_sst / trials
        assert np.allclose(np.diag(mean_sst), n / m, rtol=0.1)
        assert np.abs(mean_sst[~np.eye(m, dtype=bool)]).max() < 0.15


# -------------------------------------------------------------- sketch ----
@pytest.mark.parametrize("s", [1, 2, 4])
def test_sketch_equals_materialised_product(s):
    """The streaming pass of Sec. 2 equals S A with S as a dense matrix."""
    n, d, m = 333, 7, 24
    rng = np.random.default_rng(0)
    A = rng.standard_normal((n, d))
    bucket, sign = O.hash_draw(9, 4, s, m, n)
    S = O.sketch_matrix(m, s, bucket, sign) * np.sqrt(s)  # raw +-1 entries
    SA = O.sketch(A, m, s, bucket, sign)
    assert np.allclose(SA, S @ A, rtol=0, atol=1e-12)
    # CSR path on the same values
    rowptr, col, val = synth.csr_uniform(n, d, 3, 1, np.float64)
    C = O.CSR(n, d, rowptr, col, val)
    assert np.allclose(O.sketch(C, m, s, bucket, sign), S @ C.todense(), rtol=0, atol=1e-12)


def test_sketch_adjoint_dot_product():
    """<S A, G> = <A, S^T G> for the normalised sketch (adjoint of a linear map)."""
    n, d, m, s = 500, 6, 32, 4
    rng = np.random.default_rng(1)
    A = rng.standard_normal((n, d))
    G = rng.standard_normal((m, d))
    bucket, sign = O.hash_draw(1, 0, s, m, n)
    SA = O.sketch(A, m, s, bucket, sign) / np.sqrt(s)
    STG = O.sketch_adjoint(G, n, s, bucket, sign)
    assert abs((SA * G).sum() - (A * STG).sum()) < 1e-10 * np.abs(SA).sum()
    S = O.sketch_matrix(m, s, bucket, sign)
    assert np.allclose(STG, S.T @ G, atol=1e-13)


# ---------------------------------------------------------------- gram ----
def test_gram_against_matmul_and_expectation():
    """H = (1/s) (SA)^T SA + shift I; averaged over draws it tends to A^T A
    (E[S^T S] = I, App. A), error ~ 1/sqrt(trials)."""
    n, d, m, s = 400, 5, 40, 2
    rng = np.random.default_rng(2)
    A = rng.standard_normal((n, d))
    acc = np.zeros((d, d))
    trials = 400
    for t in range(trials):
        bucket, sign = O.hash_draw(77, t, s, m, n)
        SA = O.sketch(A, m, s, bucket, sign)
        H = O.gram(SA, 1.0 / s, 0.25)
        assert np.allclose(H, SA.T @ SA / s + 0.25 * np.eye(d), rtol=1e-13, atol=1e-12)
        acc += H - 0.25 * np.eye(d)
    G = A.T @ A
    rel = np.linalg.norm(acc / trials - G) / np.linalg.norm(G)
    assert rel < 3.0 * np.sqrt(d / m) / np.sqrt(trials) * 3


# ------------------------------------------------------------ gradient ----
def test_resid_grad_is_minus_gradient():
    """g = A^T (b - A x) = -grad f(x) for f = 1/2 ||Ax - b||^2 (Eq. 1):
    central differences in FP64; r = b - A x."""
    n, d = 200, 6
    rng = np.random.default_rng(3)
    A = rng.standard_normal((n, d))
    b = rng.standard_normal(n)
    x = rng.standard_normal(d)
    r, g = O.resid_grad(A, b, x, want_r=True)
    assert np.allclose(r, b - A @ x, rtol=0, atol=1e-12)
    f = lambda z: 0.5 * np.sum((A @ z - b) ** 2)
    h = 1e-5
    fd = np.array([(f(x + h * e) - f(x - h * e)) / (2 * h) for e in np.eye(d)])
    assert np.allclose(-g, fd, rtol=1e-7, atol=1e-6)
    rowptr, col, val = synth.csr_uniform(n, d, 2, 4, np.float64)
    C = O.CSR(n, d, rowptr, col, val)
    Ad = C.todense()
    r2, g2 = O.resid_grad(C, b, x, want_r=True)
    assert np.allclose(r2, b - Ad @ x, atol=1e-12) and np.allclose(g2, Ad.T @ (b - Ad @ x), atol=1e-11)


def test_gradient_vanishes_at_xopt():
    """At x_OPT of OLS the gradient is zero up to rounding."""
    w = synth.make("ols_dense_fp64", n=4000)
    xo = O.x_opt_ols_qr(w["A"], w["b"])
    g = O.resid_grad(w["A"], w["b"], xo)
    assert np.linalg.norm(g) <= 1e-12 * np.linalg.norm(w["A"]) * np.linalg.norm(w["b"])


# ------------------------------------------------------------ OLS step ----
def test_identity_sketch_gives_xopt_in_one_step():
    """Eq. 2 with C = R^d and S = I (m = n, h(i) = i) is a Newton step on a
    quadratic: x^1 = x^0 + (A^T A)^{-1} A^T (b - A x^0) = x_OPT."""
    n, d = 300, 8
    rng = np.random.default_rng(4)
    A = rng.standard_normal((n, d))
    b = rng.standard_normal(n)
    bucket = np.arange(n, dtype=np.int32)[None, :]
    sign = np.ones((1, n), np.int8)
    SA = O.sketch(A, n, 1, bucket, sign)
    H = O.gram(SA, 1.0)
    x0 = rng.standard_normal(d)
    x1 = x0 + O.chol_solve(H, O.resid_grad(A, b, x0))
    xl = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.allclose(x1, xl, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------- x_OPT ----
def test_xopt_solvers_agree():
    """Householder QR, refined normal equations and LAPACK lstsq give the
    same x_OPT on a 20000 x 50 problem."""
    w = synth.make("ols_dense_fp64")
    xq = O.x_opt_ols_qr(w["A"], w["b"])
    xn = O.x_opt_ols_normal(w["A"], w["b"])
    xl = np.linalg.lstsq(w["A"], w["b"], rcond=None)[0]
    G = w["A"].T @ w["A"]
    assert O.err_A(xq, xl, G) < 1e-13 and O.err_A(xn, xl, G) < 1e-13


def test_err_metric_definition():
    """||v||_A = n^{-1/2} ||A v|| (Sec. 1); err_A is the ratio of two of them."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((50, 4))
    x, xo = rng.standard_normal(4), rng.standard_normal(4)
    nA = lambda v: np.linalg.norm(A @ v) / np.sqrt(50)
    assert abs(O.err_A(x, xo, A.T @ A) - nA(x - xo) / nA(xo)) < 1e-14


# ---------------------------------------------------------- l1-ball QP ----
@pytest.mark.parametrize("seed", range(12))
def test_l1_qp_against_bruteforce(seed):
    """The exact l1-ball subproblem of Eq. 2 (Sec. 3: 'solved exactly') equals
    brute force over every face of the ball, d <= 6."""
    rng = np.random.default_rng(100 + seed)
    d = 2 + seed % 5
    M = rng.standard_normal((3 * d, d))
    H = M.T @ M + 0.1 * np.eye(d)
    g = rng.standard_normal(d) * 3
    xt = rng.standard_normal(d) * 0.3
    R = 0.2 + rng.random() * 1.5
    x = O.l1_ball_qp(H, g, xt, R)
    xb = O.l1_ball_qp_bruteforce(H, g, xt, R)
    assert np.allclose(x, xb, rtol=1e-10, atol=1e-12)
    assert np.abs(x).sum() <= R * (1 + 1e-12)
    assert O.l1_kkt_residual(H, g, xt, R, x) < 1e-13


def test_l1_projection_properties():
    """Projection onto the l1 ball (Duchi et al. 2008): feasible, idempotent,
    on the boundary when the input is outside, and the variational
    inequality <v - p, y - p> <= 0 for feasible y."""
    assert _l1_projection_pins_hold(O.project_l1_ball)


def _l1_projection_pins_hold(proj):
    """The properties above for 50 seeded (v, R), each with 5 feasible y."""
    rng = np.random.default_rng(6)
    for _ in range(50):
        v = rng.standard_normal(9) * 3
        R = rng.random() * 4 + 0.1
        p = proj(v, R)
        if np.abs(p).sum() > R * (1 + 1e-12) or not np.allclose(proj(p, R), p):
            return False
        if np.abs(v).sum() > R and abs(np.abs(p).sum() - R) >= 1e-12:
            return False
        for _ in range(5):
            y = proj(rng.standard_normal(9) * 5, R)
            if (v - p) @ (y - p) > 1e-10:
                return False
    return True


def test_l1_qp_kkt_at_dimension_200():
    """The QP at the lasso workload's dimension reaches an exact KKT point."""
    rng = np.random.default_rng(7)
    d = 200
    M = rng.standard_normal((2000, d))
    H = M.T @ M / 2000 * 1000
    xs = synth.sparse_truth(d, 20, 1)
    g = H @ xs * 1.0 + rng.standard_normal(d)
    R = 0.5 * np.abs(xs).sum()
    x = O.l1_ball_qp(H, g, np.zeros(d), R)
    assert O.l1_kkt_residual(H, g, np.zeros(d), R, x) < 1e-12


# ------------------------------------------------------- IHS iteration ----
def _gaussian_rate(m, d):
    """E||e'||^2/||e||^2 for a Gaussian sketch (inverse-Wishart moments); a
    reference value for the per-step contraction, derived here, not printed
    in the paper."""
    return np.sqrt(1 - 2 * m / (m - d - 1) + m * m * (m - 1) / ((m - d) * (m - d - 1) * (m - d - 3)))


def test_ihs_ols_converges_geometrically():
    """Thm. 2.2: the error in the A-seminorm contracts by a factor eps0 < 1/2
    per step, reaching 1e-10 in Theta(log 1/eps) steps.  20000 x 50,
    CountSketch m = 10 d."""
    w = synth.make("ols_dense_fp64")
    A, b = w["A"], w["b"]
    G = A.T @ A
    xo = O.x_opt_ols_qr(A, b)
    xs = O.ihs(A, b, O.OLS, 0.0, 500, 1, 0, 30)
    err = np.array([O.err_A(x, xo, G) for x in xs])
    assert err[0] == 1.0
    ratios = err[1:20] / err[:19]
    med = np.median(ratios)
    ref = _gaussian_rate(500, 50)
    assert med < 0.5 and 0.7 * ref < med < 1.3 * ref
    assert err[30] <= 1e-10


def test_ihs_lasso_converges_to_xopt():
    """Eq. 2 over the l1 ball converges to the constrained x_OPT (Thm. 2.2),
    here on a 20000 x 200 CSR lasso with SJLT s = 4, m = 2000."""
    w = synth.make("lasso_csr_fp64", n=20000)
    C = O.CSR(w["n"], w["d"], w["rowptr"], w["col"], w["val"])
    xo = O.x_opt_l1(C, w["b"], w["param"])
    G = C.gram()
    xs = O.ihs(C, w["b"], O.L1_BALL, w["param"], 2000, 4, 0, 25)
    err = [O.err_A(x, xo, G) for x in xs]
    assert err[-1] < 1e-10
    assert np.abs(xs[-1]).sum() <= w["param"] * (1 + 1e-12)


def test_ihs_ridge_converges():
    """Ridge (sketched Hessian plus lam I, exact gradient minus lam x)
    converges to (A^T A + lam I)^{-1} A^T b."""
    w = synth.make("ridge_dense", n=8192, d=32, m=320)
    A = w["A"].astype(np.float64)
    xo = O.x_opt_ols_normal(A, w["b"], lam=w["param"])
    xs = O.ihs(A, w["b"], O.RIDGE, w["param"], 320, 1, 0, 30)
    assert O.err_A(xs[-1], xo, A.T @ A) < 1e-10


def test_resume_is_exact():
    """Counter-based sketches make a resumed run identical: 10 steps equal
    4 steps then 6 more from x^4 starting at counter 4."""
    w = synth.make("ols_dense_fp64", n=3000, d=10, m=100)
    xs = O.ihs(w["A"], w["b"], O.OLS, 0.0, 100, 1, 3, 10)
    ys = O.ihs(w["A"], w["b"], O.OLS, 0.0, 100, 1, 3, 6, x0=xs[4], t0=4)
    assert np.array_equal(xs[10], ys[6])


# ------------------------------------------------------------- adjoint ----
def test_ridge_adjoint_against_central_differences():
    """dL/db = A v and dL/dA = r v^T - (A v) x^T for L = ||x(A, b) - x_t||^2,
    x = (A^T A + lam I)^{-1} A^T b; central differences h = 1e-6 in FP64."""
    A, b, lam, dLdx, fd_b, fd_A = _ridge_fd_case()
    x, dLdb, dLdA = O.ridge_adjoint(A, b, lam, dLdx)
    assert np.linalg.norm(fd_b - dLdb) <= 1e-6 * np.linalg.norm(dLdb)
    assert np.linalg.norm(fd_A - dLdA) <= 1e-6 * np.linalg.norm(dLdA)


def _ridge_fd_case():
    """A 60 x 5 ridge problem, dL/dx at its solution for L = ||x - x_t||^2,
    and central differences (h = 1e-6) of L in every entry of b and of A."""
    rng = np.random.default_rng(8)
    n, d, lam = 60, 5, 1e-3
    A = rng.standard_normal((n, d))
    b = rng.standard_normal(n)
    xt = rng.standard_normal(d)

    def loss(A_, b_):
        x = np.linalg.solve(A_.T @ A_ + lam * np.eye(d), A_.T @ b_)
        return np.sum((x - xt) ** 2)

    dLdx = 2 * (np.linalg.solve(A.T @ A + lam * np.eye(d), A.T @ b) - xt)
    h = 1e-6
    fd_b = np.array([(loss(A, b + h * e) - loss(A, b - h * e)) / (2 * h) for e in np.eye(n)])
    fd_A = np.zeros_like(A)
    for i in range(n):
        for j in range(d):
            E = np.zeros_like(A)
            E[i, j] = h
            fd_A[i, j] = (loss(A + E, b) - loss(A - E, b)) / (2 * h)
    return A, b, lam, dLdx, fd_b, fd_A


# ----------------------------------------------- planted-mistake checks ----
def test_pins_catch_planted_mistakes(monkeypatch):
    """A dropped sign, a transposed Gram or an off-by-one gradient term in the
    oracle each fails one of the pins above (mistakes planted on the CPU)."""
    n, d, m = 200, 5, 16
    rng = np.random.default_rng(9)
    A = rng.standard_normal((n, d))
    b = rng.standard_normal(n)
    bucket, sign = O.hash_draw(9, 4, 1, m, n)
    S = O.sketch_matrix(m, 1, bucket, sign)
    # dropped sign
    SA_bad = O.sketch(A, m, 1, bucket, np.ones_like(sign))
    assert not np.allclose(SA_bad, S @ A)
    # gradient missing the residual's b term fails the finite-difference pin
    x = rng.standard_normal(d)
    g_bad = -(A.T @ (A @ x))
    f = lambda z: 0.5 * np.sum((A @ z - b) ** 2)
    fd = np.array([(f(x + 1e-5 * e) - f(x - 1e-5 * e)) / 2e-5 for e in np.eye(d)])
    assert not np.allclose(-g_bad, fd, rtol=1e-7, atol=1e-6)
    # a step with the wrong sign diverges instead of contracting
    H = O.gram(O.sketch(A, m, 1, bucket, sign), 1.0)
    x1 = x - O.chol_solve(H, O.resid_grad(A, b, x))
    xo = np.linalg.lstsq(A, b, rcond=None)[0]
    assert O.err_A(x1, xo, A.T @ A) > O.err_A(x, xo, A.T @ A)
    # penalised QP with the sign of the penalty term flipped in the face system
    # is caught by the brute-force pin
    G = A.T @ A
    gg = A.T @ b
    lam = 0.2 * np.abs(gg).max()
    good = O.l1_penalty_qp_bruteforce(G, gg, np.zeros(d), lam)
    monkeypatch.setattr(O, "_pen_face_solve",
                        lambda H_, c_, l_, S_, s_: np.linalg.solve(H_[np.ix_(S_, S_)], c_[S_] + l_ * s_))
    try:
        bad = O.l1_penalty_qp(G, gg, np.zeros(d), lam, max_rounds=3, inner=50)
    except RuntimeError:
        bad = None  # no face passed the acceptance test: caught
    assert bad is None or not np.allclose(bad, good)


def test_pair_pin_catches_shared_halves():
    """Planted on the CPU: block 2p + 1 drawn from the same half as block 2p,
    or every sign taken from the top bit of its own bucket, fails the
    block-pair independence pin."""
    n, m, s = 40000, 96, 6
    mb = m // s
    b, sg = O.hash_draw(3, 1, s, m, n)
    same = b.copy()
    for p in range(s // 2):
        same[2 * p + 1] = b[2 * p] + mb
    assert not _pair_draws_independent(same, sg, mb)
    own = np.stack([np.where(b[k] - k * mb >= mb // 2, -1, 1) for k in range(s)]).astype(np.int8)
    assert not _pair_draws_independent(b, own, mb)


def test_projection_pins_catch_an_off_by_one_threshold():
    """Planted on the CPU: the sort-based l1 projection with its threshold
    divided by rho instead of rho + 1 fails the projection pins."""
    def proj_bad(v, R):
        if np.abs(v).sum() <= R:
            return v.copy()
        u = np.sort(np.abs(v))[::-1]
        css = np.cumsum(u)
        rho = np.nonzero(u - (css - R) / np.arange(1, v.size + 1) > 0)[0][-1]
        theta = (css[rho] - R) / max(rho, 1)
        return np.sign(v) * np.maximum(np.abs(v) - theta, 0.0)

    assert not _l1_projection_pins_hold(proj_bad)


def test_srht_pins_catch_planted_mistakes():
    """Planted on the CPU: the SRHT without its diagonal D, and a fast
    transform whose butterfly writes (u + v, v - u), each fail the
    materialised-Hadamard pins."""
    from scipy.linalg import hadamard
    rng = np.random.default_rng(21)
    n, m = 100, 12
    A = rng.standard_normal((n, 3))
    rows, sign = O.srht_draw(3, 5, m, n)
    want = (hadamard(O.srht_n2(n))[rows][:, :n] * sign[None, :].astype(float)) @ A
    assert np.allclose(O.srht_sketch(A, m, rows, sign), want, rtol=0, atol=1e-12)
    assert not np.allclose(O.srht_sketch(A, m, rows, np.ones_like(sign)), want, rtol=0,
                           atol=1e-12)

    def fwht_reversed(X):
        Y = np.array(X, dtype=np.float64, copy=True)
        h = 1
        while h < Y.shape[0]:
            Y = Y.reshape(Y.shape[0] // (2 * h), 2, h, -1)
            u, v = Y[:, 0].copy(), Y[:, 1].copy()
            Y[:, 0], Y[:, 1] = u + v, v - u
            Y = Y.reshape(-1, Y.shape[-1])
            h *= 2
        return Y

    X = rng.standard_normal((256, 4))
    assert not np.allclose(fwht_reversed(X), hadamard(256) @ X, atol=1e-11)


def _sm64_np(state, j):
    """SplitMix64 output j (uint64 array) of the generator started at
    `state` (Steele, Lea & Flood 2014), vectorised for the planted draws."""
    z = np.uint64(state) + (j.astype(np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def test_gauss_pins_catch_planted_mistakes():
    """Planted on the CPU in a restatement of the oracle's Box-Muller draw
    (which first reproduces gauss_draw): a missing factor 2 under the root, a
    missing 2 pi in the angle, or one uniform for both factors, each fail the
    standard-normal pins."""
    seed, t, m, n = 5, 0, 200, 1000
    key = O.sm64_at(O.sm64_at(O.sm64_at(seed, 0), t), 2)
    assert int(_sm64_np(key, np.array([7], dtype=np.uint64))[0]) == O.sm64_at(key, 7)
    w = _sm64_np(key, np.arange(m * n, dtype=np.uint64))
    u1 = ((w >> np.uint64(32)).astype(np.float64) + 0.5) / 4294967296.0
    u2 = ((w & np.uint64(0xFFFFFFFF)).astype(np.float64) + 0.5) / 4294967296.0
    good = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    assert np.allclose(good, O.gauss_draw(seed, t, m, n).ravel(), rtol=0, atol=1e-12)
    assert _standard_normal_pins_hold(good)
    assert not _standard_normal_pins_hold(np.sqrt(-np.log(u1)) * np.cos(2.0 * np.pi * u2))
    assert not _standard_normal_pins_hold(np.sqrt(-2.0 * np.log(u1)) * np.cos(u2))
    assert not _standard_normal_pins_hold(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u1))


def test_l2_ball_pin_catches_a_transposed_eigenbasis(monkeypatch):
    """Planted on the CPU: the p = 2 ball solver using its eigenbasis
    transposed fails the KKT pin (d = 6, the ball constraint active)."""
    rng = np.random.default_rng(33)
    d = 6
    M = rng.standard_normal((10, d))
    H = M.T @ M + 0.1 * np.eye(d)
    xt = rng.standard_normal(d)
    g = 4 * rng.standard_normal(d)
    R = 0.5 * np.linalg.norm(np.linalg.solve(H, H @ xt + g))
    assert O.l2_ball_kkt_residual(H, g, xt, R, O.l2_ball_qp(H, g, xt, R)) < 1e-12
    eigh = np.linalg.eigh

    def eigh_transposed(a):
        lam, Q = eigh(a)
        return lam, Q.T

    monkeypatch.setattr(O.np.linalg, "eigh", eigh_transposed)
    assert O.l2_ball_kkt_residual(H, g, xt, R, O.l2_ball_qp(H, g, xt, R)) > 1e-6


def test_adjoint_pin_catches_planted_mistakes():
    """Planted on the CPU: dL/dA with the sign of its (A v) x^T term flipped,
    or v solved without the ridge shift lam I, fails the central-difference
    pin."""
    A, b, lam, dLdx, fd_b, fd_A = _ridge_fd_case()
    x, dLdb, dLdA = O.ridge_adjoint(A, b, lam, dLdx)
    flipped = dLdA + 2 * np.outer(dLdb, x)
    assert np.linalg.norm(fd_A - flipped) > 1e-6 * np.linalg.norm(flipped)
    v0 = np.linalg.solve(A.T @ A, dLdx)
    assert np.linalg.norm(fd_b - A @ v0) > 1e-6 * np.linalg.norm(A @ v0)


# --------------------------------------------------------------- synth ----
def test_synth_recipes():
    """Input recipes: exact nnz per row, distinct sorted columns, AR(1)
    correlation rho^|i-j|, Zipf column frequencies."""
    rowptr, col, val = synth.csr_uniform(5000, 200, 2, 0)
    assert np.all(np.diff(rowptr) == 2)
    c = col.reshape(-1, 2)
    assert np.all(c[:, 0] < c[:, 1])
    A = synth.dense_ar1(200000, 6, 0.5, 0)
    C = np.corrcoef(A.T.astype(np.float64))
    for k in range(1, 4):
        assert abs(C[0, k] - 0.5 ** k) < 0.01
    rowptr, col, val = synth.csr_zipf(100000, 1000, 5, 1.1, 0)
    c = col.reshape(-1, 5)
    assert np.all(np.diff(c, axis=1) > 0)
    freq = np.bincount(col, minlength=1000) / col.size
    # the hottest column holds roughly p_1 of the draws (rejection of repeats lowers it a little)
    p1 = synth.zipf_probs(1000, 1.1)[0]
    assert 0.6 * p1 < freq.max() < 1.05 * p1


@pytest.mark.parametrize("s", [1, 4])
def test_sketch_error_mean_matches_closed_form(s):
    """The mean of the squared empirical sketch error over independent draws
    matches E||A^T S^T S A - A^T A||_F^2 / ||A^T A||_F^2 = (||A||_F^4 +
    ||A^T A||_F^2 - 2 sum ||a_i||^4) / (m ||A^T A||_F^2) (derived from
    P[h(i) = h(j)] = 1/m and independent signs), within 5 standard errors."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((80, 5)) * rng.uniform(0.2, 3.0, size=(80, 1))
    m = 24
    e2 = np.array([O.sketch_error(A, m, s, 7, t) ** 2 for t in range(3000)])
    want = O.sketch_error_expected_sq(A, m)
    se = e2.std(ddof=1) / np.sqrt(e2.size)
    assert abs(e2.mean() - want) <= 5 * se, (e2.mean(), want, se)
    # and a wrong normalisation (scale 1 instead of 1/s for s > 1) would miss
    if s > 1:
        assert abs(e2.mean() * s - want) > 5 * se


def test_sketch_error_zero_for_injective_hash_and_decreasing_in_m():
    """With m >= n and a draw in which no two rows share a bucket, S^T S = I
    and the error is 0 up to rounding; the mean error falls as m grows."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((6, 3))
    found = False
    for t in range(200):
        b, _ = O.hash_draw(5, t, 1, 4096, 6)
        if len(set(b[0].tolist())) == 6:
            assert O.sketch_error(A, 4096, 1, 5, t) < 1e-14
            found = True
            break
    assert found
    B = rng.standard_normal((400, 6))
    means = [np.mean([O.sketch_error(B, m, 1, 3, t) for t in range(60)]) for m in (30, 120, 480)]
    assert means[0] > means[1] > means[2]


@pytest.mark.parametrize("seed", range(6))
def test_l1_penalty_qp_against_bruteforce(seed):
    """Penalised subproblem (the experiments' LASSO form): the exact solver
    equals brute force over all supports and signs (d = 5), and its KKT
    residual vanishes; lam spans the cases x = 0, sparse and dense."""
    rng = np.random.default_rng(100 + seed)
    d = 5
    M = rng.standard_normal((3 * d, d))
    H = M.T @ M + 0.1 * np.eye(d)
    xt = rng.standard_normal(d)
    g = rng.standard_normal(d) * 3
    c = H @ xt + g
    for lam in (0.05, 0.3 * np.abs(c).max(), 0.8 * np.abs(c).max(), 1.5 * np.abs(c).max()):
        x = O.l1_penalty_qp(H, g, xt, lam)
        xb = O.l1_penalty_qp_bruteforce(H, g, xt, lam)
        assert np.allclose(x, xb, rtol=1e-10, atol=1e-12), (lam, x, xb)
        assert O.l1_penalty_kkt_residual(H, g, xt, lam, x) < 1e-12


def test_l1_penalty_qp_diagonal_closed_form():
    """Diagonal H: the minimiser is soft(c, lam) / h with c = H x^t + g."""
    rng = np.random.default_rng(7)
    d = 40
    h = rng.uniform(0.5, 4.0, d)
    H = np.diag(h)
    xt = rng.standard_normal(d)
    g = rng.standard_normal(d)
    lam = 0.7
    c = H @ xt + g
    want = np.sign(c) * np.maximum(np.abs(c) - lam, 0.0) / h
    assert np.allclose(O.l1_penalty_qp(H, g, xt, lam), want, rtol=1e-12, atol=1e-14)


def test_ihs_l1_penalty_converges_to_xopt():
    """IHS on the penalised LASSO (lam = 5, the experiments' value) reaches the
    directly computed x_OPT, geometrically."""
    w = synth.make("lasso_csr_fp64", n=40000, d=40, m=400)
    C = O.CSR(w["n"], w["d"], w["rowptr"], w["col"], w["val"])
    lam = 5.0
    xo = O.x_opt_l1_penalty(C, w["b"], lam)
    G = C.gram()
    assert O.l1_penalty_kkt_residual(G, C.rmatvec(w["b"]), np.zeros(w["d"]), lam, xo) < 1e-12
    xs = O.ihs(C, w["b"], O.L1_PENALTY, lam, 400, 4, 0, 30)
    errs = [O.err_A(x, xo, G) for x in xs]
    assert errs[-1] < 1e-10
    assert errs[10] < errs[5] < errs[1]


# --------------------------------------------------------------- SRHT ----
def test_srht_definition_against_materialised_hadamard():
    """P H D A by the definition equals the product with S materialised from
    SciPy's Sylvester Hadamard matrix, and the fast transform agrees (n padded
    to a power of two)."""
    from scipy.linalg import hadamard
    rng = np.random.default_rng(21)
    for n in (1, 7, 64, 100):
        A = rng.standard_normal((n, 3))
        m = 12
        rows, sign = O.srht_draw(3, 5, m, n)
        n2 = O.srht_n2(n)
        assert n2 >= n and n2 & (n2 - 1) == 0 and n2 < 2 * max(n, 1) + 1
        S = hadamard(n2)[rows][:, :n] * sign[None, :].astype(float)
        want = S @ A
        got = O.srht_sketch(A, m, rows, sign)
        assert np.allclose(got, want, rtol=0, atol=1e-12)
        assert np.allclose(O.srht_sketch_fast(A, m, rows, sign), want, rtol=0, atol=1e-12)


def test_fwht_is_hadamard_and_involutive():
    """The fast transform is multiplication by the Sylvester matrix, and
    applying it twice gives n2 times the input (H H = n2 I)."""
    from scipy.linalg import hadamard
    rng = np.random.default_rng(22)
    X = rng.standard_normal((256, 4))
    assert np.allclose(O.fwht_rows(X), hadamard(256) @ X, atol=1e-11)
    assert np.allclose(O.fwht_rows(O.fwht_rows(X)), 256 * X, atol=1e-9)


def test_srht_isotropy_and_uniform_rows():
    """E[S^T S] = I for S = m^{-1/2} P H D (mean over draws within 5 standard
    errors entrywise) and the sampled rows are uniform (chi-square)."""
    from scipy.linalg import hadamard
    n, m = 12, 6
    n2 = O.srht_n2(n)
    Hd = hadamard(n2)[:, :n].astype(float)
    acc = np.zeros((n, n)); acc2 = np.zeros((n, n)); T = 4000
    counts = np.zeros(n2)
    for t in range(T):
        rows, sign = O.srht_draw(11, t, m, n)
        S = Hd[rows] * sign[None, :] / np.sqrt(m)
        P = S.T @ S
        acc += P; acc2 += P * P
        np.add.at(counts, rows, 1)
    mean = acc / T
    se = np.sqrt(np.maximum(acc2 / T - mean ** 2, 1e-30) / T)
    assert np.all(np.abs(mean - np.eye(n)) <= 5 * se + 1e-12)
    from scipy.stats import chisquare
    assert chisquare(counts).pvalue > 1e-4


def test_ihs_srht_converges_to_xopt():
    """IHS with the SRHT (Sec. 2's comparison sketch) reaches x_OPT on a dense
    OLS problem at a per-step rate below 1/2."""
    w = synth.make("ols_dense_fp64", n=3000, d=20, m=200)
    A, b = w["A"], w["b"]
    xo = O.x_opt_ols_qr(A, b)
    G = A.T @ A
    xs = O.ihs(A, b, O.OLS, 0.0, 200, 1, 0, 25, sketch_kind="srht")
    errs = [O.err_A(x, xo, G) for x in xs]
    assert errs[-1] < 1e-10
    assert np.median([errs[i + 1] / errs[i] for i in range(8)]) < 0.5


# ------------------------------------------------------------ Gaussian ----
def _standard_normal_pins_hold(z):
    """Mean 0 and variance 1 within 5 standard errors, and a
    Kolmogorov-Smirnov p-value above 1e-3 against N(0, 1)."""
    from scipy.stats import kstest
    return (abs(z.mean()) < 5 / np.sqrt(z.size)
            and abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
            and kstest(z, "norm").pvalue > 1e-3)


def test_gauss_draw_is_standard_normal():
    """The Gaussian sketch's entries (Box-Muller of the counter words) have
    mean 0, variance 1 and pass a Kolmogorov-Smirnov test against N(0, 1);
    E[S^T S] = I for S = G / sqrt(m) (5 standard errors entrywise)."""
    assert _standard_normal_pins_hold(O.gauss_draw(5, 0, 200, 1000).ravel())
    n, m, T = 6, 4, 3000
    acc = np.zeros((n, n)); acc2 = np.zeros((n, n))
    for t in range(T):
        S = O.gauss_draw(9, t, m, n) / np.sqrt(m)
        P = S.T @ S
        acc += P; acc2 += P * P
    mean = acc / T
    se = np.sqrt(np.maximum(acc2 / T - mean ** 2, 1e-30) / T)
    assert np.all(np.abs(mean - np.eye(n)) <= 5 * se)


def test_ihs_gaussian_converges_to_xopt():
    """IHS with the Gaussian sketch reaches x_OPT at a rate near the
    inverse-Wishart value (0.39 at m = 10d)."""
    w = synth.make("ols_dense_fp64", n=3000, d=20, m=200)
    A, b = w["A"], w["b"]
    xo = O.x_opt_ols_qr(A, b)
    G = A.T @ A
    xs = O.ihs(A, b, O.OLS, 0.0, 200, 1, 0, 25, sketch_kind="gaussian")
    errs = [O.err_A(x, xo, G) for x in xs]
    assert errs[-1] < 1e-10
    assert np.median([errs[i + 1] / errs[i] for i in range(10)]) < 0.5


# ------------------------------------------------------------ p = 2 ball ----
def test_l2_ball_qp_identity_is_projection():
    """H = I: the minimiser is the Euclidean projection of x^t + g onto the ball."""
    rng = np.random.default_rng(31)
    d = 9
    xt = rng.standard_normal(d)
    g = 3 * rng.standard_normal(d)
    v = xt + g
    for R in (0.3 * np.linalg.norm(v), 2 * np.linalg.norm(v)):
        want = v * min(1.0, R / np.linalg.norm(v))
        assert np.allclose(O.l2_ball_qp(np.eye(d), g, xt, R), want, rtol=1e-13, atol=1e-14)


def test_l2_ball_qp_against_circle_bruteforce():
    """d = 2: the exact solver matches a brute-force minimum over 2e5 points of
    the circle (refined by golden section) and has a vanishing KKT residual."""
    rng = np.random.default_rng(32)
    for trial in range(5):
        M = rng.standard_normal((4, 2))
        H = M.T @ M + 0.1 * np.eye(2)
        xt = rng.standard_normal(2)
        g = 4 * rng.standard_normal(2)
        c = H @ xt + g
        R = 0.5 * np.linalg.norm(np.linalg.solve(H, c))
        q = lambda x: 0.5 * (x - xt) @ H @ (x - xt) - g @ (x - xt)
        th = np.linspace(0, 2 * np.pi, 200001)
        pts = R * np.stack([np.cos(th), np.sin(th)], 1)
        vals = 0.5 * np.einsum("ij,jk,ik->i", pts - xt, H, pts - xt) - (pts - xt) @ g
        t0 = th[np.argmin(vals)]
        a, b = t0 - 1e-4, t0 + 1e-4
        f = lambda t: q(R * np.array([np.cos(t), np.sin(t)]))
        gr = (np.sqrt(5) - 1) / 2
        for _ in range(200):
            c1, c2 = b - gr * (b - a), a + gr * (b - a)
            if f(c1) < f(c2):
                b = c2
            else:
                a = c1
        xb = R * np.array([np.cos(0.5 * (a + b)), np.sin(0.5 * (a + b))])
        x = O.l2_ball_qp(H, g, xt, R)
        assert np.allclose(x, xb, atol=1e-8), (x, xb)
        assert O.l2_ball_kkt_residual(H, g, xt, R, x) < 1e-12


def test_ihs_l2_ball_converges_to_xopt():
    """IHS over the p = 2 ball (radius half of ||x_OLS||) reaches x_OPT."""
    w = synth.make("ols_dense_fp64", n=3000, d=20, m=200)
    A, b = w["A"], w["b"]
    R = 0.5 * np.linalg.norm(O.x_opt_ols_qr(A, b))
    xo = O.x_opt_l2(A, b, R)
    G = A.T @ A
    assert O.l2_ball_kkt_residual(G, A.T @ b, np.zeros(20), R, xo) < 1e-12
    xs = O.ihs(A, b, O.L2_BALL, R, 200, 1, 0, 30)
    assert O.err_A(xs[-1], xo, G) < 1e-10


# ------------------------------------------------- multi-core oracle build ---
def test_multicore_oracle_build_is_bit_identical():
    """The OpenMP build that times the CPU baseline gives every thread its own
    outputs and sums each one over the same terms in the same order, so it
    returns exactly what the serial build returns: the draw, SA (dense and
    CSR, SJLT s = 3 with ragged bucket ranges over 5 threads), the Gram, the
    residual and gradient (dense and CSR) and the Gaussian G."""
    rng = np.random.default_rng(4)
    n, d, m, s = 3001, 23, 93, 3
    A = rng.standard_normal((n, d))
    b = rng.standard_normal(n)
    x = rng.standard_normal(d)
    rowptr, col, val = synth.csr_uniform(n, d, 4, 3, np.float64)
    C = O.CSR(n, d, rowptr, col, val)
    out = {}
    for threads in (1, 5):
        O.use_threads(threads)
        try:
            bk, sg = O.hash_draw(7, 2, s, m, n)
            out[threads] = [bk, sg, O.sketch(A, m, s, bk, sg), O.sketch(C, m, s, bk, sg),
                            O.gram(O.sketch(A, m, s, bk, sg), 1.0 / s, 0.5),
                            *O.resid_grad(A, b, x, want_r=True), *O.resid_grad(C, b, x, want_r=True),
                            O.resid_grad(A, b, x), O.gauss_draw(3, 1, 17, 211)]
        finally:
            O.use_threads(1)
    for a, c in zip(out[1], out[5]):
        assert a.dtype == c.dtype and np.array_equal(a, c)
