"""FP64 CPU oracle for the Iterative Hessian Sketch (Cormode & Dickens,
"Iterative Hessian Sketch in Input Sparsity Time", arXiv 1910.14166).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  The GPU
library never calls it and shares no code with it: the O(nnz) data passes and
the hash live in ``ihs_oracle.c`` (plain C loops, FP64), the d-dimensional
algebra below is plain NumPy/SciPy in FP64, each function citing the part of
the paper it states.

What is pinned, and by what (see tests/test_oracle.py):
  * hash: published SplitMix64 outputs; uniformity; the sketch lemmas of
    App. A (S S^T diagonal with the row counts, E[S S^T] = (n/m) I,
    E[S^T S] = I with diag(S^T S) = 1 on every draw).
  * sketch: brute-force S A with S materialised as a dense matrix.
  * Gram: dense matmul of the materialised sketch; E over draws -> A^T A.
  * residual / gradient: finite differences of f(x) = 1/2 ||Ax - b||^2 (Eq. 1).
  * OLS step: identity sketch gives x_OPT (numpy lstsq) in one step (Eq. 2).
  * l1-ball QP: brute force over all faces of the ball for d <= 6; KKT.
  * penalised-l1 QP: brute force over all supports and signs for d <= 6; the
    soft-threshold closed form for diagonal H; KKT.
  * sketch error (App. B): the closed form of its mean square over draws.
  * SRHT (Sec. 2): P H D A against the materialised product with SciPy's
    Sylvester Hadamard matrix; the fast transform against the definition;
    E[S^T S] = I over draws; uniform sampled rows.
  * p = 2 ball QP: the projection closed form for H = I; brute force over
    the circle for d = 2; KKT.
  * Gaussian sketch (Sec. 2): moments and a Kolmogorov-Smirnov test of the
    entries against N(0, 1); E[S^T S] = I.
  * x_OPT: Householder QR vs refined normal equations vs lstsq.
  * IHS: geometric convergence at a rate below 1/2 (Thm. 2.2).
  * ridge adjoint: central finite differences in FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ihs_oracle.c")
_SO = os.path.join(_HERE, "libihs_oracle.so")
_lock = threading.Lock()

u64 = ctypes.c_uint64
i64 = ctypes.c_int64
i32 = ctypes.c_int
f64 = ctypes.c_double
vp = ctypes.c_void_p


_SO_MT = os.path.join(_HERE, "libihs_oracle_mt.so")
_libs = {}
_active = "serial"


def build_oracle(force: bool = False) -> str:
    """Compile ihs_oracle.c with gcc (plain -O2, no fast-math, no FMA
    contraction), and the same file with -fopenmp into the multi-core build
    (the timed CPU baseline; bit-identical results, see the C file)."""
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]
    for so, extra in ((_SO, []), (_SO_MT, ["-fopenmp"])):
        if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
            tmp = so + ".tmp%d" % os.getpid()
            try:
                subprocess.check_call(base + extra + ["-o", tmp, _SRC, "-lm"])
            except subprocess.CalledProcessError:
                if extra:  # no OpenMP runtime: the multi-core build is simply absent
                    continue
                raise
            os.replace(tmp, so)
    return _SO


def _bind(L):
    L.orc_set_threads.restype = i32
    L.orc_set_threads.argtypes = [i32]
    L.orc_sm64_at.restype = u64
    L.orc_sm64_at.argtypes = [u64, u64]
    L.orc_hash.restype = i32
    L.orc_hash.argtypes = [u64, i64, i32, i64, i64, vp, vp]
    L.orc_sketch_dense.restype = None
    L.orc_sketch_dense.argtypes = [i64, i64, vp, i64, i64, i32, vp, vp, vp]
    L.orc_sketch_csr.restype = None
    L.orc_sketch_csr.argtypes = [i64, i64, vp, vp, vp, i64, i32, vp, vp, vp]
    L.orc_gram.restype = None
    L.orc_gram.argtypes = [i64, i64, vp, f64, f64, vp]
    L.orc_resid_grad_dense.restype = i32
    L.orc_resid_grad_dense.argtypes = [i64, i64, vp, i64, vp, vp, vp, vp]
    L.orc_resid_grad_csr.restype = i32
    L.orc_resid_grad_csr.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp, vp]
    L.orc_sketch_adjoint.restype = None
    L.orc_sketch_adjoint.argtypes = [i64, i64, i64, i32, vp, vp, vp, f64, vp]
    L.orc_srht_draw.restype = i32
    L.orc_srht_draw.argtypes = [u64, i64, i64, i64, i64, vp, vp]
    L.orc_srht_sketch_dense.restype = None
    L.orc_srht_sketch_dense.argtypes = [i64, i64, vp, i64, i64, vp, vp, vp]
    L.orc_gauss_draw.restype = None
    L.orc_gauss_draw.argtypes = [u64, i64, i64, i64, vp]
    return L


def _load(kind):
    with _lock:
        if kind not in _libs:
            build_oracle()
            path = _SO if kind == "serial" else _SO_MT
            if not os.path.exists(path):
                raise RuntimeError("the multi-core oracle build is unavailable (no OpenMP)")
            _libs[kind] = _bind(ctypes.CDLL(path))
    return _libs[kind]


def lib():
    """The C library the oracle's data passes run in (serial unless
    use_threads() selected the multi-core build)."""
    return _load(_active)


def use_threads(n: int) -> int:
    """Run the C loops on n threads (the multi-core build; n <= 1: the serial
    build).  Results are bit-identical either way.  Returns the threads used."""
    global _active
    if n is None or n <= 1:
        _active = "serial"
        return 1
    L = _load("mt")
    _active = "mt"
    return int(L.orc_set_threads(int(n)))


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------
# Matrices: dense np.ndarray (n x d) or a CSR triple.
# --------------------------------------------------------------------------
class CSR:
    """CSR matrix with int64 rowptr, int32 col, float64 val (the oracle's own copy)."""

    def __init__(self, n, d, rowptr, col, val):
        self.n, self.d = int(n), int(d)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)

    @property
    def shape(self):
        return (self.n, self.d)

    def todense(self):
        out = np.zeros((self.n, self.d))
        for i in range(self.n):
            a, b = self.rowptr[i], self.rowptr[i + 1]
            out[i, self.col[a:b]] += self.val[a:b]
        return out

    def matvec(self, x):
        """A x (the residual's product in Eq. 2's gradient)."""
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        out = np.zeros(self.n)
        np.add.at(out, rows, self.val * x[self.col])
        return out

    def gram(self):
        """A^T A in FP64 (for x_OPT and the error metric)."""
        d = self.d
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        # A^T A = sum over rows of outer products; build via a dense column block product.
        try:
            import scipy.sparse as sp
            M = sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, d))
            return np.asarray((M.T @ M).todense())
        except ImportError:  # plain fallback
            G = np.zeros((d, d))
            for i in range(self.n):
                a, b = self.rowptr[i], self.rowptr[i + 1]
                c, v = self.col[a:b], self.val[a:b]
                G[np.ix_(c, c)] += np.outer(v, v)
            return G

    def rmatvec(self, r):
        """A^T r (the gradient of Eq. 2)."""
        out = np.zeros(self.d)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        np.add.at(out, self.col, self.val * r[rows])
        return out


def as_f64(A):
    if isinstance(A, CSR):
        return A
    return np.ascontiguousarray(A, dtype=np.float64)


# --------------------------------------------------------------------------
# Sketch draw and data passes (C loops).
# --------------------------------------------------------------------------
def sm64_at(state: int, j: int) -> int:
    """Output j of a SplitMix64 generator started at `state` (Steele, Lea & Flood 2014)."""
    return int(lib().orc_sm64_at(u64(state & 0xFFFFFFFFFFFFFFFF), u64(j)))


def hash_draw(seed: int, t: int, s: int, m: int, n: int):
    """Sketch S^{t} of Sec. 2: bucket (global row of S, int32 [s, n]) and sign (int8 [s, n])."""
    bucket = np.empty((s, n), dtype=np.int32)
    sign = np.empty((s, n), dtype=np.int8)
    rc = lib().orc_hash(u64(seed & 0xFFFFFFFFFFFFFFFF), i64(t), i32(s), i64(m), i64(n),
                        _p(bucket), _p(sign))
    if rc != 0:
        raise ValueError("invalid sketch shape: m=%d s=%d" % (m, s))
    return bucket, sign


def sketch(A, m: int, s: int, bucket, sign):
    """Raw SA (unscaled +-1 entries), m x d FP64, by the streaming pass of Sec. 2."""
    bucket = np.ascontiguousarray(bucket, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    if isinstance(A, CSR):
        SA = np.empty((m, A.d))
        lib().orc_sketch_csr(A.n, A.d, _p(A.rowptr), _p(A.col), _p(A.val), m, s,
                             _p(bucket), _p(sign), _p(SA))
        return SA
    A = as_f64(A)
    n, d = A.shape
    SA = np.empty((m, d))
    lib().orc_sketch_dense(n, d, _p(A), d, m, s, _p(bucket), _p(sign), _p(SA))
    return SA


def gram(SA, scale: float, shift: float = 0.0):
    """H = scale * SA^T SA + shift * I (Sec. 1), plain triple loop."""
    SA = np.ascontiguousarray(SA, dtype=np.float64)
    m, d = SA.shape
    H = np.empty((d, d))
    lib().orc_gram(m, d, _p(SA), f64(scale), f64(shift), _p(H))
    return H


def resid_grad(A, b, x, want_r: bool = False):
    """r = b - A x and g = A^T r (Eq. 2's linear term), rows in order, FP64."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = b.shape[0]
    r = np.empty(n) if want_r else None
    if isinstance(A, CSR):
        g = np.empty(A.d)
        rc = lib().orc_resid_grad_csr(A.n, A.d, _p(A.rowptr), _p(A.col), _p(A.val), _p(b),
                                      _p(x), _p(r) if want_r else None, _p(g))
    else:
        A = as_f64(A)
        g = np.empty(A.shape[1])
        rc = lib().orc_resid_grad_dense(A.shape[0], A.shape[1], _p(A), A.shape[1], _p(b), _p(x),
                                        _p(r) if want_r else None, _p(g))
    if rc != 0:
        raise MemoryError("oracle residual buffer")
    return (r, g) if want_r else g


def sketch_adjoint(G, n: int, s: int, bucket, sign):
    """S^T G for the normalised sketch (entries sign/sqrt(s), App. A), n x d
    FP64: the adjoint of the streaming product of Sec. 2, a gather by bucket."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    m, d = G.shape
    out = np.empty((n, d))
    lib().orc_sketch_adjoint(n, d, m, s, _p(np.ascontiguousarray(bucket, dtype=np.int32)),
                             _p(np.ascontiguousarray(sign, dtype=np.int8)), _p(G),
                             f64(1.0 / np.sqrt(s)), _p(out))
    return out


def sketch_matrix(m: int, s: int, bucket, sign):
    """Dense S (m x n) of Sec. 2 with entries sign/sqrt(s) (App. A): only for
    brute-force pins on tiny n."""
    n = bucket.shape[1]
    S = np.zeros((m, n))
    for k in range(s):
        for i in range(n):
            S[bucket[k, i], i] += sign[k, i] / np.sqrt(s)
    return S


# --------------------------------------------------------------------------
# d-dimensional algebra (FP64, NumPy / SciPy primitives).
# --------------------------------------------------------------------------
def chol_solve(H, g):
    """Solve H delta = g through the Cholesky factor H = L L^T (OLS step of Eq. 2)."""
    from scipy.linalg import solve_triangular
    L = np.linalg.cholesky(H)
    y = solve_triangular(L, g, lower=True)
    return solve_triangular(L.T, y, lower=False)


def project_l1_ball(v, R):
    """Euclidean projection onto {x : ||x||_1 <= R} (Duchi, Shalev-Shwartz,
    Singer & Chandra 2008, sort-based)."""
    if np.abs(v).sum() <= R:
        return v.copy()
    u = np.sort(np.abs(v))[::-1]
    css = np.cumsum(u)
    j = np.arange(1, v.size + 1)
    rho = np.nonzero(u - (css - R) / j > 0)[0][-1]
    theta = (css[rho] - R) / (rho + 1.0)
    return np.sign(v) * np.maximum(np.abs(v) - theta, 0.0)


def _l1_face_solve(H, c, R, S, sgn):
    """Minimise 1/2 x^T H x - c^T x on {x_S^T sgn = R, x_{S^c} = 0}: the
    bordered KKT system [H_SS sgn; sgn^T 0][z; mu] = [c_S; R] (one face of the
    l1 ball in Eq. 2's subproblem, solved exactly as Sec. 3 asks)."""
    k = len(S)
    K = np.zeros((k + 1, k + 1))
    K[:k, :k] = H[np.ix_(S, S)]
    K[:k, k] = sgn
    K[k, :k] = sgn
    rhs = np.concatenate([c[S], [R]])
    sol = np.linalg.solve(K, rhs)
    return sol[:k], sol[k]


def l1_kkt_residual(H, g, xt, R, x):
    """Relative KKT violation of x for the l1-ball QP of Eq. 2 (0 at the exact
    solution, the certificate of Sec. 3's "solved exactly")."""
    c = H @ xt + g
    grad = H @ x - c
    scale = max(np.abs(c).max(), 1e-300)
    if np.abs(x).sum() < R * (1 - 1e-12):
        return np.abs(grad).max() / scale
    S = np.nonzero(x)[0]
    if S.size == 0:
        return np.inf
    mu = -np.mean(grad[S] * np.sign(x[S]))
    on = np.abs(grad[S] + mu * np.sign(x[S])).max()
    off = 0.0
    mask = np.ones(x.size, bool)
    mask[S] = False
    if mask.any():
        off = max(0.0, (np.abs(grad[mask]) - mu).max())
    return max(on, off, max(0.0, -mu), abs(np.abs(x).sum() - R) / max(R, 1e-300)) / scale


def l1_ball_qp(H, g, xt, R, tol=1e-13, max_rounds=200, inner=200):
    """Exact minimiser of the l1-ball subproblem of Eq. 2:
        argmin_{||x||_1 <= R} 1/2 (x - xt)^T H (x - xt) - g^T (x - xt).
    The paper solves each subproblem "exactly" (Sec. 3); this oracle reads that
    as: the unconstrained Newton point if it is feasible; otherwise FISTA (Beck
    & Teboulle 2009) with the l1-ball projection locates the support and signs,
    and the bordered KKT system on that face gives the exact point, accepted
    only when its signs match and the off-support optimality holds."""
    c = H @ xt + g
    xu = chol_solve(H, c)
    if np.abs(xu).sum() <= R:
        return xu
    Lip = np.linalg.eigvalsh(H)[-1]
    x = project_l1_ball(xt, R)
    y = x.copy()
    tk = 1.0
    for _ in range(max_rounds):
        for _ in range(inner):
            xn = project_l1_ball(y - (H @ y - c) / Lip, R)
            tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
            y = xn + ((tk - 1.0) / tn) * (xn - x)
            x, tk = xn, tn
        S = np.nonzero(x)[0]
        if S.size == 0:
            continue
        sgn = np.sign(x[S])
        z, mu = _l1_face_solve(H, c, R, S, sgn)
        if mu < 0 or np.any(z * sgn <= 0):
            continue
        xf = np.zeros_like(x)
        xf[S] = z
        grad = H @ xf - c
        mask = np.ones(x.size, bool)
        mask[S] = False
        if (not mask.any()) or np.all(np.abs(grad[mask]) <= mu * (1.0 + 1e-9) + tol * np.abs(c).max()):
            return xf
    raise RuntimeError("l1-ball QP did not reach an exact KKT point")


def l1_ball_qp_bruteforce(H, g, xt, R):
    """Eq. 2's l1-ball subproblem by brute force for tiny d: the unconstrained
    point if feasible, else the best point over every face of the ball (all
    sign patterns in {-1,0,1}^d)."""
    import itertools
    d = H.shape[0]
    c = H @ xt + g
    q = lambda x: 0.5 * x @ H @ x - c @ x
    xu = np.linalg.solve(H, c)
    if np.abs(xu).sum() <= R:
        return xu
    best, bq = None, np.inf
    for pat in itertools.product((-1, 0, 1), repeat=d):
        pat = np.array(pat)
        S = np.nonzero(pat)[0]
        if S.size == 0:
            continue
        z, _ = _l1_face_solve(H, c, R, S, pat[S].astype(float))
        if np.any(z * pat[S] < 0):
            continue
        x = np.zeros(d)
        x[S] = z
        if q(x) < bq:
            best, bq = x, q(x)
    return best


def soft_threshold(v, tau):
    """Proximal map of tau ||.||_1 (the penalised LASSO of Sec. 3's
    experiments): sign(v) max(|v| - tau, 0)."""
    return np.sign(v) * np.maximum(np.abs(v) - tau, 0.0)


def _pen_face_solve(H, c, lam, S, sgn):
    """Stationary point of 1/2 x^T H x - c^T x + lam sgn^T x_S on {x_{S^c} = 0}:
    H_SS x_S = c_S - lam sgn (one face of the penalised form of Eq. 2's
    subproblem, Sec. 3's experiments)."""
    return np.linalg.solve(H[np.ix_(S, S)], c[S] - lam * sgn)


def l1_penalty_objective(H, g, xt, lam, x):
    """Eq. 2's subproblem with the penalty of Sec. 3's experiments:
    1/2 (x - xt)^T H (x - xt) - g^T (x - xt) + lam ||x||_1."""
    e = np.asarray(x) - xt
    return float(0.5 * e @ H @ e - g @ e + lam * np.abs(x).sum())


def l1_penalty_kkt_residual(H, g, xt, lam, x):
    """Relative violation of 0 in H (x - xt) - g + lam d||x||_1 for the
    penalised subproblem of Eq. 2 (0 at the optimum)."""
    c = H @ xt + g
    grad = H @ x - c
    scale = max(np.abs(c).max(), lam, 1e-300)
    S = x != 0
    on = np.abs(grad[S] + lam * np.sign(x[S])).max() if S.any() else 0.0
    off = max(0.0, (np.abs(grad[~S]) - lam).max()) if (~S).any() else 0.0
    return max(on, off) / scale


def l1_penalty_qp(H, g, xt, lam, tol=1e-13, max_rounds=200, inner=200):
    """Exact minimiser of the penalised-LASSO subproblem (the experiments' form,
    Sec. 5: 1/2 ||Ax - b||^2 + lam ||x||_1, each subproblem solved exactly):
        argmin_x 1/2 (x - xt)^T H (x - xt) - g^T (x - xt) + lam ||x||_1.
    Proximal FISTA (Beck & Teboulle 2009; soft thresholding) locates the
    support and signs; the stationarity system H_SS x_S = c_S - lam sgn on that
    support (c = H xt + g) gives the exact point, accepted only when its signs
    match and |(H x - c)_j| <= lam off the support."""
    c = H @ xt + g
    if np.abs(c).max() <= lam:
        return np.zeros_like(c)
    Lip = np.linalg.eigvalsh(H)[-1]
    x = np.array(xt, dtype=np.float64)
    y = x.copy()
    tk = 1.0
    for _ in range(max_rounds):
        for _ in range(inner):
            xn = soft_threshold(y - (H @ y - c) / Lip, lam / Lip)
            tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
            y = xn + ((tk - 1.0) / tn) * (xn - x)
            x, tk = xn, tn
        S = np.nonzero(x)[0]
        if S.size == 0:
            continue
        sgn = np.sign(x[S])
        z = _pen_face_solve(H, c, lam, S, sgn)
        if np.any(z * sgn <= 0):
            continue
        xf = np.zeros_like(x)
        xf[S] = z
        grad = H @ xf - c
        mask = np.ones(x.size, bool)
        mask[S] = False
        if (not mask.any()) or np.all(np.abs(grad[mask]) <= lam * (1.0 + 1e-9) + tol * np.abs(c).max()):
            return xf
    raise RuntimeError("penalised l1 QP did not reach an exact KKT point")


def l1_penalty_qp_bruteforce(H, g, xt, lam):
    """The penalised subproblem of Eq. 2 by brute force for tiny d: the best
    stationary point over every support and sign pattern in {-1,0,1}^d
    (x = 0 included)."""
    import itertools
    d = H.shape[0]
    best, bq = np.zeros(d), l1_penalty_objective(H, g, xt, lam, np.zeros(d))
    c = H @ xt + g
    for pat in itertools.product((-1, 0, 1), repeat=d):
        pat = np.array(pat)
        S = np.nonzero(pat)[0]
        if S.size == 0:
            continue
        z = _pen_face_solve(H, c, lam, S, pat[S].astype(float))
        if np.any(z * pat[S] <= 0):
            continue
        x = np.zeros(d)
        x[S] = z
        q = l1_penalty_objective(H, g, xt, lam, x)
        if q < bq:
            best, bq = x, q
    return best


def l2_ball_qp(H, g, xt, R, iters: int = 400):
    """Exact minimiser of the p = 2 ball subproblem (Sec. 1's C = {x : ||x||_2 <= R}):
        argmin_{||x||_2 <= R} 1/2 (x - xt)^T H (x - xt) - g^T (x - xt).
    With c = H xt + g: the Newton point H^{-1} c if it lies in the ball; else
    x(mu) = (H + mu I)^{-1} c on the sphere, mu > 0 the root of
    ||x(mu)|| = R, found on the eigenbasis of H (numpy.linalg.eigh) by
    bisection on [0, ||c|| / R] to the last bit (||x(mu)|| falls with mu)."""
    c = H @ xt + g
    xn = chol_solve(H, c)
    if np.linalg.norm(xn) <= R:
        return xn
    lam, Q = np.linalg.eigh(H)
    bq = Q.T @ c
    norm = lambda mu: np.sqrt(np.sum((bq / (lam + mu)) ** 2))
    lo, hi = 0.0, np.linalg.norm(c) / R
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if norm(mid) > R:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    return Q @ (bq / (lam + mu))


def l2_ball_kkt_residual(H, g, xt, R, x):
    """Relative KKT violation of x for the p = 2 ball subproblem (Sec. 1's
    norm balls, Eq. 2): stationarity H (x - xt) - g + mu x = 0 with mu >= 0,
    and mu (||x|| - R) = 0."""
    c = H @ xt + g
    grad = H @ x - c
    scale = max(np.abs(c).max(), 1e-300)
    nx = np.linalg.norm(x)
    if nx < R * (1 - 1e-12):
        return np.abs(grad).max() / scale
    mu = -float(grad @ x) / (nx * nx)
    return max(np.abs(grad + mu * x).max(), max(0.0, -mu) * nx, abs(nx - R) / R * scale) / scale


# --------------------------------------------------------------------------
# IHS (Eq. 2) and its fixed point.
# --------------------------------------------------------------------------
OLS, L1_BALL, RIDGE, L1_PENALTY, L2_BALL = 0, 1, 2, 3, 4


def ihs(A, b, kind: int, param: float, m: int, s: int, seed: int, iters: int, x0=None,
        t0: int = 0, keep_sketch: bool = False, sketch_kind: str = "sparse"):
    """Iterates x^0..x^iters of Eq. 2 with a fresh sketch per step.

    Iteration t (t = t0, t0+1, ...) draws the sketch with counter t, builds
    H = (1/s) (SA)^T SA (+ lam I for ridge) and g = A^T (b - A x^t) (- lam x^t
    for ridge), then takes the QP step: Cholesky for OLS / ridge, the exact
    l1-ball QP for LASSO, the exact penalised QP for L1_PENALTY.  x^0 = 0
    unless x0 is given.  sketch_kind "srht" uses S = m^{-1/2} P H D (Sec. 2)
    instead of the sparse embedding: H = (1/m) (P H D A)^T (P H D A);
    "gaussian" uses S = G / sqrt(m): H = (1/m) (G A)^T (G A)."""
    A = as_f64(A)
    n, d = A.shape
    x = np.zeros(d) if x0 is None else np.array(x0, dtype=np.float64)
    xs = [x.copy()]
    sk = []
    for t in range(t0, t0 + iters):
        shift = param if kind == RIDGE else 0.0
        if sketch_kind == "srht":
            rows, sgn = srht_draw(seed, t, m, n)
            SA = srht_sketch_fast(A, m, rows, sgn)
            H = gram(SA, 1.0 / m, shift)
        elif sketch_kind == "gaussian":
            H = gram(gauss_sketch(A, m, seed, t), 1.0 / m, shift)
        else:
            bucket, sign = hash_draw(seed, t, s, m, n)
            SA = sketch(A, m, s, bucket, sign)
            H = gram(SA, 1.0 / s, shift)
        g = resid_grad(A, b, x)
        if kind == RIDGE:
            g = g - param * x
        if kind == L1_BALL:
            x = l1_ball_qp(H, g, x, param)
        elif kind == L1_PENALTY:
            x = l1_penalty_qp(H, g, x, param)
        elif kind == L2_BALL:
            x = l2_ball_qp(H, g, x, param)
        else:
            x = x + chol_solve(H, g)
        xs.append(x.copy())
        if keep_sketch:
            sk.append((SA, H, g))
    return (xs, sk) if keep_sketch else xs


def ata(A):
    """A^T A in FP64: the Hessian of Eq. 1 (x_OPT, the norm ||.||_A)."""
    A = as_f64(A)
    if isinstance(A, CSR):
        return A.gram()
    return A.T @ A


def atb(A, b):
    """A^T b in FP64: the linear term of Eq. 1."""
    A = as_f64(A)
    if isinstance(A, CSR):
        return A.rmatvec(b)
    return A.T @ b


def x_opt_ols_qr(A, b):
    """x_OPT of Eq. 1 with C = R^d by Householder QR (numpy.linalg.qr)."""
    Q, Rm = np.linalg.qr(as_f64(A))
    from scipy.linalg import solve_triangular
    return solve_triangular(Rm, Q.T @ b, lower=False)


def x_opt_ols_normal(A, b, lam: float = 0.0, refine: int = 3):
    """x_OPT of Eq. 1 with C = R^d (lam > 0: ridge, not in the paper) from the
    normal equations (A^T A + lam I) x = A^T b, Cholesky in FP64 plus `refine`
    rounds of iterative refinement with FP64 residuals."""
    A = as_f64(A)
    G = ata(A) + lam * np.eye(A.shape[1])
    x = chol_solve(G, atb(A, b))
    for _ in range(refine):
        g = resid_grad(A, b, x) - lam * x
        x = x + chol_solve(G, g)
    return x


def x_opt_l1(A, b, R):
    """x_OPT of Eq. 1 over the l1 ball: the QP with H = A^T A, x^t = 0, g = A^T b."""
    A = as_f64(A)
    G = ata(A)
    return l1_ball_qp(G, atb(A, b), np.zeros(A.shape[1]), R)


def x_opt_l1_penalty(A, b, lam):
    """x_OPT of the penalised LASSO of Sec. 3's experiments,
    1/2 ||Ax - b||^2 + lam ||x||_1: the subproblem above with H = A^T A,
    x^t = 0, g = A^T b."""
    A = as_f64(A)
    return l1_penalty_qp(ata(A), atb(A, b), np.zeros(A.shape[1]), lam)


def x_opt_l2(A, b, R):
    """x_OPT of Eq. 1 over the p = 2 ball: the subproblem with H = A^T A, x^t = 0, g = A^T b."""
    A = as_f64(A)
    return l2_ball_qp(ata(A), atb(A, b), np.zeros(A.shape[1]), R)


def err_A(x, xopt, G):
    """||x - x_OPT||_A / ||x_OPT||_A with ||v||_A = n^{-1/2} ||A v|| (Def. of
    an eps-solution approximation); G = A^T A, the n^{-1/2} factors cancel."""
    e = np.asarray(x) - xopt
    return float(np.sqrt(max(e @ G @ e, 0.0)) / np.sqrt(xopt @ G @ xopt))


def ridge_adjoint(A, b, lam, dLdx):
    """Exact gradients of L(x(A, b)) for the ridge solution
    x = (A^T A + lam I)^{-1} A^T b (ridge is not in the paper; its nearest
    constraint is Sec. 1's p = 2 ball): v = (A^T A + lam I)^{-1} dL/dx,
    dL/db = A v,  dL/dA = r v^T - (A v) x^T with r = b - A x.  Dense FP64
    solves."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    G = A.T @ A + lam * np.eye(A.shape[1])
    x = chol_solve(G, A.T @ b)
    v = chol_solve(G, dLdx)
    r = b - A @ x
    Av = A @ v
    return x, Av, np.outer(r, v) - np.outer(Av, x)


def srht_n2(n: int) -> int:
    """Rows of the SRHT's Hadamard transform (Sec. 2): the least power of two
    >= n (A is padded with zero rows)."""
    return 1 << max(0, (int(n) - 1).bit_length())


def srht_draw(seed: int, t: int, m: int, n: int):
    """SRHT of Sec. 2 (S = P H D): sampled rows (int32 [m], in [0, n2)) and signs (int8 [n])."""
    n2 = srht_n2(n)
    rows = np.empty(m, dtype=np.int32)
    sign = np.empty(n, dtype=np.int8)
    rc = lib().orc_srht_draw(u64(seed & 0xFFFFFFFFFFFFFFFF), i64(t), i64(m), i64(n), i64(n2),
                             _p(rows), _p(sign))
    if rc != 0:
        raise ValueError("invalid SRHT shape")
    return rows, sign


def srht_sketch(A, m: int, rows, sign):
    """Raw P H D A (m x d, FP64) by the definition (Sec. 2, SRHT), O(m n d)."""
    A = np.ascontiguousarray(as_f64(A))
    n, d = A.shape
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    SA = np.empty((m, d))
    lib().orc_srht_sketch_dense(n, d, _p(A), d, m, _p(rows), _p(sign), _p(SA))
    return SA


def fwht_rows(X):
    """Unnormalised Walsh-Hadamard transform (the H of Sec. 2's SRHT) along
    axis 0 (length a power of two), by the recursive definition H_{2k} = [H_k H_k; H_k -H_k]: stage h
    replaces each pair (u, v) at distance h by (u + v, u - v)."""
    Y = np.array(X, dtype=np.float64, copy=True)
    n2 = Y.shape[0]
    h = 1
    while h < n2:
        Y = Y.reshape(n2 // (2 * h), 2, h, *Y.shape[1:])
        u = Y[:, 0].copy()
        v = Y[:, 1].copy()
        Y[:, 0] = u + v
        Y[:, 1] = u - v
        Y = Y.reshape(n2, *Y.shape[3:])
        h *= 2
    return Y


def srht_sketch_fast(A, m: int, rows, sign):
    """P H D A of Sec. 2's SRHT through the fast transform (the same numbers
    as srht_sketch up to the order of the additions): pad D A to n2 rows,
    transform, take rows."""
    A = as_f64(A)
    n, d = A.shape
    X = np.zeros((srht_n2(n), d))
    X[:n] = np.asarray(sign, dtype=np.float64)[:, None] * A
    return fwht_rows(X)[np.asarray(rows)]


def gauss_draw(seed: int, t: int, m: int, n: int):
    """G (m x n, FP64) of the Gaussian sketch S = G / sqrt(m) (Sec. 2)."""
    G = np.empty((m, n))
    lib().orc_gauss_draw(u64(seed & 0xFFFFFFFFFFFFFFFF), i64(t), i64(m), i64(n), _p(G))
    return G


def gauss_sketch(A, m: int, seed: int, t: int):
    """Raw G A (m x d, FP64) for Sec. 2's Gaussian sketch of counter t (Gram
    scale 1/m)."""
    A = as_f64(A)
    return gauss_draw(seed, t, m, A.shape[0]) @ A


def sketch_error(A, m: int, s: int, seed: int, t: int):
    """Empirical sketch error of the experiments (App. B):
    ||A^T S^T S A - A^T A||_F / ||A^T A||_F for the sketch of counter t, with
    S^T S normalised as in Sec. 2 (Gram scale 1/s)."""
    n = A.n if isinstance(A, CSR) else np.asarray(A).shape[0]
    bucket, sign = hash_draw(seed, t, s, m, n)
    H = gram(sketch(A, m, s, bucket, sign), 1.0 / s)
    G = ata(A)
    return float(np.linalg.norm(H - G) / np.linalg.norm(G))


def sketch_error_expected_sq(A, m: int):
    """E ||A^T S^T S A - A^T A||_F^2 / ||A^T A||_F^2 over the draw, for a
    CountSketch with m rows and for the SJLT of Sec. 2 with m rows in total
    (s blocks of m/s, scale 1/s): (||A||_F^4 + ||A^T A||_F^2 - 2 sum_i ||a_i||^4)
    / (m ||A^T A||_F^2).  Derivation: A^T S^T S A - A^T A = sum_{i != j}
    sigma_i sigma_j [h(i) = h(j)] a_i a_j^T, whose terms are uncorrelated except
    (i, j) with (j, i); P[h(i) = h(j)] = 1/m, and the s independent blocks of
    the SJLT each contribute (s/m)(...) scaled by 1/s^2."""
    A = as_f64(A)
    if isinstance(A, CSR):
        raise TypeError("dense A only")
    A = np.asarray(A)
    G = A.T @ A
    row2 = np.einsum("ij,ij->i", A, A)
    fro2 = float(row2.sum())
    num = fro2 * fro2 + float(np.sum(G * G)) - 2.0 * float(np.sum(row2 * row2))
    return num / (m * float(np.sum(G * G)))
