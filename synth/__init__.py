"""Seeded synthetic inputs shaped like the workloads of the IHS paper.

This module only draws data: it holds none of the method's arithmetic, and
both the GPU library's tests and the CPU oracle take their inputs from here.
The paper's own datasets (Table "datasets", App. B) are not available; these
recipes stand in for them:

  ols_dense_fp64   A n x d iid N(0,1) FP64, b = A x* + N(0,1)          (20000 x 50)
  lasso_csr_fp64   CSR n x d, exactly k nnz/row at uniform distinct
                   columns, values N(0,1) FP64; x* with d/10 nonzeros;
                   R = ||x*||_1 / 2                                     (1e6 x 200, k = 2)
  ols_dense_ar1    A n x d FP32 with rows N(0, Sigma), Sigma_ij = rho^|i-j|,
                   drawn by the AR(1) recurrence over columns;
                   b = A x* + 0.1 N(0,1) in FP64                        (1048576 x 500)
  ridge_dense      A n x d FP32 iid N(0,1), b = A x* + N(0,1),
                   x_target ~ N(0, I) from a second seed                (262144 x 256)
  lasso_csr_zipf   CSR n x d, exactly k nnz/row, distinct columns drawn
                   by Zipf(alpha) over column ranks (rank -> column by a
                   seeded permutation, duplicates in a row redrawn),
                   values N(0,1) FP32; x* with 100 nonzeros; R = ||x*||_1/2
                                                                        (1e7 x 1000, k = 5)
Every generator is a pure function of its arguments (numpy PCG64).
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def dense_gaussian(n, d, seed, dtype=np.float64):
    rng = _rng(seed)
    return rng.standard_normal((n, d), dtype=np.float64).astype(dtype, copy=False)


def dense_ar1(n, d, rho, seed, dtype=np.float32):
    """Rows N(0, Sigma) with Sigma_ij = rho^|i-j|: a_1 = z_1,
    a_j = rho a_{j-1} + sqrt(1 - rho^2) z_j, computed in FP32 column by column."""
    rng = _rng(seed)
    A = np.empty((n, d), dtype=np.float32)
    c = np.float32(np.sqrt(1.0 - rho * rho))
    r = np.float32(rho)
    prev = rng.standard_normal(n, dtype=np.float32)
    A[:, 0] = prev
    for j in range(1, d):
        z = rng.standard_normal(n, dtype=np.float32)
        prev = r * prev + c * z
        A[:, j] = prev
    return A.astype(dtype, copy=False)


def csr_uniform(n, d, k, seed, dtype=np.float64):
    """Exactly k nonzeros per row at distinct uniformly chosen columns (sorted)."""
    rng = _rng(seed)
    cols = np.empty((n, k), dtype=np.int32)
    todo = np.arange(n)
    while todo.size:
        c = rng.integers(0, d, size=(todo.size, k), dtype=np.int32)
        c.sort(axis=1)
        ok = np.all(c[:, 1:] != c[:, :-1], axis=1) if k > 1 else np.ones(todo.size, bool)
        cols[todo[ok]] = c[ok]
        todo = todo[~ok]
    val = rng.standard_normal(n * k).astype(dtype)
    rowptr = np.arange(0, n * k + 1, k, dtype=np.int64)
    return rowptr, cols.reshape(-1), val


def zipf_probs(d, alpha):
    p = np.arange(1, d + 1, dtype=np.float64) ** (-alpha)
    return p / p.sum()


def csr_zipf(n, d, k, alpha, seed, dtype=np.float32):
    """Exactly k nonzeros per row; column ranks ~ Zipf(alpha) over 1..d mapped to
    columns by a seeded permutation; rows with a repeated column are redrawn."""
    rng = _rng(seed)
    perm = rng.permutation(d).astype(np.int32)
    cdf = np.cumsum(zipf_probs(d, alpha))
    cdf[-1] = 1.0
    cols = np.empty((n, k), dtype=np.int32)
    todo = np.arange(n)
    while todo.size:
        u = rng.random((todo.size, k))
        c = perm[np.searchsorted(cdf, u, side="right").clip(0, d - 1)]
        c.sort(axis=1)
        ok = np.all(c[:, 1:] != c[:, :-1], axis=1) if k > 1 else np.ones(todo.size, bool)
        cols[todo[ok]] = c[ok]
        todo = todo[~ok]
    val = rng.standard_normal(n * k).astype(dtype)
    rowptr = np.arange(0, n * k + 1, k, dtype=np.int64)
    return rowptr, cols.reshape(-1), val


def _csr_matvec(n, rowptr, col, val, x):
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    out = np.zeros(n)
    np.add.at(out, rows, val.astype(np.float64) * x[col])
    return out


def sparse_truth(d, nnz, seed):
    rng = _rng(seed)
    x = np.zeros(d)
    sup = rng.choice(d, size=nnz, replace=False)
    x[sup] = rng.standard_normal(nnz)
    return x


# --------------------------------------------------------------------------
# The five workloads.  `n` (and for the sparse ones `d`) may be scaled down
# for tests; the defaults are the full sizes.
# --------------------------------------------------------------------------
WORKLOADS = {
    "ols_dense_fp64": dict(n=20000, d=50, m=500, s=1, iters=10, kind="ols", precision="fp64"),
    "lasso_csr_fp64": dict(n=1_000_000, d=200, m=2000, s=4, iters=15, kind="l1", precision="fp64"),
    "ols_dense_ar1": dict(n=1_048_576, d=500, m=5000, s=1, iters=0, kind="ols", precision="tf32"),
    "ridge_dense": dict(n=262_144, d=256, m=2560, s=1, iters=0, kind="ridge", precision="tf32"),
    "lasso_csr_zipf": dict(n=10_000_000, d=1000, m=10000, s=8, iters=20, kind="l1", precision="tf32"),
}


def make(name, n=None, d=None, m=None, seed=0):
    """Draw one workload.  Returns a dict with the matrix (dense ndarray, or
    CSR arrays rowptr/col/val), b (FP64), x_star, and the method parameters."""
    w = dict(WORKLOADS[name])
    if n is not None:
        w["n"] = int(n)
    if d is not None:
        w["d"] = int(d)
    if m is not None:
        w["m"] = int(m)
    n, d = w["n"], w["d"]
    out = dict(name=name, **w)
    rng = _rng(seed + 1_000_003)
    if name == "ols_dense_fp64":
        A = dense_gaussian(n, d, seed, np.float64)
        xs = rng.standard_normal(d)
        b = A @ xs + rng.standard_normal(n)
        out.update(A=A, b=b, x_star=xs, param=0.0)
    elif name == "lasso_csr_fp64":
        rowptr, col, val = csr_uniform(n, d, 2, seed, np.float64)
        xs = sparse_truth(d, max(1, d // 10), seed + 7)
        b = _csr_matvec(n, rowptr, col, val, xs) + rng.standard_normal(n)
        out.update(rowptr=rowptr, col=col, val=val, b=b, x_star=xs, param=0.5 * np.abs(xs).sum())
    elif name == "ols_dense_ar1":
        A = dense_ar1(n, d, 0.5, seed)
        xs = rng.standard_normal(d)
        b = A.astype(np.float64) @ xs + 0.1 * rng.standard_normal(n)
        out.update(A=A, b=b, x_star=xs, param=0.0)
    elif name == "ridge_dense":
        A = dense_gaussian(n, d, seed, np.float32)
        xs = rng.standard_normal(d)
        b = A.astype(np.float64) @ xs + rng.standard_normal(n)
        xt = _rng(seed + 1).standard_normal(d)
        out.update(A=A, b=b, x_star=xs, x_target=xt, param=1e-3)
    elif name == "lasso_csr_zipf":
        rowptr, col, val = csr_zipf(n, d, 5, 1.1, seed, np.float32)
        xs = sparse_truth(d, min(100, d), seed + 7)
        b = _csr_matvec(n, rowptr, col, val, xs) + rng.standard_normal(n)
        out.update(rowptr=rowptr, col=col, val=val, b=b, x_star=xs, param=0.5 * np.abs(xs).sum())
    else:
        raise KeyError(name)
    return out
