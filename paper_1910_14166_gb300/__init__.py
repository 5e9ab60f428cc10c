"""Python binding of libihs.so, the GB300 Iterative Hessian Sketch library
(Cormode & Dickens, "Iterative Hessian Sketch in Input Sparsity Time",
arXiv 1910.14166).

The binding only marshals arguments: every step of the method runs in the
library's CUDA kernels, reached through the C ABI declared in include/ihs.h
(same function names).  PyTorch supplies device memory and the current CUDA
stream.  There is no CPU fallback: if the library cannot be built or loaded,
importing this package raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

IHS_OK = 0
STATUS_NAMES = {0: "IHS_OK", 1: "IHS_ERR_ARG", 2: "IHS_ERR_CUDA", 3: "IHS_ERR_OOM",
                4: "IHS_ERR_NOT_SPD", 5: "IHS_ERR_NOT_CONVERGED", 6: "IHS_ERR_NONFINITE",
                7: "IHS_ERR_TIMEOUT", 8: "IHS_ERR_UNSUPPORTED"}
DENSE, CSR = 0, 1
F64, F32 = 0, 1
OLS, L1_BALL, RIDGE, L1_PENALTY, L2_BALL = 0, 1, 2, 3, 4
PREC = {"fp64": 0, "tf32": 1, "bf16": 2}
KIND = {"ols": OLS, "l1": L1_BALL, "ridge": RIDGE, "l1pen": L1_PENALTY, "l2": L2_BALL}
SKETCH = {"sparse": 0, "srht": 1, "gaussian": 2}
FLAG_NO_FUSE, FLAG_SERIAL, FLAG_CLUSTER, FLAG_NO_LOOKAHEAD, FLAG_FP64_FACTOR = 1, 2, 4, 8, 16
FLAG_NO_GRAPH = 32


def option_flags(fuse=True, serial=False, cluster=False, lookahead=True, fp64_factor=False,
                 graph=True):
    """The IHS_FLAG_* word of ihs_options for IHS()'s keyword options."""
    return ((0 if fuse else FLAG_NO_FUSE) | (FLAG_SERIAL if serial else 0)
            | (FLAG_CLUSTER if cluster else 0) | (0 if lookahead else FLAG_NO_LOOKAHEAD)
            | (FLAG_FP64_FACTOR if fp64_factor else 0) | (0 if graph else FLAG_NO_GRAPH))


class IHSError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        msg = _lib.ihs_status_str(self.status).decode() if _lib else str(status)
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(self.status, "?"), msg))


class _Matrix(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dtype", ctypes.c_int), ("n", ctypes.c_int64),
                ("d", ctypes.c_int64), ("ld", ctypes.c_int64), ("val", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("rowptr", ctypes.c_void_p),
                ("rowptr_i64", ctypes.c_int), ("nnz", ctypes.c_int64)]


class _Constraint(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("param", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("s", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int), ("qp_max_iter", ctypes.c_int),
                ("qp_tol", ctypes.c_double), ("flags", ctypes.c_int), ("sketch", ctypes.c_int)]


class _Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("qp_fista_iters", ctypes.c_int),
                ("status", ctypes.c_int), ("step_norm", ctypes.c_double),
                ("qp_active_rounds", ctypes.c_int), ("graph", ctypes.c_int)]


def _load():
    path = _build.build()
    L = ctypes.CDLL(path)
    vp, i64, i32, u64, f64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                              ctypes.c_double)
    sig = {
        "ihs_create": [ctypes.POINTER(vp), ctypes.POINTER(_Matrix), vp,
                       ctypes.POINTER(_Constraint), ctypes.POINTER(_Options), vp],
        "ihs_sketch": [vp, i64],
        "ihs_gradient": [vp, vp, vp, vp],
        "ihs_sketch_gradient": [vp, i64, vp, vp],
        "ihs_step": [vp, vp],
        "ihs_solve": [vp, vp, i64, i32, ctypes.POINTER(_Report)],
        "ihs_sync": [vp],
        "ihs_get_sketch": [vp, vp, ctypes.POINTER(i32), vp, ctypes.POINTER(f64)],
        "ihs_adjoint": [vp, vp, vp, vp, vp, ctypes.POINTER(_Report)],
        "ihs_hash": [u64, i64, i32, i64, i64, vp, vp, vp],
        "ihs_sketch_adjoint": [u64, i64, i32, i64, i64, i64, vp, vp, vp],
        "ihs_profile": [vp, i32],
        "ihs_profile_read": [vp, ctypes.POINTER(f64), ctypes.POINTER(i32), ctypes.POINTER(i64)],
        "ihs_gradient_noalloc": [ctypes.POINTER(_Matrix), vp, vp, f64, vp, vp],
        "ihs_exact_gram": [vp, vp],
        "ihs_trim_memory": [],
        "ihs_selftest_wait": [vp],
        "ihs_selftest_rsqrt": [vp, vp, vp, i64, vp],
        "ihs_sketch_error": [vp, i64, vp, ctypes.POINTER(f64)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.ihs_destroy.argtypes = [vp]
    L.ihs_destroy.restype = None
    L.ihs_status_str.argtypes = [ctypes.c_int]
    L.ihs_status_str.restype = ctypes.c_char_p
    return L


_lib = _load()
LIB_PATH = _build.LIB
STAGES = ["sort", "sketch", "sketch_fix", "gram", "factor", "grad", "step"]
EXPORTS = ["ihs_create", "ihs_sketch", "ihs_gradient", "ihs_sketch_gradient", "ihs_step",
           "ihs_solve", "ihs_sync", "ihs_get_sketch", "ihs_adjoint", "ihs_destroy", "ihs_status_str", "ihs_hash",
           "ihs_sketch_adjoint", "ihs_profile", "ihs_profile_read", "ihs_gradient_noalloc"]


def _check(st, where):
    if st != IHS_OK:
        raise IHSError(st, where)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need_cuda(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def _need(t, name, shape, dtypes, device):
    """Checks the C ABI cannot make (it sees bare pointers): a contiguous CUDA
    tensor of this shape, one of these dtypes, on this device."""
    _need_cuda(t, name)
    if t.dtype not in dtypes:
        raise TypeError("%s must be %s" % (name, "/".join(str(x).replace("torch.", "")
                                                           for x in dtypes)))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, not %s" % (name, tuple(shape), tuple(t.shape)))
    if t.device != device:
        raise ValueError("%s must be on %s, not %s" % (name, device, t.device))


_F64 = (torch.float64,)


def ihs_hash(seed, t, s, m, n):
    """Sketch draw of Sec. 2 on the GPU: (bucket int32 [s, n], sign int8 [s, n])."""
    bucket = torch.empty((s, n), dtype=torch.int32, device="cuda")
    sign = torch.empty((s, n), dtype=torch.int8, device="cuda")
    _check(_lib.ihs_hash(seed & 0xFFFFFFFFFFFFFFFF, t, s, m, n, _ptr(bucket), _ptr(sign), _stream()),
           "ihs_hash")
    return bucket, sign


def ihs_sketch_adjoint(seed, t, s, m, n, G):
    """S^T G (n x d FP64) for the normalised sketch of counter t; G is m x d
    (its rows are gathered by bucket, so it must hold all m of them)."""
    _need_cuda(G, "G")
    if G.dim() != 2 or G.shape[0] != m:
        raise ValueError("G must be a 2-D tensor with m = %d rows" % m)
    G = G.to(torch.float64)
    with torch.cuda.device(G.device):
        out = torch.empty((n, G.shape[1]), dtype=torch.float64, device=G.device)
        _check(_lib.ihs_sketch_adjoint(seed & 0xFFFFFFFFFFFFFFFF, t, s, m, n, G.shape[1],
                                       _ptr(G), _ptr(out), _stream()), "ihs_sketch_adjoint")
    return out


def ihs_gradient_noalloc(A, b, x, lam=0.0):
    """g = A^T (b - A x) - lam x for a dense CUDA tensor A, through the entry
    point that allocates no device memory inside the library (its scratch is
    a fixed array in the library; see include/ihs.h).  Only the output g is
    allocated here, by the caller's side (PyTorch).

    The C entry point cannot see tensor types or lengths, so they are checked
    here before anything is launched: A 2-D float32/float64, b float64 with
    A.shape[0] entries, x float64 with A.shape[1], all on one device; the call
    runs with that device current."""
    for t_, nm in ((A, "A"), (b, "b"), (x, "x")):
        _need_cuda(t_, nm)
    if A.dim() != 2 or A.dtype not in (torch.float32, torch.float64):
        raise TypeError("A must be a 2-D float32/float64 tensor")
    if b.dtype != torch.float64 or x.dtype != torch.float64:
        raise TypeError("b and x must be float64")
    if b.dim() != 1 or b.numel() != A.shape[0]:
        raise ValueError("b must hold A.shape[0] = %d values" % A.shape[0])
    if x.dim() != 1 or x.numel() != A.shape[1]:
        raise ValueError("x must hold A.shape[1] = %d values" % A.shape[1])
    if b.device != A.device or x.device != A.device:
        raise ValueError("A, b and x must be on one device")
    M = _Matrix()
    M.kind, M.n, M.d, M.ld = DENSE, A.shape[0], A.shape[1], max(A.stride(0), A.shape[1])
    M.dtype = F32 if A.dtype == torch.float32 else F64
    M.val = A.data_ptr() if A.numel() else None
    with torch.cuda.device(A.device):
        g = torch.empty(A.shape[1], dtype=torch.float64, device=A.device)
        _check(_lib.ihs_gradient_noalloc(ctypes.byref(M), _ptr(b) if b.numel() else None,
                                         _ptr(x), float(lam), _ptr(g), _stream()),
               "ihs_gradient_noalloc")
    return g


def trim_memory():
    """Return the library's cached device workspace memory to the device
    (contexts keep reusing it otherwise; see ihs_trim_memory)."""
    _check(_lib.ihs_trim_memory(), "ihs_trim_memory")


def selftest_rsqrt(p):
    """The FP64 Cholesky's pivot reciprocal square root and CUDA's rsqrt of
    each entry of p (a CUDA float64 tensor of positive finite values), as two
    new tensors (ours, CUDA's)."""
    _need_cuda(p, "p")
    if p.dtype != torch.float64:
        raise TypeError("p must be float64")
    p = p.contiguous()
    out, ref = torch.empty_like(p), torch.empty_like(p)
    _check(_lib.ihs_selftest_rsqrt(_ptr(p), _ptr(out), _ptr(ref), p.numel(), _stream()),
           "ihs_selftest_rsqrt")
    return out, ref


def selftest_wait():
    """Run the bounded-wait self-test on the current stream and return its
    status code (IHS_ERR_TIMEOUT = 7 when the wait gave up as designed)."""
    return int(_lib.ihs_selftest_wait(_stream()))


class IHS:
    """One problem (A, b, C) of Eq. 1 with its workspaces on the GPU.

    A: a 2-D CUDA tensor (float32 or float64, row-major) or a CSR triple
    (rowptr int32/int64, col int32, val float32/float64) with shape=(n, d).
    b: CUDA float64 vector.  The tensors are borrowed and must outlive the
    object.  kind: 'ols', 'l1' (ball, param = radius), 'l1pen' (penalised,
    param = lambda), 'l2' (p = 2 ball, param = radius) or 'ridge' (param =
    lambda).
    precision: 'fp64' (plain), 'tf32' or 'bf16' (mixed).  fuse=False,
    serial=True, cluster=True, lookahead=False and fp64_factor=True set
    IHS_FLAG_NO_FUSE, IHS_FLAG_SERIAL, IHS_FLAG_CLUSTER, IHS_FLAG_NO_LOOKAHEAD
    and IHS_FLAG_FP64_FACTOR, and graph=False sets IHS_FLAG_NO_GRAPH; sketch:
    'sparse' (CountSketch / SJLT), 'srht' or 'gaussian' (the paper's dense
    comparisons)."""

    def __init__(self, A, b, kind="ols", param=0.0, m=None, s=1, seed=0, precision="fp64",
                 shape=None, qp_max_iter=0, qp_tol=0.0, fuse=True, serial=False, cluster=False,
                 sketch="sparse", lookahead=True, fp64_factor=False, graph=True):
        self._keep = [A, b]
        _need_cuda(b, "b")
        if b.dtype != torch.float64 or b.dim() != 1:
            raise TypeError("b must be a float64 vector")
        M = _Matrix()
        if isinstance(A, torch.Tensor):
            _need_cuda(A, "A")
            if A.dim() != 2 or A.dtype not in (torch.float32, torch.float64):
                raise TypeError("dense A must be a 2-D float32/float64 tensor")
            _need(b, "b", (A.shape[0],), _F64, A.device)
            M.kind, M.n, M.d = DENSE, A.shape[0], A.shape[1]
            M.ld = A.stride(0)
            M.dtype = F32 if A.dtype == torch.float32 else F64
            M.val = A.data_ptr()
            M.col = None
            M.rowptr = None
            M.nnz = A.numel()
        else:
            rowptr, col, val = A
            if shape is None:
                raise ValueError("CSR input needs shape=(n, d)")
            _need(b, "b", (shape[0],), _F64, b.device)
            _need(rowptr, "rowptr", (shape[0] + 1,), (torch.int32, torch.int64), b.device)
            _need(val, "val", (val.numel(),), (torch.float32, torch.float64), b.device)
            _need(col, "col", (val.numel(),), (torch.int32,), b.device)
            M.kind, M.n, M.d, M.ld = CSR, shape[0], shape[1], shape[1]
            M.dtype = F32 if val.dtype == torch.float32 else F64
            M.val, M.col, M.rowptr = val.data_ptr(), col.data_ptr(), rowptr.data_ptr()
            M.rowptr_i64 = 1 if rowptr.dtype == torch.int64 else 0
            M.nnz = val.numel()
        self.n, self.d = int(M.n), int(M.d)
        self.m = int(m if m is not None else 10 * self.d)
        self.s = int(s)
        self.kind = kind
        self.precision = precision
        C = _Constraint(KIND[kind], float(param))
        O = _Options(self.m, self.s, seed & 0xFFFFFFFFFFFFFFFF, PREC[precision], int(qp_max_iter),
                     float(qp_tol), option_flags(fuse, serial, cluster, lookahead, fp64_factor,
                                                 graph),
                     SKETCH[sketch])
        h = ctypes.c_void_p()
        self.device = b.device
        # the context keeps the stream current at creation: take b's device's
        with torch.cuda.device(self.device):
            _check(_lib.ihs_create(ctypes.byref(h), ctypes.byref(M), _ptr(b), ctypes.byref(C),
                                   ctypes.byref(O), _stream()), "ihs_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.ihs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _x(self, x, name="x"):
        _need(x, name, (self.d,), _F64, self.device)

    def sketch(self, t):
        with torch.cuda.device(self.device):
            _check(_lib.ihs_sketch(self._h, int(t)), "ihs_sketch")

    def gradient(self, x, want_r=False):
        self._x(x)
        with torch.cuda.device(self.device):
            g = torch.empty(self.d, dtype=torch.float64, device=self.device)
            r = torch.empty(self.n, dtype=torch.float64, device=self.device) if want_r else None
            _check(_lib.ihs_gradient(self._h, _ptr(x), _ptr(g), _ptr(r)), "ihs_gradient")
        return (r, g) if want_r else g

    def sketch_gradient(self, t, x):
        """Sketch of counter t (SA, Hessian, factor) and g at x from one pass
        over A where the fused pass applies (ihs_sketch_gradient)."""
        self._x(x)
        with torch.cuda.device(self.device):
            g = torch.empty(self.d, dtype=torch.float64, device=self.device)
            _check(_lib.ihs_sketch_gradient(self._h, int(t), _ptr(x), _ptr(g)),
                   "ihs_sketch_gradient")
        return g

    def step(self, x):
        self._x(x)
        with torch.cuda.device(self.device):
            _check(_lib.ihs_step(self._h, _ptr(x)), "ihs_step")

    def sync(self):
        with torch.cuda.device(self.device):
            _check(_lib.ihs_sync(self._h), "ihs_sync")

    def solve(self, x=None, t0=0, iters=10):
        if x is None:
            x = torch.zeros(self.d, dtype=torch.float64, device=self.device)
        self._x(x)
        rep = _Report()
        with torch.cuda.device(self.device):
            _check(_lib.ihs_solve(self._h, _ptr(x), int(t0), int(iters), ctypes.byref(rep)),
                   "ihs_solve")
        return x, rep

    def get_sketch(self):
        dt = ctypes.c_int()
        scale = ctypes.c_double()
        with torch.cuda.device(self.device):
            _check(_lib.ihs_get_sketch(self._h, None, ctypes.byref(dt), None,
                                       ctypes.byref(scale)), "ihs_get_sketch")
            SA = torch.empty((self.m, self.d),
                             dtype=torch.float64 if dt.value == F64 else torch.float32,
                             device=self.device)
            H = torch.empty((self.d, self.d), dtype=torch.float64, device=self.device)
            _check(_lib.ihs_get_sketch(self._h, _ptr(SA), ctypes.byref(dt), _ptr(H),
                                       ctypes.byref(scale)), "ihs_get_sketch")
        return SA, H, scale.value

    def exact_gram(self):
        """A^T A in FP64 (d x d CUDA tensor), computed by the library."""
        with torch.cuda.device(self.device):
            G = torch.empty((self.d, self.d), dtype=torch.float64, device=self.device)
            _check(_lib.ihs_exact_gram(self._h, _ptr(G)), "ihs_exact_gram")
        return G

    def sketch_error(self, t, G):
        """||(1/s)(S_t A)^T (S_t A) - G||_F / ||G||_F for the sketch of counter t."""
        _need(G, "G", (self.d, self.d), _F64, self.device)
        err = ctypes.c_double()
        with torch.cuda.device(self.device):
            _check(_lib.ihs_sketch_error(self._h, int(t), _ptr(G), ctypes.byref(err)),
                   "ihs_sketch_error")
        return err.value

    def profile(self, enable=True):
        """Enable stage timing (CUDA events on the context's stream) and reset totals."""
        _check(_lib.ihs_profile(self._h, 1 if enable else 0), "ihs_profile")

    def profile_read(self):
        """(ms per stage summed, instances per stage, library kernel launches)."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int * n)()
        launches = ctypes.c_int64()
        _check(_lib.ihs_profile_read(self._h, ms, cnt, ctypes.byref(launches)), "ihs_profile_read")
        return ({k: ms[i] for i, k in enumerate(STAGES)}, {k: cnt[i] for i, k in enumerate(STAGES)},
                launches.value)

    def adjoint(self, x, dLdx, want_A=True):
        self._x(x)
        self._x(dLdx, "dLdx")
        A = self._keep[0]
        rep = _Report()
        with torch.cuda.device(self.device):
            dLdb = torch.empty(self.n, dtype=torch.float64, device=self.device)
            dLdA = torch.empty_like(A) if (want_A and isinstance(A, torch.Tensor)) else None
            _check(_lib.ihs_adjoint(self._h, _ptr(x), _ptr(dLdx), _ptr(dLdb), _ptr(dLdA),
                                    ctypes.byref(rep)), "ihs_adjoint")
        return dLdb, dLdA, rep
