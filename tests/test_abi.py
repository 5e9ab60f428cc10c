"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a,
loads, and exports every function that include/ihs.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ihs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?\**\s*\b(ihs_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ihs_create", "ihs_sketch", "ihs_step", "ihs_solve", "ihs_gradient",
                     "ihs_adjoint", "ihs_destroy", "ihs_hash", "ihs_sketch_adjoint",
                     "ihs_get_sketch", "ihs_status_str", "ihs_sync"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1910_14166_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.ihs_status_str.restype = ctypes.c_char_p
    assert lib.ihs_status_str(0) == b"ok"
    assert b"positive definite" in lib.ihs_status_str(4)


def test_library_is_built_for_sm103a():
    """The fatbin carries sm_103a code (cuobjdump --list-elf lists the ELF
    names; only the architecture list is read)."""
    import shutil
    import subprocess
    from paper_1910_14166_gb300 import build
    path = build.build()
    tool = shutil.which("cuobjdump") or "/usr/local/cuda/bin/cuobjdump"
    if not os.path.exists(tool):
        return
    out = subprocess.run([tool, "--list-elf", path], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_python_binding_rejects_cpu_tensors():
    import pytest
    import torch
    import paper_1910_14166_gb300 as ihs
    with pytest.raises(TypeError):
        ihs.IHS(torch.zeros(10, 2), torch.zeros(10, dtype=torch.float64))


def header_enums():
    """Every NAME = value of the header's enums."""
    src = open(os.path.join(ROOT, "include", "ihs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    vals = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            if "=" in item:
                name, v = (t.strip() for t in item.split("="))
                nxt = int(v)
            else:
                name = item
            vals[name] = nxt
            nxt += 1
    return vals


def test_binding_constants_match_the_header():
    """The Python binding marshals the same codes the header defines: status
    codes, storage kinds, constraint kinds, precisions, sketches, option flags
    and profiling stages."""
    import paper_1910_14166_gb300 as ihs
    h = header_enums()
    for code, name in ihs.STATUS_NAMES.items():
        assert h[name] == code, name
    assert (h["IHS_DENSE"], h["IHS_CSR"], h["IHS_F64"], h["IHS_F32"]) == (
        ihs.DENSE, ihs.CSR, ihs.F64, ihs.F32)
    kinds = {"ols": "IHS_OLS", "l1": "IHS_L1_BALL", "ridge": "IHS_RIDGE",
             "l1pen": "IHS_L1_PENALTY", "l2": "IHS_L2_BALL"}
    for k, name in kinds.items():
        assert ihs.KIND[k] == h[name], k
    for p, name in {"fp64": "IHS_PREC_FP64", "tf32": "IHS_PREC_TF32",
                    "bf16": "IHS_PREC_BF16"}.items():
        assert ihs.PREC[p] == h[name], p
    for sk, name in {"sparse": "IHS_SKETCH_SPARSE", "srht": "IHS_SKETCH_SRHT",
                     "gaussian": "IHS_SKETCH_GAUSSIAN"}.items():
        assert ihs.SKETCH[sk] == h[name], sk
    assert ihs.option_flags() == 0
    assert ihs.option_flags(fuse=False) == h["IHS_FLAG_NO_FUSE"]
    assert ihs.option_flags(serial=True) == h["IHS_FLAG_SERIAL"]
    assert ihs.option_flags(cluster=True) == h["IHS_FLAG_CLUSTER"]
    assert ihs.option_flags(lookahead=False) == h["IHS_FLAG_NO_LOOKAHEAD"]
    assert ihs.option_flags(graph=False) == h["IHS_FLAG_NO_GRAPH"]
    assert ihs.option_flags(fp64_factor=True) == h["IHS_FLAG_FP64_FACTOR"]
    assert ihs.option_flags(False, True, True, False, True) == 31
    stages = [n for n in sorted(h, key=h.get) if n.startswith("IHS_ST_") and n != "IHS_ST_COUNT"]
    assert [s[len("IHS_ST_"):].lower() for s in stages[:len(ihs.STAGES)]] == ihs.STAGES


def test_create_rejects_invalid_options_before_touching_the_device():
    """ihs_create's argument checks run on the host before any CUDA call:
    unknown flag bits, an unknown sketch, m not divisible by s, m < d, an
    unknown constraint kind and a non-positive ball radius each return
    IHS_ERR_ARG (the device pointers are never dereferenced)."""
    import paper_1910_14166_gb300 as ihs
    lib = ihs._lib
    M = ihs._Matrix()
    M.kind, M.dtype, M.n, M.d, M.ld = ihs.DENSE, ihs.F32, 1000, 10, 10
    M.val = 0x1000  # never read: every case fails a host-side check first
    b = ctypes.c_void_p(0x2000)

    def create(flags=0, sketch=0, m=100, s=1, kind=ihs.OLS, param=0.0):
        C = ihs._Constraint(kind, param)
        O = ihs._Options(m, s, 0, 1, 0, 0.0, flags, sketch)
        h = ctypes.c_void_p()
        return lib.ihs_create(ctypes.byref(h), ctypes.byref(M), b, ctypes.byref(C),
                              ctypes.byref(O), None)

    ERR_ARG = 1
    assert create(flags=64) == ERR_ARG
    assert create(flags=1 << 30) == ERR_ARG
    assert create(sketch=3) == ERR_ARG
    assert create(m=101, s=2) == ERR_ARG
    assert create(m=5) == ERR_ARG
    assert create(kind=7) == ERR_ARG
    assert create(kind=ihs.L1_BALL, param=0.0) == ERR_ARG
    assert create(sketch=1, s=2, m=100) == ERR_ARG


def test_entry_points_reject_bad_arguments_before_touching_the_device():
    """Every entry point checks its arguments on the host before its first
    CUDA call: a null context, a negative counter or size, s not dividing m,
    more than 2^31 buckets and null buffers return IHS_ERR_ARG (1), and an
    oversize d returns IHS_ERR_UNSUPPORTED (8), with no device in this
    process.  A null context passed to ihs_destroy is a no-op."""
    import paper_1910_14166_gb300 as ihs
    lib = ihs._lib
    ERR_ARG, UNSUPPORTED = 1, 8
    buf = ctypes.c_void_p(0x1000)  # never dereferenced: each call fails a host check first
    dbl, i32, i64 = ctypes.c_double(), ctypes.c_int(), ctypes.c_int64()
    rep = ihs._Report()
    ms = (ctypes.c_double * 8)()

    assert lib.ihs_sketch(None, 0) == ERR_ARG
    assert lib.ihs_gradient(None, buf, buf, None) == ERR_ARG
    assert lib.ihs_sketch_gradient(None, 0, buf, buf) == ERR_ARG
    assert lib.ihs_step(None, buf) == ERR_ARG
    assert lib.ihs_sync(None) == ERR_ARG
    assert lib.ihs_solve(None, buf, 0, 1, ctypes.byref(rep)) == ERR_ARG
    assert lib.ihs_get_sketch(None, None, ctypes.byref(i32), None, ctypes.byref(dbl)) == ERR_ARG
    assert lib.ihs_exact_gram(None, buf) == ERR_ARG
    assert lib.ihs_sketch_error(None, 0, buf, ctypes.byref(dbl)) == ERR_ARG
    assert lib.ihs_adjoint(None, buf, buf, buf, None, ctypes.byref(rep)) == ERR_ARG
    assert lib.ihs_profile(None, 1) == ERR_ARG
    assert lib.ihs_profile_read(None, ms, None, ctypes.byref(i64)) == ERR_ARG
    lib.ihs_destroy(None)

    # stateless draw and gather: (seed, t, s, m, n)
    for s, m, n, t in ((0, 10, 5, 0), (65, 130, 5, 0), (3, 10, 5, 0), (1, 10, -1, 0),
                       (1, 10, 5, -1), (1, 1 << 31, 5, 0)):
        assert lib.ihs_hash(0, t, s, m, n, buf, buf, None) == ERR_ARG, (s, m, n, t)
    assert lib.ihs_hash(0, 0, 1, 10, 5, None, buf, None) == ERR_ARG
    assert lib.ihs_sketch_adjoint(0, 0, 1, 10, 5, 0, buf, buf, None) == ERR_ARG
    assert lib.ihs_sketch_adjoint(0, 0, 2, 10, 5, 3, None, buf, None) == ERR_ARG
    assert lib.ihs_sketch_adjoint(0, 0, 3, 10, 5, 3, buf, buf, None) == ERR_ARG

    # self-test of the pivot root: nothing to do for n = 0, null buffers refused
    assert lib.ihs_selftest_rsqrt(None, None, None, 0, None) == 0
    assert lib.ihs_selftest_rsqrt(None, buf, buf, 4, None) == ERR_ARG

    # no-allocation gradient
    M = ihs._Matrix()
    M.kind, M.dtype, M.n, M.d, M.ld, M.val = ihs.DENSE, ihs.F32, 100, 8, 8, 0x1000
    assert lib.ihs_gradient_noalloc(None, buf, buf, 0.0, buf, None) == ERR_ARG
    assert lib.ihs_gradient_noalloc(ctypes.byref(M), None, buf, 0.0, buf, None) == ERR_ARG
    M.ld = 7
    assert lib.ihs_gradient_noalloc(ctypes.byref(M), buf, buf, 0.0, buf, None) == ERR_ARG
    M.ld, M.kind = 8, ihs.CSR
    assert lib.ihs_gradient_noalloc(ctypes.byref(M), buf, buf, 0.0, buf, None) == ERR_ARG
    M.kind, M.d, M.ld = ihs.DENSE, 1025, 1025
    assert lib.ihs_gradient_noalloc(ctypes.byref(M), buf, buf, 0.0, buf, None) == UNSUPPORTED


def test_create_reports_unsupported_sizes_before_touching_the_device():
    """Sizes the library does not handle return IHS_ERR_UNSUPPORTED (8) from
    ihs_create's host-side checks: d > 1024, a dense s * n of 2^31 or more,
    and the SRHT over a CSR matrix (no device in this process)."""
    import paper_1910_14166_gb300 as ihs
    lib = ihs._lib
    UNSUPPORTED = 8
    b = ctypes.c_void_p(0x2000)

    def create(M, m, s, sketch=0):
        C = ihs._Constraint(ihs.OLS, 0.0)
        O = ihs._Options(m, s, 0, 1, 0, 0.0, 0, sketch)
        h = ctypes.c_void_p()
        return lib.ihs_create(ctypes.byref(h), ctypes.byref(M), b, ctypes.byref(C),
                              ctypes.byref(O), None)

    M = ihs._Matrix()
    M.kind, M.dtype, M.n, M.d, M.ld, M.val = ihs.DENSE, ihs.F32, 1000, 1025, 1025, 0x1000
    assert create(M, 2050, 1) == UNSUPPORTED
    M.n, M.d, M.ld = 1 << 26, 10, 10
    assert create(M, 640, 64) == UNSUPPORTED
    M.kind, M.n, M.col, M.rowptr, M.nnz = ihs.CSR, 1000, 0x3000, 0x4000, 2000
    assert create(M, 100, 1, sketch=1) == UNSUPPORTED
