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
