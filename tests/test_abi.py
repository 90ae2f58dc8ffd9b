"""The C-ABI library builds for sm_103a and exports every entry point that
include/lra.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(lra_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("lra_precondition", "lra_multiplier_destroy", "lra_ca_workspace_size", "lra_ca_run",
              "lra_cur_apply", "lra_residual_sample", "lra_version"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1710_07946_gb300 import build
    lib = build.build()
    L = ctypes.CDLL(lib)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    L.lra_version.restype = ctypes.c_char_p
    assert b"sm_103a" in L.lra_version()


def test_host_validation_without_gpu():
    """Argument checks run on the host before any CUDA call."""
    from paper_1710_07946_gb300 import build
    L = ctypes.CDLL(build.build())
    L.lra_precondition.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                   ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    L.lra_precondition.restype = ctypes.c_int
    h = ctypes.c_void_p()
    # bad kind, bad depth, n not a multiple of 2^d
    assert L.lra_precondition(ctypes.byref(h), 7, 0, 8, 1, None, None) == 1
    import numpy as np
    perm = np.arange(6, dtype=np.int32); sg = np.ones(6, dtype=np.int8)
    assert L.lra_precondition(ctypes.byref(h), 1, 0, 6, 2, perm.ctypes.data, sg.ctypes.data) == 1
    # bad side
    assert L.lra_precondition(ctypes.byref(h), 1, 2, 6, 1, perm.ctypes.data, sg.ctypes.data) == 1
    bad = perm.copy(); bad[0] = 1
    assert L.lra_precondition(ctypes.byref(h), 1, 0, 6, 1, bad.ctypes.data, sg.ctypes.data) == 1
    # unsorted sparse rows
    rows = np.array([[1, 0]], dtype=np.int32).repeat(3, 0); s2 = np.ones((3, 2), np.int8)
    assert L.lra_precondition(ctypes.byref(h), 2, 0, 3, 2, rows.ctypes.data, s2.ctypes.data) == 1
