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


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes mirror of a struct in include/lra.h has the C compiler's size
    and field offsets (a field added on one side only would make the library
    read the caller's arguments at the wrong places)."""
    import shutil
    import subprocess
    import paper_1710_07946_gb300 as lra
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    mirrors = {"lra_problem": lra._Problem, "lra_ca_params": lra._Params, "lra_batch": lra._Batch,
               "lra_cur_batch": lra._CurBatch, "lra_hmatrix": lra._HMatrix, "lra_gauss_blocks": lra._Gauss,
               "lra_cur": lra._Cur}
    lines = ['#include <stdio.h>', '#include "lra.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_new_arguments_rejected_without_gpu():
    """The CTA-pair count, the stage tuner's schedules and the single-LRA grid size
    are checked on the host, before any CUDA call."""
    import numpy as np
    import paper_1710_07946_gb300 as lra
    L = lra._load()
    nb, k = 4, 8
    X = np.zeros((64, 3))                           # never read: the calls stop at the host checks
    pc = lra._Problem()
    pc.src, pc.dtype, pc.m, pc.n = 1, 0, 64, 64     # Laplace kernel, FP64 entries
    pc.X = pc.Y = X.ctypes.data
    blocks = np.array([[0, 16, 16, 16]] * nb, dtype=np.int64)
    offs = np.zeros((nb, 2), dtype=np.int64)
    cb = lra._Batch()
    cb.blocks, cb.offsets, cb.nb, cb.max_len = blocks.ctypes.data, offs.ctypes.data, nb, 16
    par = lra._params(k, 2, 1.05, 1e-6, 100, lra.LRA_MODE_FP64)
    dummy = np.zeros(4096, dtype=np.float64)
    cur = lra._CurBatch()
    for f in ("I", "J", "C", "U", "R", "logvol", "info"):
        setattr(cur, f, dummy.ctypes.data)
    I0 = np.zeros((nb, k), dtype=np.int32)
    cb.pair_blocks = nb + 1                          # more pair blocks than blocks
    assert L.lra_ca_run_batched(ctypes.byref(pc), ctypes.byref(cb), ctypes.byref(par), I0.ctypes.data,
                                ctypes.byref(cur), dummy.ctypes.data, dummy.nbytes, None) == lra.LRA_ERR_INVALID_ARG
    cb.pair_blocks = -1
    assert L.lra_ca_run_batched(ctypes.byref(pc), ctypes.byref(cb), ctypes.byref(par), I0.ctypes.data,
                                ctypes.byref(cur), dummy.ctypes.data, dummy.nbytes, None) == lra.LRA_ERR_INVALID_ARG
    cb.pair_blocks = 0
    Q = np.zeros((nb, 2), dtype=np.int32)
    best = ctypes.c_int32()
    for sched in ([[2, 2, 4, 6] + [0] * 6], [[0, 2] + [0] * 8], [[2, -1, 4, 8] + [0] * 6]):
        tab = np.array(sched, dtype=np.int32)     # sizes not ending at k; no sizes; negative margin
        st = L.lra_ca_batched_tune_stages(ctypes.byref(pc), None, ctypes.byref(cb), ctypes.byref(par),
                                          I0.ctypes.data, ctypes.byref(cur), dummy.ctypes.data, dummy.nbytes,
                                          Q.ctypes.data, 2, Q.ctypes.data, 2, dummy.ctypes.data, 1e-6,
                                          tab.ctypes.data, len(tab), 1, None, ctypes.byref(best), None, None)
        assert st == lra.LRA_ERR_INVALID_ARG, sched
    p1 = lra._params(k, 2, 1.05, 1e-6, 100, lra.LRA_MODE_FP64, ctas=-1)
    pc1 = lra._Problem()
    pc1.src, pc1.dtype, pc1.m, pc1.n = 1, 0, 64, 64
    pc1.X = pc1.Y = X.ctypes.data
    size = ctypes.c_size_t()
    assert L.lra_ca_workspace_size(ctypes.byref(pc1), ctypes.byref(p1), None, ctypes.byref(size)) == \
        lra.LRA_ERR_INVALID_ARG
