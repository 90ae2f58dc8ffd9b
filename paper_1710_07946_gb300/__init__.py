"""GB300 (sm_103a) library for superfast cross-approximation CUR low-rank
approximation (Pan, Luan, Svadlenka, Zhao, arXiv:1710.07946).

This module is the thin Python binding of the C ABI declared in include/lra.h:
the functions named ``lra_*`` marshal torch tensors (device memory, streams)
into the library's calls and do nothing else; every step of the computation
runs in the library's CUDA kernels.  There is no CPU fallback: importing the
binding without a built library, or calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass
from typing import Optional

import torch

from . import build as _build

__all__ = [
    "LRA_OK", "LRA_ERR_INVALID_ARG", "LRA_ERR_CUDA", "LRA_ERR_NONFINITE", "LRA_ERR_TIMEOUT", "LRA_ERR_WORKSPACE",
    "LRA_WARN_RANK_DEFICIENT", "LRA_WARN_NOT_CONVERGED", "LraError", "Problem", "Multiplier",
    "lra_precondition", "lra_precondition_fourier", "lra_multiplier_destroy", "lra_ca_workspace_size", "lra_ca_run", "lra_cur_apply",
    "lra_residual_sample", "lra_version", "library_path", "lra_launch_count", "lra_profile_enable",
    "lra_profile_collect", "lra_ca_run_noalloc", "Batch", "lra_ca_run_batched", "lra_residual_sample_batched",
    "lra_gauss_cur_forward", "lra_gauss_cur_backward", "GaussCurApply", "gauss_cur_apply",
]

LRA_OK, LRA_ERR_INVALID_ARG, LRA_ERR_CUDA, LRA_ERR_NONFINITE, LRA_ERR_TIMEOUT, LRA_ERR_WORKSPACE = 0, 1, 2, 3, 4, 5
LRA_WARN_RANK_DEFICIENT, LRA_WARN_NOT_CONVERGED = 16, 17
LRA_F64, LRA_F32, LRA_BF16 = 0, 1, 2
LRA_DENSE, LRA_KERNEL_LAPLACE, LRA_KERNEL_GAUSSIAN = 0, 1, 2
LRA_MULT_NONE, LRA_MULT_ARHT, LRA_MULT_SPARSE_PM1, LRA_MULT_BIDIAG, LRA_MULT_ARFT = 0, 1, 2, 3, 4
LRA_SIDE_RIGHT, LRA_SIDE_LEFT = 0, 1
LRA_MODE_FP64, LRA_MODE_MIXED = 0, 1
LRA_INFO_LEN = 8
LRA_MAX_STAGES = 8

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "NONFINITE", 4: "TIMEOUT", 5: "WORKSPACE",
           16: "WARN_RANK_DEFICIENT", 17: "WARN_NOT_CONVERGED"}


class LraError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}")
        self.status = status


class _Problem(ct.Structure):
    _fields_ = [("src", ct.c_int32), ("dtype", ct.c_int32), ("m", ct.c_int64), ("n", ct.c_int64),
                ("W", ct.c_void_p), ("ldw", ct.c_int64), ("X", ct.c_void_p), ("Y", ct.c_void_p),
                ("length_scale", ct.c_double)]


class _Params(ct.Structure):
    _fields_ = [("k", ct.c_int32), ("sweeps", ct.c_int32), ("h", ct.c_double), ("rank_tol", ct.c_double),
                ("max_swaps", ct.c_int32), ("mode", ct.c_int32), ("nstages", ct.c_int32),
                ("rank_margin", ct.c_int32), ("k_stages", ct.c_int32 * LRA_MAX_STAGES), ("ctas", ct.c_int32)]


class _Batch(ct.Structure):
    _fields_ = [("blocks", ct.c_void_p), ("offsets", ct.c_void_p), ("order", ct.c_void_p), ("nb", ct.c_int32),
                ("max_len", ct.c_int64), ("cta_threads", ct.c_int32), ("ctas_per_sm", ct.c_int32),
                ("pair_blocks", ct.c_int32)]


class _CurBatch(ct.Structure):
    _fields_ = [("I", ct.c_void_p), ("J", ct.c_void_p), ("C", ct.c_void_p), ("U", ct.c_void_p),
                ("R", ct.c_void_p), ("logvol", ct.c_void_p), ("info", ct.c_void_p), ("work", ct.c_void_p)]


class _HMatrix(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("levels", ct.c_int32), ("kmax", ct.c_int32), ("nfar", ct.c_int32),
                ("nfar_groups", ct.c_int32), ("nnear", ct.c_int32), ("nnear_groups", ct.c_int32),
                ("far", ct.c_void_p), ("far_offsets", ct.c_void_p), ("C", ct.c_void_p), ("U", ct.c_void_p),
                ("R", ct.c_void_p), ("info", ct.c_void_p), ("far_groups", ct.c_void_p), ("near", ct.c_void_p),
                ("near_groups", ct.c_void_p), ("I", ct.c_void_p), ("J", ct.c_void_p)]


class _Gauss(ct.Structure):
    _fields_ = [("X", ct.c_void_p), ("Y", ct.c_void_p), ("I", ct.c_void_p), ("J", ct.c_void_p),
                ("nb", ct.c_int32), ("m", ct.c_int32), ("n", ct.c_int32), ("k", ct.c_int32),
                ("length_scale", ct.c_double)]


class _Cur(ct.Structure):
    _fields_ = [("I", ct.c_void_p), ("J", ct.c_void_p), ("C", ct.c_void_p), ("U", ct.c_void_p),
                ("R", ct.c_void_p), ("logvol", ct.c_void_p), ("info", ct.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        _build.build()
    L = ct.CDLL(_build.LIB)
    vp, i32, i64, f64, sz = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_double, ct.c_size_t
    P, PP, PC = ct.POINTER(_Problem), ct.POINTER(_Params), ct.POINTER(_Cur)
    L.lra_precondition.argtypes = [ct.POINTER(vp), i32, i32, i64, i32, vp, vp]
    L.lra_precondition_fourier.argtypes = [ct.POINTER(vp), i64, i32, vp, vp]
    L.lra_multiplier_destroy.argtypes = [vp]
    L.lra_ca_workspace_size.argtypes = [P, PP, vp, ct.POINTER(sz)]
    L.lra_ca_run.argtypes = [P, PP, vp, vp, PC, vp, sz, vp]
    L.lra_ca_run_noalloc.argtypes = [P, PP, vp, vp, PC, vp]
    L.lra_ca_run_warm.argtypes = [P, PP, vp, vp, vp, PC, vp, sz, vp]
    L.lra_cur_apply.argtypes = [vp, vp, vp, i64, i64, i32, vp, i32, vp, i32, vp, sz, vp]
    L.lra_cur_apply_workspace_size.argtypes = [i64, i32, i32, ct.POINTER(sz)]
    L.lra_residual_sample.argtypes = [P, vp, vp, vp, i32, vp, i32, vp, i32, vp, vp, vp, sz, vp]
    L.lra_residual_sample_workspace_size.argtypes = [i32, i32, i32, ct.POINTER(sz)]
    PB, PCB = ct.POINTER(_Batch), ct.POINTER(_CurBatch)
    L.lra_ca_batched_workspace_size.argtypes = [P, PB, PP, ct.POINTER(sz)]
    L.lra_ca_run_batched.argtypes = [P, PB, PP, vp, PCB, vp, sz, vp]
    L.lra_residual_sample_batched.argtypes = [P, PB, i32, PCB, vp, i32, vp, i32, vp, vp]
    L.lra_ca_batched_tune.argtypes = [P, PB, PP, vp, PCB, vp, sz, vp, i32, ct.POINTER(i32), ct.POINTER(i32), vp]
    L.lra_ca_batched_tune_stages.argtypes = [P, P, PB, PP, vp, PCB, vp, sz, vp, i32, vp, i32, vp, f64, vp, i32, i32,
                                             vp, ct.POINTER(i32), vp, vp]
    L.lra_cynical_batched_workspace_size.argtypes = [P, PB, PP, i32, i32, ct.POINTER(sz)]
    L.lra_cynical_run_batched.argtypes = [P, PB, PP, i32, i32, vp, vp, vp, PCB, vp, sz, vp]
    L.lra_cynical_batched_tune.argtypes = [P, PB, PP, i32, i32, vp, vp, vp, PCB, vp, sz, vp, i32,
                                           ct.POINTER(i32), ct.POINTER(i32), vp]
    L.lra_oversample_batched_workspace_size.argtypes = [P, PB, PP, i32, ct.POINTER(sz)]
    L.lra_oversample_batched.argtypes = [P, PB, PP, i32, PCB, PCB, vp, sz, vp]
    L.lra_multiplier_apply.argtypes = [P, vp, vp, i64, vp]
    L.lra_rhtcur_workspace_size.argtypes = [P, PP, ct.POINTER(sz)]
    L.lra_ca_lev_batched_workspace_size.argtypes = [P, PB, i32, i32, i32, i32, ct.POINTER(sz)]
    PH = ct.POINTER(_HMatrix)
    L.lra_hmatvec_workspace_size.argtypes = [PH, ct.POINTER(sz)]
    L.lra_hmatvec.argtypes = [P, PH, vp, vp, vp, sz, vp]
    L.lra_ca_lev_batched.argtypes = [P, PB, i32, i32, i32, i32, f64, vp, vp, PCB, vp, sz, vp]
    L.lra_rhtcur_run.argtypes = [P, vp, PP, ct.POINTER(_Cur), vp, sz, vp]
    L.lra_gather_rows.argtypes = [P, vp, i32, vp, vp, vp]
    L.lra_oversample_cycle_batched_workspace_size.argtypes = [P, PB, PP, i32, i32, ct.POINTER(sz)]
    L.lra_oversample_cycle_batched.argtypes = [P, PB, PP, i32, i32, PCB, PCB, vp, sz, vp]
    L.lra_prjvol_batched_workspace_size.argtypes = [P, PB, PP, i32, ct.POINTER(sz)]
    L.lra_prjvol_batched.argtypes = [P, PB, PP, i32, PCB, PCB, vp, sz, vp]
    L.lra_residual_sample_batched_rect.argtypes = [P, PB, i32, i32, PCB, vp, i32, vp, i32, vp, vp]
    L.lra_ca_batched_shapes.argtypes = [vp, vp, i32]
    L.lra_ca_batched_shapes.restype = i32
    PG = ct.POINTER(_Gauss)
    L.lra_gauss_cur_forward.argtypes = [PG, vp, i32, vp, vp, vp]
    L.lra_gauss_cur_backward.argtypes = [PG, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]
    L.lra_version.restype = ct.c_char_p
    L.lra_launch_count.restype = ct.c_int64
    L.lra_profile_enable.argtypes = [i32]
    L.lra_profile_collect.argtypes = [i32, vp, vp, vp, ct.POINTER(i32)]
    for f in ("lra_precondition", "lra_precondition_fourier", "lra_multiplier_destroy", "lra_ca_workspace_size", "lra_ca_run", "lra_ca_run_warm",
              "lra_ca_run_noalloc",
              "lra_cur_apply", "lra_cur_apply_workspace_size", "lra_residual_sample",
              "lra_residual_sample_workspace_size", "lra_profile_enable", "lra_profile_collect",
              "lra_ca_batched_workspace_size", "lra_ca_run_batched", "lra_residual_sample_batched",
              "lra_ca_batched_tune", "lra_ca_batched_tune_stages", "lra_cynical_batched_workspace_size", "lra_cynical_run_batched",
              "lra_cynical_batched_tune", "lra_oversample_batched_workspace_size", "lra_oversample_batched",
              "lra_oversample_cycle_batched_workspace_size", "lra_oversample_cycle_batched", "lra_multiplier_apply",
              "lra_gather_rows", "lra_rhtcur_workspace_size", "lra_rhtcur_run", "lra_ca_lev_batched_workspace_size",
              "lra_ca_lev_batched", "lra_hmatvec_workspace_size", "lra_hmatvec",
              "lra_residual_sample_batched_rect", "lra_prjvol_batched_workspace_size", "lra_prjvol_batched",
              "lra_gauss_cur_forward", "lra_gauss_cur_backward"):
        getattr(L, f).restype = ct.c_int
    _lib = L
    return L


def _check(st: int, where: str):
    if st != LRA_OK:
        raise LraError(st, where)


def _dev(t: Optional[torch.Tensor], dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _workspace(nbytes: int, device) -> torch.Tensor:
    # 256-byte aligned: torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


@dataclass
class Problem:
    """An m x n input on the device: a dense row-major matrix or a kernel on
    two point sets (targets X: m x 3, sources Y: n x 3, FP64)."""

    src: int
    m: int
    n: int
    W: Optional[torch.Tensor] = None
    X: Optional[torch.Tensor] = None
    Y: Optional[torch.Tensor] = None
    length_scale: float = 1.0
    entries: str = "f64"

    @staticmethod
    def dense(W: torch.Tensor) -> "Problem":
        if W.dim() != 2 or W.dtype not in (torch.float64, torch.float32):
            raise TypeError("dense W must be a 2-D float64 or float32 CUDA tensor")
        _dev(W, name="W")
        return Problem(LRA_DENSE, W.shape[0], W.shape[1], W=W)

    @staticmethod
    def kernel(kind: str, X: torch.Tensor, Y: torch.Tensor, length_scale: float = 1.0,
               entries: str = "f64") -> "Problem":
        """Kernel entries w_ij = K(x_i, y_j) evaluated on demand; ``entries``
        'f32' evaluates the Laplace kernel in FP32 (correctly rounded ops)."""
        src = {"laplace": LRA_KERNEL_LAPLACE, "gaussian": LRA_KERNEL_GAUSSIAN}[kind]
        if entries not in ("f64", "f32", "bf16"):
            raise ValueError("entries must be 'f64', 'f32' or 'bf16'")
        _dev(X, torch.float64, "X"); _dev(Y, torch.float64, "Y")
        return Problem(src, X.shape[0], Y.shape[0], X=X, Y=Y, length_scale=length_scale, entries=entries)

    def _c(self) -> _Problem:
        p = _Problem()
        p.src, p.m, p.n = self.src, self.m, self.n
        if self.W is not None:
            p.dtype = LRA_F32 if self.W.dtype == torch.float32 else LRA_F64
            p.W, p.ldw = self.W.data_ptr(), self.W.stride(0)
        if self.X is not None:
            p.X, p.Y = self.X.data_ptr(), self.Y.data_ptr()
            p.dtype = {"f64": LRA_F64, "f32": LRA_F32, "bf16": LRA_BF16}[self.entries]
        p.length_scale = float(self.length_scale)
        return p


class Multiplier:
    """Owner of a library multiplier handle (lra_precondition)."""

    def __init__(self, handle: int, kind: int, n: int):
        self.handle, self.kind, self.n = handle, kind, n

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.lra_multiplier_destroy(self.handle)
        except Exception:
            pass
        self.handle = None


def lra_version() -> str:
    return _load().lra_version().decode()


def lra_precondition(kind: str, n: int, depth_or_nnz: int, perm_or_rows, signs, side: str = "right") -> Multiplier:
    """Multiplier M (n x n) of W' = W M (``side`` 'right') or W' = M^T W ('left',
    n = the problem's m): ``kind`` 'arht' (2^{-d/2} D H_{n,d} P), 'sparse'
    (+-1/sqrt(nnz) entries) or 'bidiag' (2^{-q/2} prod (I + D_i S) P_i, q =
    depth_or_nnz factors; perm_or_rows, signs q x n).  perm_or_rows / signs: host
    int32 / int8 arrays (numpy or CPU tensors) holding the random draws."""
    import numpy as np
    L = _load()
    k = {"arht": LRA_MULT_ARHT, "sparse": LRA_MULT_SPARSE_PM1, "bidiag": LRA_MULT_BIDIAG}[kind]
    sd = {"right": LRA_SIDE_RIGHT, "left": LRA_SIDE_LEFT}[side]
    idx = np.ascontiguousarray(np.asarray(perm_or_rows), dtype=np.int32).reshape(-1)
    sg = np.ascontiguousarray(np.asarray(signs), dtype=np.int8).reshape(-1)
    h = ct.c_void_p()
    _check(L.lra_precondition(ct.byref(h), k, sd, int(n), int(depth_or_nnz), idx.ctypes.data, sg.ctypes.data),
           "lra_precondition")
    return Multiplier(h.value, k, n)


def lra_precondition_fourier(n: int, depth: int, perm, diag) -> Multiplier:
    """Abridged randomized Fourier multiplier in real form, [Re M, Im M] (n x 2n)
    with M = 2^{-d/2} D Omega_{n,d} P: perm (n int32) and diag (n x 2 float64,
    the real and imaginary parts of D on the complex unit circle) are host
    arrays of the random draws.  The pre-processed W' has 2n columns."""
    import numpy as np
    L = _load()
    idx = np.ascontiguousarray(np.asarray(perm), dtype=np.int32).reshape(-1)
    dg = np.ascontiguousarray(np.asarray(diag), dtype=np.float64).reshape(-1)
    if dg.size != 2 * idx.size:
        raise ValueError("diag must hold n (real, imaginary) pairs")
    h = ct.c_void_p()
    _check(L.lra_precondition_fourier(ct.byref(h), int(n), int(depth), idx.ctypes.data, dg.ctypes.data),
           "lra_precondition_fourier")
    return Multiplier(h.value, LRA_MULT_ARFT, n)


def lra_multiplier_destroy(mult: Multiplier) -> None:
    if mult is not None and mult.handle:
        _check(_load().lra_multiplier_destroy(mult.handle), "lra_multiplier_destroy")
        mult.handle = None


def lra_multiplier_apply(problem: Problem, multiplier: Optional[Multiplier], out: Optional[torch.Tensor] = None,
                         stream=None) -> torch.Tensor:
    """W' = W M written out as a dense m x n FP64 tensor; every entry is the value
    the C-A gathers form on the fly, so a C-A run on Problem.dense(W') picks the
    pivots of a run on (W, M).  ``out`` (m x n float64, unit column stride) is
    written in place when given."""
    dev = (problem.W if problem.W is not None else problem.X).device
    ncols = 2 * problem.n if (multiplier is not None and multiplier.kind == LRA_MULT_ARFT) else problem.n
    if out is None:
        out = torch.empty(problem.m, ncols, dtype=torch.float64, device=dev)
    if out.dim() != 2 or tuple(out.shape) != (problem.m, ncols) or out.dtype != torch.float64 or \
            out.stride(1) != 1:
        raise ValueError("out must be an m x n' float64 tensor with unit column stride (n' = columns of W')")
    _dev(out, torch.float64, "out")
    pc = problem._c()
    _check(_load().lra_multiplier_apply(ct.byref(pc), multiplier.handle if multiplier is not None else None,
                                        out.data_ptr(), out.stride(0), _stream(stream)), "lra_multiplier_apply")
    return out


def lra_gather_rows(problem: Problem, I: torch.Tensor, out: Optional[torch.Tensor] = None,
                    status: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """R = W[I, :] (k x n FP64) from the original input: the row factor of the
    CUR of W when the generators came from a materialised W' = W M.  ``out``:
    k x n float64 (contiguous) or None; ``status``: a device int32 scalar that a
    row index outside [0, m) sets to LRA_ERR_INVALID_ARG."""
    _dev(I, torch.int32, "I")
    k = I.numel()
    if out is None:
        out = torch.empty(k, problem.n, dtype=torch.float64, device=I.device)
    if out.numel() != k * problem.n or out.dtype != torch.float64 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 tensor of k x n entries")
    pc = problem._c()
    _check(_load().lra_gather_rows(ct.byref(pc), I.data_ptr(), k, out.data_ptr(),
                                   status.data_ptr() if status is not None else None, _stream(stream)),
           "lra_gather_rows")
    return out


def _params(k, sweeps, h, rank_tol, max_swaps, mode, stages=None, rank_margin=0, ctas=0) -> _Params:
    p = _Params()
    p.k, p.sweeps, p.h, p.rank_tol, p.max_swaps, p.mode = int(k), int(sweeps), float(h), float(rank_tol), \
        int(max_swaps), int(mode)
    p.ctas = int(ctas)
    if stages is not None:
        stages = [int(x) for x in stages]
        if not 1 <= len(stages) <= LRA_MAX_STAGES:
            raise ValueError(f"1..{LRA_MAX_STAGES} stages")
        p.nstages, p.rank_margin = len(stages), int(rank_margin)
        for i, v in enumerate(stages):
            p.k_stages[i] = v
    return p


def _check_cur_out(out: dict, m: int, n: int, k: int, sweeps: int) -> None:
    """Raise unless every output tensor of a C-A run is a contiguous device
    tensor of the dtype and size the library writes (I, J: k int32; C: m k,
    U: k k, R: k n, logvol: 2 sweeps float64; info: LRA_INFO_LEN int32)."""
    want = dict(I=(torch.int32, k), J=(torch.int32, k), C=(torch.float64, m * k), U=(torch.float64, k * k),
                R=(torch.float64, k * n), logvol=(torch.float64, 2 * sweeps), info=(torch.int32, LRA_INFO_LEN))
    for f, (dt, numel) in want.items():
        if f not in out:
            raise ValueError(f"out is missing {f}")
        t = out[f]
        _dev(t, dt, f)
        if t.numel() < numel or not t.is_contiguous():
            raise ValueError(f"out[{f!r}] must be a contiguous {dt} tensor of at least {numel} elements")


def lra_ca_workspace_size(problem: Problem, k: int, sweeps: int = 3, h: float = 1.01, rank_tol: float = 1e-13,
                          max_swaps: int = 1000, mode: int = LRA_MODE_FP64,
                          multiplier: Optional[Multiplier] = None, ctas: int = 0) -> int:
    L = _load()
    out = ct.c_size_t()
    pc, pp = problem._c(), _params(k, sweeps, h, rank_tol, max_swaps, mode, ctas=ctas)
    _check(L.lra_ca_workspace_size(ct.byref(pc), ct.byref(pp), multiplier.handle if multiplier else None,
                                   ct.byref(out)), "lra_ca_workspace_size")
    return out.value


def lra_ca_run(problem: Problem, I0: torch.Tensor, k: int, sweeps: int = 3, h: float = 1.01,
               rank_tol: float = 1e-13, max_swaps: int = 1000, mode: int = LRA_MODE_FP64,
               multiplier: Optional[Multiplier] = None, out: Optional[dict] = None,
               workspace: Optional[torch.Tensor] = None, stream=None, J0: Optional[torch.Tensor] = None,
               ctas: int = 0) -> dict:
    """C-A CUR approximation W ~ C U R of W' = W M (see lra_ca_run in lra.h).

    I0: device int32 tensor of k distinct initial rows; J0 (optional): k columns
    warm-starting the first column step (lra_ca_run_warm: resume from a previous
    run's I, J); ctas: CTAs sharing the run (0: the library's choice;
    lra_ca_tune picks one by timing).  Returns a dict of
    device tensors I, J, C (m x k), U (k x k), R (k x n), logvol (2*sweeps),
    info (rank, swaps, loops, status); the call is asynchronous on ``stream``.
    Pass ``out`` (same dict layout) and ``workspace`` to reuse buffers."""
    L = _load()
    dev = (problem.W if problem.W is not None else problem.X).device
    _dev(I0, torch.int32, "I0")
    if J0 is not None:
        _dev(J0, torch.int32, "J0")
    pc, pp = problem._c(), _params(k, sweeps, h, rank_tol, max_swaps, mode, ctas=ctas)
    mh = multiplier.handle if multiplier else None
    if out is None:
        out = dict(I=torch.empty(k, dtype=torch.int32, device=dev), J=torch.empty(k, dtype=torch.int32, device=dev),
                   C=torch.empty(problem.m, k, dtype=torch.float64, device=dev),
                   U=torch.empty(k, k, dtype=torch.float64, device=dev),
                   R=torch.empty(k, problem.n, dtype=torch.float64, device=dev),
                   logvol=torch.empty(2 * sweeps, dtype=torch.float64, device=dev),
                   info=torch.empty(LRA_INFO_LEN, dtype=torch.int32, device=dev))
    _check_cur_out(out, problem.m, problem.n, k, sweeps)
    if workspace is None:
        nb = ct.c_size_t()
        _check(L.lra_ca_workspace_size(ct.byref(pc), ct.byref(pp), mh, ct.byref(nb)), "lra_ca_workspace_size")
        workspace = _workspace(nb.value, dev)
    cur = _Cur()
    for f in ("I", "J", "C", "U", "R", "logvol", "info"):
        setattr(cur, f, _dev(out[f], name=f).data_ptr())
    _check(L.lra_ca_run_warm(ct.byref(pc), ct.byref(pp), mh, I0.data_ptr(), None if J0 is None else J0.data_ptr(),
                             ct.byref(cur), workspace.data_ptr(), workspace.numel(), _stream(stream)), "lra_ca_run")
    out["_workspace"] = workspace
    return out


def lra_rhtcur_run(problem: Problem, Hbar: torch.Tensor, h: float = 1.01, rank_tol: float = 1e-13,
                   max_swaps: int = 1000, out: Optional[dict] = None, workspace: Optional[torch.Tensor] = None,
                   stream=None) -> dict:
    """CUR LRA with Gaussian sampling (Algorithm algrhtcur, lbar = l = k): rows
    from the sketch S = W Hbar (Hbar: n x k float64 CUDA tensor of Gaussian
    draws), columns from W[I, :].  Returns lra_ca_run's dict (logvol: 2 values)."""
    L = _load()
    dev = (problem.W if problem.W is not None else problem.X).device
    _dev(Hbar, torch.float64, "Hbar")
    if Hbar.dim() != 2 or Hbar.shape[0] != problem.n:
        raise ValueError("Hbar must be n x k")
    k = Hbar.shape[1]
    pc, pp = problem._c(), _params(k, 1, h, rank_tol, max_swaps, LRA_MODE_FP64)
    if out is None:
        out = dict(I=torch.empty(k, dtype=torch.int32, device=dev), J=torch.empty(k, dtype=torch.int32, device=dev),
                   C=torch.empty(problem.m, k, dtype=torch.float64, device=dev),
                   U=torch.empty(k, k, dtype=torch.float64, device=dev),
                   R=torch.empty(k, problem.n, dtype=torch.float64, device=dev),
                   logvol=torch.empty(2, dtype=torch.float64, device=dev),
                   info=torch.empty(LRA_INFO_LEN, dtype=torch.int32, device=dev))
    if workspace is None:
        nb = ct.c_size_t()
        _check(L.lra_rhtcur_workspace_size(ct.byref(pc), ct.byref(pp), ct.byref(nb)), "lra_rhtcur_workspace_size")
        workspace = _workspace(nb.value, dev)
    cur = _Cur()
    for f in ("I", "J", "C", "U", "R", "logvol", "info"):
        setattr(cur, f, _dev(out[f], name=f).data_ptr())
    _check(L.lra_rhtcur_run(ct.byref(pc), Hbar.data_ptr(), ct.byref(pp), ct.byref(cur), workspace.data_ptr(),
                            workspace.numel(), _stream(stream)), "lra_rhtcur_run")
    out["_workspace"] = workspace
    return out


def lra_ca_run_noalloc(problem: Problem, I0: torch.Tensor, out: dict, k: int, sweeps: int = 3, h: float = 1.01,
                       rank_tol: float = 1e-13, max_swaps: int = 1000, mode: int = LRA_MODE_FP64,
                       multiplier: Optional[Multiplier] = None, stream=None) -> dict:
    """lra_ca_run on the library's static device scratch (see lra_ca_run_noalloc
    in lra.h): nothing is allocated, so ``out`` must hold the output tensors
    (I, J, C, U, R, logvol, info as returned by lra_ca_run)."""
    L = _load()
    _dev(I0, torch.int32, "I0")
    _check_cur_out(out, problem.m, problem.n, k, sweeps)
    pc, pp = problem._c(), _params(k, sweeps, h, rank_tol, max_swaps, mode)
    cur = _Cur()
    for f in ("I", "J", "C", "U", "R", "logvol", "info"):
        setattr(cur, f, _dev(out[f], name=f).data_ptr())
    _check(L.lra_ca_run_noalloc(ct.byref(pc), ct.byref(pp), multiplier.handle if multiplier else None,
                                I0.data_ptr(), ct.byref(cur), _stream(stream)), "lra_ca_run_noalloc")
    return out


def lra_cur_apply(C: torch.Tensor, U: torch.Tensor, R: torch.Tensor, X: torch.Tensor,
                  Y: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
    """Y = C (U (R X)) on the device.  C and R are float64 (FP64 products) or
    both float32 / bfloat16 (stored factors, FP32 products with one refinement
    step, see lra_cur_apply in lra.h); U, X and Y are float64."""
    L = _load()
    dt = {torch.float64: LRA_F64, torch.float32: LRA_F32, torch.bfloat16: LRA_BF16}.get(C.dtype)
    if dt is None or R.dtype != C.dtype:
        raise TypeError("C and R must both be float64, float32 or bfloat16")
    _dev(C, C.dtype, "C"); _dev(R, C.dtype, "R")
    for t, nm in ((U, "U"), (X, "X")):
        _dev(t, torch.float64, nm)
    m, k = C.shape
    n = R.shape[1]
    X2 = X if X.dim() == 2 else X.view(-1, 1)
    nrhs = X2.shape[1]
    if Y is None:
        Y = torch.empty(m, nrhs, dtype=torch.float64, device=C.device)
    if workspace is None:
        nb = ct.c_size_t()
        _check(L.lra_cur_apply_workspace_size(n, k, nrhs, ct.byref(nb)), "lra_cur_apply_workspace_size")
        workspace = _workspace(nb.value, C.device)
    _check(L.lra_cur_apply(C.data_ptr(), U.data_ptr(), R.data_ptr(), m, n, k, X2.data_ptr(), nrhs, Y.data_ptr(),
                           dt, workspace.data_ptr(), workspace.numel(), _stream(stream)), "lra_cur_apply")
    return Y


def lra_cur_apply_workspace_size(n: int, k: int, nrhs: int) -> int:
    """Bytes of device workspace lra_cur_apply needs (any storage dtype)."""
    nb = ct.c_size_t()
    _check(_load().lra_cur_apply_workspace_size(int(n), int(k), int(nrhs), ct.byref(nb)),
           "lra_cur_apply_workspace_size")
    return max(int(nb.value), 256)


def lra_residual_sample(problem: Problem, C: torch.Tensor, U: torch.Tensor, R: torch.Tensor, Q: torch.Tensor,
                        S: torch.Tensor, E: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Statistics [mean, var, mean|e|, max|e|, fro ratio] (device FP64 tensor of
    5) of the sample E[Q,S] of W - C U R."""
    L = _load()
    k = C.shape[1]
    q, s = Q.numel(), S.numel()
    stats = torch.empty(5, dtype=torch.float64, device=C.device)
    nb = ct.c_size_t()
    _check(L.lra_residual_sample_workspace_size(k, q, s, ct.byref(nb)), "lra_residual_sample_workspace_size")
    ws = _workspace(nb.value, C.device)
    pc = problem._c()
    _check(L.lra_residual_sample(ct.byref(pc), C.data_ptr(), U.data_ptr(), R.data_ptr(), k,
                                 _dev(Q, torch.int32, "Q").data_ptr(), q, _dev(S, torch.int32, "S").data_ptr(), s,
                                 stats.data_ptr(), E.data_ptr() if E is not None else None, ws.data_ptr(),
                                 ws.numel(), _stream(stream)), "lra_residual_sample")
    return stats


def lra_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(_load().lra_launch_count())


def lra_profile_enable(on: bool = True) -> None:
    """Bracket every later kernel launch with CUDA events on its stream."""
    _check(_load().lra_profile_enable(1 if on else 0), "lra_profile_enable")


def lra_profile_collect(max_kernels: int = 32) -> dict:
    """{kernel name: (total ms, launches)} since the last collect (waits for the events)."""
    L = _load()
    NAME = 32
    names = ct.create_string_buffer(max_kernels * NAME)
    ms = (ct.c_double * max_kernels)()
    cnt = (ct.c_int64 * max_kernels)()
    n = ct.c_int32()
    _check(L.lra_profile_collect(max_kernels, names, ms, cnt, ct.byref(n)), "lra_profile_collect")
    out = {}
    for i in range(min(n.value, max_kernels)):
        nm = names.raw[i * NAME:(i + 1) * NAME].split(b"\0", 1)[0].decode()
        out[nm] = (ms[i], int(cnt[i]))
    return out


class Batch:
    """Device buffers of a batch of blocks W[r0:r0+nr, c0:c0+nc] of one input
    (the C ABI's lra_batch and lra_cur_batch).  Allocation and uploads happen
    here, once; lra_ca_run_batched / lra_residual_sample_batched then only
    launch kernels, so they can be captured in a CUDA graph."""

    def __init__(self, problem: Problem, blocks, k: int, sweeps: int, I0, h: float = 1.01, rank_tol: float = 1e-6,
                 max_swaps: int = 1000, order="lpt", device=None, mode: int = LRA_MODE_FP64, stages=None,
                 rank_margin: int = 2, store_factors: bool = True, pair_min_len: Optional[int] = None):
        """``stages``: ascending generator sizes ending at k (the size of each block is
        fitted to its nucleus rank: a larger stage runs while rank >= size - rank_margin);
        None runs every block at min(k, rows, cols).  ``store_factors`` False keeps
        only I, J, U (no C, R buffers: a matrix-free lra_hmatvec recomputes their
        entries).  ``pair_min_len``: blocks with more rows or columns than this run
        first, each on a pair of CTAs (lra_batch.pair_blocks; None: none do)."""
        import numpy as np
        blocks = np.ascontiguousarray(np.asarray(blocks, dtype=np.int64).reshape(-1, 4))
        nb = len(blocks)
        dev = device or (problem.W if problem.W is not None else problem.X).device
        kb = np.minimum(k, np.minimum(blocks[:, 1], blocks[:, 3]))
        csz, rsz = blocks[:, 1] * kb, kb * blocks[:, 3]
        offs = np.zeros((nb, 2), dtype=np.int64)
        offs[1:, 0] = np.cumsum(csz)[:-1]
        offs[1:, 1] = np.cumsum(rsz)[:-1]
        if isinstance(order, str) and order == "lpt":
            order = np.argsort(-(blocks[:, 1] * blocks[:, 3]), kind="stable").astype(np.int32)
        npairs = 0
        if pair_min_len is not None:
            if order is None:
                order = np.arange(nb, dtype=np.int32)
            order = np.asarray(order, dtype=np.int32)
            big = np.maximum(blocks[order, 1], blocks[order, 3]) > int(pair_min_len)
            order = np.concatenate([order[big], order[~big]]).astype(np.int32)
            npairs = int(big.sum())
        self.problem, self.k, self.sweeps, self.nb = problem, int(k), int(sweeps), nb
        self.blocks_np, self.offs_np, self.kb = blocks, offs, kb
        self.params = _params(k, sweeps, h, rank_tol, max_swaps, mode, stages, rank_margin)
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)
        self.blocks, self.offs = t(blocks, np.int64), t(offs, np.int64)
        self.order = None if order is None else t(order, np.int32)
        self.I0 = t(np.asarray(I0).reshape(nb, k), np.int32)
        self.store_factors = bool(store_factors)
        self.out = dict(I=torch.zeros(nb, k, dtype=torch.int32, device=dev),
                        J=torch.zeros(nb, k, dtype=torch.int32, device=dev),
                        U=torch.zeros(nb, k, k, dtype=torch.float64, device=dev),
                        logvol=torch.zeros(nb, 2 * sweeps, dtype=torch.float64, device=dev),
                        info=torch.zeros(nb, LRA_INFO_LEN, dtype=torch.int32, device=dev))
        if self.store_factors:
            self.out["C"] = torch.zeros(max(int(csz.sum()), 1), dtype=torch.float64, device=dev)
            self.out["R"] = torch.zeros(max(int(rsz.sum()), 1), dtype=torch.float64, device=dev)
        self.cb = _Batch()
        self.cb.blocks, self.cb.offsets = self.blocks.data_ptr(), self.offs.data_ptr()
        self.cb.order = self.order.data_ptr() if self.order is not None else None
        self.cb.nb, self.cb.max_len = nb, int(max(blocks[:, 1].max(), blocks[:, 3].max()))
        self.cb.pair_blocks = npairs
        self.work = torch.zeros(nb, dtype=torch.float64, device=dev)   # per-block algorithmic flops
        self.cur = _CurBatch()
        for f in ("I", "J", "C", "U", "R", "logvol", "info"):
            setattr(self.cur, f, self.out[f].data_ptr() if f in self.out else None)
        self.cur.work = self.work.data_ptr()
        self.pc = problem._c()
        L = _load()
        nbytes = ct.c_size_t()
        _check(L.lra_ca_batched_workspace_size(ct.byref(self.pc), ct.byref(self.cb), ct.byref(self.params),
                                               ct.byref(nbytes)), "lra_ca_batched_workspace_size")
        self.workspace = _workspace(nbytes.value, dev)

    def block(self, b: int, host: Optional[dict] = None) -> dict:
        """Host copies of block b's results (for checks).  ``host``: the batch's
        outputs already copied to the host ({name: numpy array}), to avoid one
        device read-back per block."""
        (r0, nr, c0, nc) = self.blocks_np[b]
        oc, orr = self.offs_np[b]
        o = host if host is not None else {key: v.cpu().numpy() for key, v in self.out.items()}
        info = o["info"][b]
        kb = int(info[6]) if info[6] > 0 else int(self.kb[b])
        return dict(I=o["I"][b, :kb], J=o["J"][b, :kb],
                    C=o["C"][oc:oc + nr * kb].reshape(nr, kb) if "C" in o else None,
                    U=o["U"][b].reshape(-1)[:kb * kb].reshape(kb, kb),
                    R=o["R"][orr:orr + kb * nc].reshape(kb, nc) if "R" in o else None, logvol=o["logvol"][b],
                    rank=int(info[0]), swaps=int(info[1]), loops=int(info[2]), status=int(info[3]),
                    fp32_steps=int(info[4]), fp64_steps=int(info[5]), k=kb)


def lra_ca_batched_shapes() -> list:
    """The (threads per CTA, CTAs per SM) shapes the batched kernel is built for."""
    L = _load()
    t = (ct.c_int32 * 16)(); c = (ct.c_int32 * 16)()
    n = L.lra_ca_batched_shapes(t, c, 16)
    return [(t[i], c[i]) for i in range(min(n, 16))]


def lra_ca_batched_tune(batch: Batch, reps: int = 2, stream=None) -> dict:
    """Autotuner: times the whole batch in every CTA shape, stores the fastest in
    ``batch`` (later lra_ca_run_batched calls use it) and returns
    {(threads, ctas): ms}.  Synchronises the stream."""
    L = _load()
    shapes = lra_ca_batched_shapes()
    ms = (ct.c_float * len(shapes))()
    th, cs = ct.c_int32(), ct.c_int32()
    _check(L.lra_ca_batched_tune(ct.byref(batch.pc), ct.byref(batch.cb), ct.byref(batch.params),
                                 batch.I0.data_ptr(), ct.byref(batch.cur), batch.workspace.data_ptr(),
                                 batch.workspace.numel(), _stream(stream), int(reps), ct.byref(th), ct.byref(cs), ms),
           "lra_ca_batched_tune")
    batch.cb.cta_threads, batch.cb.ctas_per_sm = th.value, cs.value
    return {shp: ms[i] for i, shp in enumerate(shapes) if ms[i] >= 0}


def lra_ca_batched_tune_stages(batch: Batch, schedules, Q: torch.Tensor, S: torch.Tensor,
                               exact: Optional[Problem] = None, tol: float = 1e-6, reps: int = 2,
                               stats: Optional[torch.Tensor] = None, stream=None) -> dict:
    """Autotuner of the staged generator sizes (see lra_ca_batched_tune_stages in
    lra.h): times the batch under every schedule, keeps the schedules under which
    every block's sampled error (rows Q, columns S: nb x q, nb x s device int32,
    against ``exact``'s entries) is <= tol, stores the fastest in ``batch`` (later
    lra_ca_run_batched calls use it; its results are left in batch.out) and
    returns {(sizes, margin): (ms, max error)}.  ``schedules``: ascending size
    tuples ending at batch.k, or (sizes, margin) pairs (default margin: the
    batch's).  Synchronises the stream."""
    import numpy as np
    rows = []
    for sc in schedules:
        if len(sc) == 2 and isinstance(sc[0], (tuple, list)):
            sizes, margin = tuple(int(x) for x in sc[0]), int(sc[1])
        else:
            sizes, margin = tuple(int(x) for x in sc), int(batch.params.rank_margin)
        if not 1 <= len(sizes) <= LRA_MAX_STAGES:
            raise ValueError(f"1..{LRA_MAX_STAGES} sizes per schedule")
        rows.append((sizes, margin))
    tab = np.zeros((len(rows), 2 + LRA_MAX_STAGES), dtype=np.int32)
    for i, (sizes, margin) in enumerate(rows):
        tab[i, 0], tab[i, 1] = len(sizes), margin
        tab[i, 2:2 + len(sizes)] = sizes
    if stats is None:
        stats = torch.empty(batch.nb, 5, dtype=torch.float64, device=batch.blocks.device)
    if exact is not None and (exact.m, exact.n) != (batch.problem.m, batch.problem.n):
        raise ValueError("exact must have the batch problem's shape")
    ms = (ct.c_float * len(rows))()
    err = (ct.c_double * len(rows))()
    best = ct.c_int32()
    pe = exact._c() if exact is not None else None
    _check(_load().lra_ca_batched_tune_stages(
        ct.byref(batch.pc), ct.byref(pe) if pe is not None else None, ct.byref(batch.cb), ct.byref(batch.params),
        batch.I0.data_ptr(), ct.byref(batch.cur), batch.workspace.data_ptr(), batch.workspace.numel(),
        _dev(Q, torch.int32, "Q").data_ptr(), Q.shape[1], _dev(S, torch.int32, "S").data_ptr(), S.shape[1],
        _dev(stats, torch.float64, "stats").data_ptr(), float(tol), tab.ctypes.data_as(ct.c_void_p), len(rows),
        int(reps), _stream(stream), ct.byref(best), ms, err), "lra_ca_batched_tune_stages")
    sizes, margin = rows[best.value]
    batch.params.nstages, batch.params.rank_margin = len(sizes), margin
    for i in range(LRA_MAX_STAGES):
        batch.params.k_stages[i] = sizes[i] if i < len(sizes) else 0
    batch.stages, batch.rank_margin = sizes, margin
    return {rows[i]: (ms[i], err[i]) for i in range(len(rows))}


def _cyn_workspace(batch: Batch, kind: int, q: int):
    key = (int(kind), int(q))
    if getattr(batch, "_cyn_key", None) != key:
        nbytes = ct.c_size_t()
        _check(_load().lra_cynical_batched_workspace_size(ct.byref(batch.pc), ct.byref(batch.cb),
                                                          ct.byref(batch.params), int(kind), int(q),
                                                          ct.byref(nbytes)), "lra_cynical_batched_workspace_size")
        batch._cyn_ws, batch._cyn_key = _workspace(nbytes.value, batch.blocks.device), key
    return batch._cyn_ws


def lra_cynical_batched_tune(batch: Batch, q: int, K: torch.Tensor, L: torch.Tensor, I0s: torch.Tensor,
                             reps: int = 2, stream=None) -> dict:
    """Autotuner of the cynical kernel (Tests 3 runs): times every CTA shape, stores
    the fastest in ``batch`` and returns {(threads, ctas): ms}.  Synchronises."""
    L_ = _load()
    ws = _cyn_workspace(batch, 0, q)
    shapes = lra_ca_batched_shapes()
    ms = (ct.c_float * len(shapes))()
    th, cs = ct.c_int32(), ct.c_int32()
    _check(L_.lra_cynical_batched_tune(ct.byref(batch.pc), ct.byref(batch.cb), ct.byref(batch.params), 0, int(q),
                                       K.data_ptr(), L.data_ptr(), I0s.data_ptr(), ct.byref(batch.cur),
                                       ws.data_ptr(), ws.numel(), _stream(stream), int(reps), ct.byref(th),
                                       ct.byref(cs), ms), "lra_cynical_batched_tune")
    batch.cb.cta_threads, batch.cb.ctas_per_sm = th.value, cs.value
    return {shp: ms[i] for i, shp in enumerate(shapes) if ms[i] >= 0}


def lra_cynical_run_batched(batch: Batch, kind: int, q: int, K: torch.Tensor, L: torch.Tensor, I0s: torch.Tensor,
                            stream=None) -> None:
    """Cynical CUR of every block (kind 0: Tests 3 with the sketch sets K, L;
    kind 1: Tests 4 from the column sets L, K receiving the computed rows and L
    the computed columns): an r x r generator (r = batch.k) inside a q x q sketch,
    from the sketch initial rows I0s (nb x r).  Results in batch.out."""
    L_ = _load()
    for t, nm, shp in ((K, "K", (batch.nb, q)), (L, "L", (batch.nb, q)), (I0s, "I0s", (batch.nb, batch.k))):
        _dev(t, torch.int32, nm)
        if tuple(t.shape) != shp or not t.is_contiguous():
            raise ValueError(f"{nm} must be a contiguous {shp} int32 tensor")
    _cyn_workspace(batch, kind, q)
    _check(L_.lra_cynical_run_batched(ct.byref(batch.pc), ct.byref(batch.cb), ct.byref(batch.params), int(kind),
                                      int(q), K.data_ptr(), L.data_ptr(), I0s.data_ptr(), ct.byref(batch.cur),
                                      batch._cyn_ws.data_ptr(), batch._cyn_ws.numel(), _stream(stream)),
           "lra_cynical_run_batched")


class Oversampled:
    """Device outputs of lra_oversample_batched (or, with pmax > 0,
    lra_oversample_cycle_batched; with prjvol, lra_prjvol_batched) for a
    processed Batch: rectangular k_b x l_b generators (l_b = min(k_b + pextra,
    ncols))."""

    def __init__(self, batch: Batch, pextra: int, pmax: int = 0, prjvol: bool = False):
        import numpy as np
        b, k, p = batch, batch.k, int(pextra)
        self.pmax = int(pmax)
        blocks = b.blocks_np
        lcap = np.minimum(k + p, blocks[:, 3])
        csz, rsz = blocks[:, 1] * lcap, np.minimum(k, np.minimum(blocks[:, 1], blocks[:, 3])) * blocks[:, 3]
        offs = np.zeros((b.nb, 2), dtype=np.int64)
        offs[1:, 0] = np.cumsum(csz)[:-1]
        offs[1:, 1] = np.cumsum(rsz)[:-1]
        dev = b.blocks.device
        self.batch, self.pextra, self.offs_np = b, p, offs
        self.offs = torch.from_numpy(offs).to(dev)
        self.out = dict(I=torch.zeros(b.nb, k, dtype=torch.int32, device=dev),
                        J=torch.zeros(b.nb, k + p, dtype=torch.int32, device=dev),
                        C=torch.zeros(max(int(csz.sum()), 1), dtype=torch.float64, device=dev),
                        U=torch.zeros(b.nb, k + p, k, dtype=torch.float64, device=dev),
                        R=torch.zeros(max(int(rsz.sum()), 1), dtype=torch.float64, device=dev),
                        logvol=torch.zeros(1, dtype=torch.float64, device=dev),
                        info=torch.zeros(b.nb, LRA_INFO_LEN, dtype=torch.int32, device=dev))
        self.cb = _Batch()
        self.cb.blocks, self.cb.offsets = b.blocks.data_ptr(), self.offs.data_ptr()
        self.cb.order = b.cb.order
        self.cb.nb, self.cb.max_len = b.nb, b.cb.max_len
        self.cur = _CurBatch()
        for f in ("I", "J", "C", "U", "R", "logvol", "info"):
            setattr(self.cur, f, self.out[f].data_ptr())
        nbytes = ct.c_size_t()
        self.prjvol = bool(prjvol)
        if self.prjvol:
            _check(_load().lra_prjvol_batched_workspace_size(ct.byref(b.pc), ct.byref(self.cb), ct.byref(b.params), p,
                                                             ct.byref(nbytes)), "lra_prjvol_batched_workspace_size")
        else:
            _check(_load().lra_oversample_cycle_batched_workspace_size(ct.byref(b.pc), ct.byref(self.cb),
                                                                       ct.byref(b.params), p, self.pmax,
                                                                       ct.byref(nbytes)),
                   "lra_oversample_cycle_batched_workspace_size")
        self.workspace = _workspace(nbytes.value, dev)

    def block(self, i: int) -> dict:
        (r0, nr, c0, nc) = self.batch.blocks_np[i]
        o = {key: v.cpu().numpy() for key, v in self.out.items()}
        info = o["info"][i]
        k, l = int(info[6]), int(info[7])
        oc, orr = self.offs_np[i]
        return dict(I=o["I"][i, :k], J=o["J"][i, :l], C=o["C"][oc:oc + nr * l].reshape(nr, l),
                    U=o["U"][i].reshape(-1)[:l * k].reshape(l, k), R=o["R"][orr:orr + k * nc].reshape(k, nc),
                    rank=int(info[0]), status=int(info[3]), k=k, l=l, cycles=int(info[1]), ptried=int(info[2]),
                    swaps=int(info[1]), srank=int(info[2]))


def lra_oversample_batched(batch: Batch, pextra: int, ov: Optional[Oversampled] = None, stream=None) -> Oversampled:
    """Rectangular generators grown from the batch's square ones (run lra_ca_run_batched first)."""
    ov = ov or Oversampled(batch, pextra)
    _check(_load().lra_oversample_batched(ct.byref(batch.pc), ct.byref(ov.cb), ct.byref(batch.params), ov.pextra,
                                          ct.byref(batch.cur), ct.byref(ov.cur), ov.workspace.data_ptr(),
                                          ov.workspace.numel(), _stream(stream)), "lra_oversample_batched")
    return ov


def lra_oversample_cycle_batched(batch: Batch, pextra: int, pmax: int, max_cycles: int,
                                 ov: Optional[Oversampled] = None, stream=None) -> Oversampled:
    """Rectangular generators grown greedily from the batch's square ones, then
    refined by expansion/contraction cycles (p = 1..pmax, at most max_cycles
    kept) until they pass the local h-maximality test at the batch's h."""
    ov = ov or Oversampled(batch, pextra, pmax)
    if ov.pmax < int(pmax):
        raise ValueError("the Oversampled workspace was sized for a smaller pmax")
    par = _Params()
    ct.memmove(ct.byref(par), ct.byref(batch.params), ct.sizeof(_Params))
    par.max_swaps = int(max_cycles)
    _check(_load().lra_oversample_cycle_batched(ct.byref(batch.pc), ct.byref(ov.cb), ct.byref(par), ov.pextra,
                                                int(pmax), ct.byref(batch.cur), ct.byref(ov.cur),
                                                ov.workspace.data_ptr(), ov.workspace.numel(), _stream(stream)),
           "lra_oversample_cycle_batched")
    return ov


def lra_prjvol_batched(batch: Batch, pextra: int, ov: Optional[Oversampled] = None, max_swaps: Optional[int] = None,
                       stream=None) -> Oversampled:
    """Generators of maximal r-projective volume in each block's row strip
    W'[I, :] (Algorithm algprjvlm: Algorithm alg1tor's pivoted QR at the batch's
    rank_tol, dominance swaps on R' at the batch's h, greedy expansion to
    l_b = min(k_b + pextra, ncols)); run lra_ca_run_batched first.  max_swaps
    defaults to the batch's.  block(i) gives srank (r_b) and swaps."""
    ov = ov or Oversampled(batch, pextra, prjvol=True)
    if not ov.prjvol:
        raise ValueError("the Oversampled buffers were sized for lra_oversample_batched")
    par = _Params()
    ct.memmove(ct.byref(par), ct.byref(batch.params), ct.sizeof(_Params))
    if max_swaps is not None:
        par.max_swaps = int(max_swaps)
    _check(_load().lra_prjvol_batched(ct.byref(batch.pc), ct.byref(ov.cb), ct.byref(par), ov.pextra,
                                      ct.byref(batch.cur), ct.byref(ov.cur), ov.workspace.data_ptr(),
                                      ov.workspace.numel(), _stream(stream)), "lra_prjvol_batched")
    return ov


class LevBatch:
    """Device buffers of a batch of blocks for lra_ca_lev_batched: C-A
    iterations with DMM08 Algorithm 1 on the sketches (kind 0 Exactly(k),
    1 Expected(k) with rank r SVD-based leverage scores; 2, 3 the same with
    uniform scores, no SVD stage), ``draws`` uniforms per step."""

    def __init__(self, problem: Problem, blocks, k: int, r: int, iters: int, kind: int, I0, draws,
                 rank_tol: float = 1e-6, order="lpt"):
        import numpy as np
        blocks = np.ascontiguousarray(np.asarray(blocks, dtype=np.int64).reshape(-1, 4))
        nb = len(blocks)
        dev = (problem.W if problem.W is not None else problem.X).device
        csz, rsz = blocks[:, 1] * k, k * blocks[:, 3]
        offs = np.zeros((nb, 2), dtype=np.int64)
        offs[1:, 0] = np.cumsum(csz)[:-1]
        offs[1:, 1] = np.cumsum(rsz)[:-1]
        if isinstance(order, str) and order == "lpt":
            order = np.argsort(-(blocks[:, 1] * blocks[:, 3]), kind="stable").astype(np.int32)
        self.problem, self.k, self.r, self.iters, self.kind, self.nb = problem, int(k), int(r), int(iters), \
            int(kind), nb
        self.rank_tol = float(rank_tol)
        self.blocks_np, self.offs_np = blocks, offs
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)
        self.blocks, self.offs = t(blocks, np.int64), t(offs, np.int64)
        self.order = None if order is None else t(order, np.int32)
        self.max_len = int(max(blocks[:, 1].max(), blocks[:, 3].max()))
        self.I0 = t(np.asarray(I0).reshape(nb, k), np.int32)
        draws = torch.as_tensor(draws, dtype=torch.float64).reshape(-1)
        if draws.numel() != nb * 2 * self.iters * self.max_len:
            raise ValueError("draws: nb x (2 iters) x max_len uniforms")
        self.draws = draws.to(dev).contiguous()
        self.out = dict(I=torch.zeros(nb, k, dtype=torch.int32, device=dev),
                        J=torch.zeros(nb, k, dtype=torch.int32, device=dev),
                        C=torch.zeros(max(int(csz.sum()), 1), dtype=torch.float64, device=dev),
                        U=torch.zeros(nb, k, k, dtype=torch.float64, device=dev),
                        R=torch.zeros(max(int(rsz.sum()), 1), dtype=torch.float64, device=dev),
                        logvol=torch.zeros(1, dtype=torch.float64, device=dev),
                        info=torch.zeros(nb, LRA_INFO_LEN, dtype=torch.int32, device=dev))
        self.cb = _Batch()
        self.cb.blocks, self.cb.offsets = self.blocks.data_ptr(), self.offs.data_ptr()
        self.cb.order = self.order.data_ptr() if self.order is not None else None
        self.cb.nb, self.cb.max_len = nb, self.max_len
        self.cur = _CurBatch()
        for f in ("I", "J", "C", "U", "R", "logvol", "info"):
            setattr(self.cur, f, self.out[f].data_ptr())
        self.pc = problem._c()
        nbytes = ct.c_size_t()
        _check(_load().lra_ca_lev_batched_workspace_size(ct.byref(self.pc), ct.byref(self.cb), self.k, self.r,
                                                         self.iters, self.kind, ct.byref(nbytes)),
               "lra_ca_lev_batched_workspace_size")
        self.workspace = _workspace(nbytes.value, dev)

    def block(self, b: int) -> dict:
        (r0, nr, c0, nc) = self.blocks_np[b]
        oc, orr = self.offs_np[b]
        o = {key: v.cpu().numpy() for key, v in self.out.items()}
        info = o["info"][b]
        kI, kJ = int(info[6]), int(info[7])
        return dict(I=o["I"][b, :kI], J=o["J"][b, :kJ], C=o["C"][oc:oc + nr * kJ].reshape(nr, kJ),
                    U=o["U"][b].reshape(-1)[:kJ * kI].reshape(kJ, kI), R=o["R"][orr:orr + kI * nc].reshape(kI, nc),
                    rank=int(info[0]), status=int(info[3]), kI=kI, kJ=kJ)


def lra_ca_lev_batched(lb: LevBatch, stream=None) -> None:
    """Run C-A with leverage-score sampling on every block of ``lb`` (asynchronous)."""
    _check(_load().lra_ca_lev_batched(ct.byref(lb.pc), ct.byref(lb.cb), lb.k, lb.r, lb.iters, lb.kind, lb.rank_tol,
                                      lb.I0.data_ptr(), lb.draws.data_ptr(), ct.byref(lb.cur),
                                      lb.workspace.data_ptr(), lb.workspace.numel(), _stream(stream)),
           "lra_ca_lev_batched")


def lra_residual_sample_oversampled(ov: Oversampled, Q: torch.Tensor, S: torch.Tensor,
                                    stats: Optional[torch.Tensor] = None, stream=None,
                                    problem: Optional[Problem] = None) -> torch.Tensor:
    """Per-block residual sample statistics (nb x 5) of rectangular generators."""
    b = ov.batch
    if stats is None:
        stats = torch.empty(b.nb, 5, dtype=torch.float64, device=b.blocks.device)
    pc = b.pc if problem is None else problem._c()
    _check(_load().lra_residual_sample_batched_rect(ct.byref(pc), ct.byref(ov.cb), b.k, b.k + ov.pextra,
                                                    ct.byref(ov.cur), _dev(Q, torch.int32, "Q").data_ptr(),
                                                    Q.shape[1], _dev(S, torch.int32, "S").data_ptr(), S.shape[1],
                                                    stats.data_ptr(), _stream(stream)),
           "lra_residual_sample_batched_rect")
    return stats


class HMatrix:
    """A kernel matrix K(P, P) (M_ii = 0) partitioned FMM-style: far blocks (the
    interaction-list pairs of every level, rows (nf, >= 6): row0, nrows, col0,
    ncols, level, target box) whose generators a batched C-A run computes, and
    near blocks (touching leaves, rows (nn, >= 5): row0, nrows, col0, ncols,
    target leaf) formed on the fly; y = M x by lra_hmatvec.  ``I0`` holds the
    C-A initial rows per far block (nf x k, block-local)."""

    def __init__(self, problem: Problem, far, near, levels: int, I0, k: int = 64, sweeps: int = 3, h: float = 1.05,
                 rank_tol: float = 1e-6, stages=(28, 40, 64), rank_margin: int = 2, matrix_free: bool = False):
        """``matrix_free``: keep only the generators' I, J and U (no C, R): each
        matvec re-evaluates their entries from the points, bit for bit as stored."""
        import numpy as np
        far = np.asarray(far, dtype=np.int64)
        near = np.asarray(near, dtype=np.int64)
        dev = problem.X.device
        self.problem, self.n, self.levels, self.matrix_free = problem, problem.m, int(levels), bool(matrix_free)
        self.batch = Batch(problem, far[:, :4], k, sweeps, I0, h=h, rank_tol=rank_tol, stages=stages,
                           rank_margin=rank_margin, store_factors=not matrix_free)
        # groups: runs of consecutive blocks with the same (level, target box) / target leaf
        fg = []
        for i in range(len(far)):
            if i == 0 or far[i, 4] != far[i - 1, 4] or far[i, 5] != far[i - 1, 5]:
                fg.append([far[i, 4], far[i, 0], far[i, 1], i, 0])
            fg[-1][4] += 1
        ng = []
        for i in range(len(near)):
            if i == 0 or near[i, 4] != near[i - 1, 4]:
                ng.append([near[i, 0], near[i, 1], i, 0])
            ng[-1][3] += 1
        t = lambda a, w: torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.int64).reshape(-1, w))).to(dev)
        self.far_groups, self.near = t(fg, 5), t(near[:, :4], 4)
        self.near_groups = t(ng, 4)
        H = _HMatrix()
        H.n, H.levels, H.kmax = self.n, self.levels, int(k)
        H.nfar, H.nfar_groups, H.nnear, H.nnear_groups = len(far), len(fg), len(near), len(ng)
        b = self.batch
        H.far, H.far_offsets = b.blocks.data_ptr(), b.offs.data_ptr()
        H.U, H.info = b.out["U"].data_ptr(), b.out["info"].data_ptr()
        if self.matrix_free:
            H.C = H.R = None
            H.I, H.J = b.out["I"].data_ptr(), b.out["J"].data_ptr()
        else:
            H.C, H.R = b.out["C"].data_ptr(), b.out["R"].data_ptr()
        H.far_groups, H.near, H.near_groups = (self.far_groups.data_ptr(), self.near.data_ptr(),
                                               self.near_groups.data_ptr())
        self.H = H
        nbytes = ct.c_size_t()
        _check(_load().lra_hmatvec_workspace_size(ct.byref(H), ct.byref(nbytes)), "lra_hmatvec_workspace_size")
        self.workspace = _workspace(nbytes.value, dev)

    def build(self, stream=None) -> None:
        """Compute every far block's generators (lra_ca_run_batched)."""
        lra_ca_run_batched(self.batch, stream)

    def matvec(self, x: torch.Tensor, y: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        _dev(x, torch.float64, "x")
        if y is None:
            y = torch.empty_like(x)
        pc = self.problem._c()
        _check(_load().lra_hmatvec(ct.byref(pc), ct.byref(self.H), x.data_ptr(), _dev(y, torch.float64, "y").data_ptr(),
                                   self.workspace.data_ptr(), self.workspace.numel(), _stream(stream)),
               "lra_hmatvec")
        return y


def lra_residual_sample_lev(lb: "LevBatch", Q: torch.Tensor, S: torch.Tensor, stats: Optional[torch.Tensor] = None,
                            stream=None) -> torch.Tensor:
    """Per-block residual sample statistics (nb x 5) of a LevBatch's k_I x k_J generators."""
    if stats is None:
        stats = torch.empty(lb.nb, 5, dtype=torch.float64, device=lb.blocks.device)
    _check(_load().lra_residual_sample_batched_rect(ct.byref(lb.pc), ct.byref(lb.cb), lb.k, lb.k, ct.byref(lb.cur),
                                                    _dev(Q, torch.int32, "Q").data_ptr(), Q.shape[1],
                                                    _dev(S, torch.int32, "S").data_ptr(), S.shape[1],
                                                    stats.data_ptr(), _stream(stream)),
           "lra_residual_sample_batched_rect")
    return stats


def lra_ca_run_batched(batch: Batch, stream=None) -> None:
    """C-A CUR of every block of `batch` in one persistent launch (results in batch.out)."""
    L = _load()
    _check(L.lra_ca_run_batched(ct.byref(batch.pc), ct.byref(batch.cb), ct.byref(batch.params),
                                batch.I0.data_ptr(), ct.byref(batch.cur), batch.workspace.data_ptr(),
                                batch.workspace.numel(), _stream(stream)), "lra_ca_run_batched")


def lra_residual_sample_batched(batch: Batch, Q: torch.Tensor, S: torch.Tensor, stats: Optional[torch.Tensor] = None,
                                stream=None, problem: Optional[Problem] = None) -> torch.Tensor:
    """Per-block residual sample statistics (nb x 5) of a batched run; Q (nb x q), S (nb x s) device int32.
    ``problem`` (default: the batch's) gives the entries the residual is measured against, e.g. the
    FP64 kernel for a run on FP32 entries."""
    L = _load()
    if stats is None:
        stats = torch.empty(batch.nb, 5, dtype=torch.float64, device=batch.blocks.device)
    pc = batch.pc if problem is None else problem._c()
    if problem is not None and (problem.m, problem.n) != (batch.problem.m, batch.problem.n):
        raise ValueError("residual problem must have the batch problem's shape")
    _check(L.lra_residual_sample_batched(ct.byref(pc), ct.byref(batch.cb), batch.k, ct.byref(batch.cur),
                                         _dev(Q, torch.int32, "Q").data_ptr(), Q.shape[1],
                                         _dev(S, torch.int32, "S").data_ptr(), S.shape[1], stats.data_ptr(),
                                         _stream(stream)), "lra_residual_sample_batched")
    return stats


def _gauss_struct(X, Y, I, J, ell):
    for t, nm, dt in ((X, "X", torch.float64), (Y, "Y", torch.float64), (I, "I", torch.int32), (J, "J", torch.int32)):
        _dev(t, dt, nm)
    g = _Gauss()
    g.X, g.Y, g.I, g.J = X.data_ptr(), Y.data_ptr(), I.data_ptr(), J.data_ptr()
    g.nb, g.m, g.n, g.k = X.shape[0], X.shape[1], Y.shape[1], I.shape[1]
    g.length_scale = float(ell)
    return g


def lra_gauss_cur_forward(X, Y, I, J, ell, x, stream=None):
    """y[b] = C U R x[b] on Gaussian blocks at fixed pivots.  X (nb, m, 3), Y (nb, n, 3)
    float64; I, J (nb, k) int32; x (nb, n, nrhs) float32.  Returns (y, ctx)."""
    L = _load()
    g = _gauss_struct(X, Y, I, J, ell)
    _dev(x, torch.float32, "x")
    nb, n, nrhs = x.shape
    y = torch.empty(nb, g.m, nrhs, dtype=torch.float32, device=x.device)
    ctx = torch.empty(nb, g.k * g.k + 2 * g.k * nrhs, dtype=torch.float64, device=x.device)
    _check(L.lra_gauss_cur_forward(ct.byref(g), x.data_ptr(), nrhs, y.data_ptr(), ctx.data_ptr(), _stream(stream)),
           "lra_gauss_cur_forward")
    return y, ctx


def lra_gauss_cur_backward(X, Y, I, J, ell, x, dy, ctx, entry_grads=False, stream=None):
    """Backward of lra_gauss_cur_forward: returns dict(dx, dell (nb,) float64[, dC, dR, dG])."""
    L = _load()
    g = _gauss_struct(X, Y, I, J, ell)
    _dev(x, torch.float32, "x"); _dev(dy, torch.float32, "dy"); _dev(ctx, torch.float64, "ctx")
    nb, n, nrhs = x.shape
    dx = torch.empty_like(x)
    dell = torch.empty(nb, dtype=torch.float64, device=x.device)
    out = dict(dx=dx, dell=dell)
    ptrs = [None, None, None]
    if entry_grads:
        out["dC"] = torch.empty(nb, g.m, g.k, dtype=torch.float32, device=x.device)
        out["dR"] = torch.empty(nb, g.k, g.n, dtype=torch.float32, device=x.device)
        out["dG"] = torch.empty(nb, g.k, g.k, dtype=torch.float32, device=x.device)
        ptrs = [out["dC"].data_ptr(), out["dR"].data_ptr(), out["dG"].data_ptr()]
    _check(L.lra_gauss_cur_backward(ct.byref(g), x.data_ptr(), dy.data_ptr(), nrhs, ctx.data_ptr(), dx.data_ptr(),
                                    dell.data_ptr(), ptrs[0], ptrs[1], ptrs[2], _stream(stream)),
           "lra_gauss_cur_backward")
    return out


class GaussCurApply(torch.autograd.Function):
    """y = C U R x on Gaussian-kernel blocks at fixed pivots, differentiable in x
    and in the length scale ell (a 0-dim tensor); the forward and the hand-written
    backward both run in the library's kernels."""

    @staticmethod
    def forward(ctx, x, ell, X, Y, I, J):
        e = float(ell)
        y, c = lra_gauss_cur_forward(X, Y, I, J, e, x.contiguous())
        ctx.save_for_backward(x, X, Y, I, J, c)
        ctx.ell = e
        ctx.ell_meta = (ell.dtype, ell.device) if torch.is_tensor(ell) else None
        return y

    @staticmethod
    def backward(ctx, dy):
        x, X, Y, I, J, c = ctx.saved_tensors
        g = lra_gauss_cur_backward(X, Y, I, J, ctx.ell, x, dy.contiguous().float(), c)
        dell = None
        if ctx.ell_meta is not None:
            dell = g["dell"].sum().to(ctx.ell_meta[0])
        return g["dx"], dell, None, None, None, None


def gauss_cur_apply(x, ell, X, Y, I, J):
    """Differentiable y = C U R x (see GaussCurApply)."""
    return GaussCurApply.apply(x, ell, X, Y, I, J)
