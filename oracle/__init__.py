"""FP64 CPU oracle for C-A CUR low-rank approximation (ctypes wrapper).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.
The CUDA library neither imports nor links it, and this package imports
nothing from the library: the two meet only through the seeded inputs of
``lra_inputs``.

Each function states the paper passage it follows (section, algorithm or
equation label of arXiv:1710.07946); the arithmetic lives in ``lra_oracle.c``.
"""
from __future__ import annotations

import ctypes as ct
import numpy as np

from . import build as _build

_lib = None


class _Problem(ct.Structure):
    _fields_ = [
        ("src", ct.c_int32), ("dtype", ct.c_int32), ("m", ct.c_int64), ("n", ct.c_int64),
        ("W", ct.c_void_p), ("ldw", ct.c_int64), ("X", ct.c_void_p), ("Y", ct.c_void_p),
        ("ell", ct.c_double), ("mkind", ct.c_int32), ("depth", ct.c_int32),
        ("perm", ct.c_void_p), ("dsign", ct.c_void_p), ("nnz", ct.c_int32),
        ("srow", ct.c_void_p), ("ssign", ct.c_void_p), ("brow", ct.c_void_p), ("bval", ct.c_void_p),
        ("mside", ct.c_int32), ("frow", ct.c_void_p), ("fwt", ct.c_void_p), ("dre", ct.c_void_p),
        ("dim", ct.c_void_p),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        P = ct.POINTER(_Problem)
        vp, i32, i64, f64 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_double
        L.orc_gather_rows.argtypes = [P, vp, i32, vp]
        L.orc_gather_cols_t.argtypes = [P, vp, i32, vp]
        L.orc_gather_rows_orig.argtypes = [P, vp, i32, vp]
        L.orc_maxvol.argtypes = [vp, i32, i64, vp, f64, i32, vp, vp, vp, vp]
        L.orc_maxvol.restype = ct.c_int
        L.orc_nucleus.argtypes = [vp, i32, f64, vp]
        L.orc_nucleus.restype = i32
        L.orc_ca_run.argtypes = [P, i32, i32, vp, f64, i32, f64, vp, vp, vp, vp, vp, vp, vp]
        L.orc_ca_run.restype = ct.c_int
        L.orc_ca_run_warm.argtypes = [P, i32, i32, vp, vp, f64, i32, f64, vp, vp, vp, vp, vp, vp, vp]
        L.orc_ca_run_warm.restype = ct.c_int
        L.orc_ca_run_adaptive.argtypes = [P, vp, i32, i32, i32, vp, f64, i32, f64, vp, vp, vp, vp, vp, vp, vp]
        L.orc_ca_run_adaptive.restype = ct.c_int
        L.orc_bidiag_columns.argtypes = [i64, i32, vp, vp, vp, vp]
        L.orc_fourier_columns.argtypes = [i64, i32, vp, vp, vp, vp, vp]
        L.orc_fourier_abridged.argtypes = [i64, i32, vp, vp]
        L.orc_nucleus_rect.argtypes = [vp, i32, i32, f64, vp]
        L.orc_residual_sample_rect.argtypes = [P, vp, vp, vp, i32, i32, vp, i32, vp, i32, vp, vp]
        L.orc_nucleus_rect.restype = i32
        L.orc_oversample.argtypes = [P, vp, vp, i32, i32, f64, f64, vp, vp, vp, vp, vp]
        L.orc_oversample.restype = ct.c_int
        L.orc_oversample_cycle.argtypes = [P, vp, vp, i32, i32, i32, i32, f64, f64, vp, vp, vp, vp, vp]
        L.orc_oversample_cycle.restype = ct.c_int
        L.orc_alg1tor.argtypes = [vp, i32, i64, f64, vp]
        L.orc_alg1tor.restype = i32
        L.orc_prjvol.argtypes = [P, vp, vp, i32, i32, f64, i32, f64, vp, vp, vp, vp, vp]
        L.orc_prjvol.restype = ct.c_int
        L.orc_rhtcur.argtypes = [P, vp, i32, f64, i32, f64, vp, vp, vp, vp, vp, vp, vp]
        L.orc_rhtcur.restype = ct.c_int
        L.orc_jacobi_eig.argtypes = [vp, vp, i32]
        L.orc_jacobi_eig.restype = None
        L.orc_lev_scores.argtypes = [vp, i32, i64, i32, vp]
        L.orc_lev_scores.restype = i32
        L.orc_lev_sample.argtypes = [vp, i64, i32, i32, vp, vp]
        L.orc_lev_sample.restype = i32
        L.orc_ca_lev.argtypes = [P, i32, i32, i32, i32, vp, vp, f64, vp, vp, vp, vp, vp, vp]
        L.orc_ca_lev.restype = ct.c_int
        L.orc_cynical.argtypes = [P, i32, i32, i32, vp, vp, vp, i32, f64, i32, f64, vp, vp, vp, vp, vp, vp]
        L.orc_cynical.restype = ct.c_int
        L.orc_cur_apply.argtypes = [vp, vp, vp, i64, i64, i32, vp, i32, vp]
        L.orc_residual_sample.argtypes = [P, vp, vp, vp, i32, vp, i32, vp, i32, vp, vp]
        L.orc_brute_maxvol.argtypes = [vp, i32, i32, vp]
        L.orc_brute_maxvol.restype = f64
        L.orc_hadamard_abridged.argtypes = [i64, i32, vp]
        L.orc_multiplier_dense.argtypes = [P, vp]
        L.orc_jacobi_svd.argtypes = [vp, i32, i32, vp, vp, vp]
        L.orc_gauss_cur_apply.argtypes = [vp, i64, vp, i64, vp, vp, i32, f64, vp, i32, vp, vp, vp, vp]
        L.orc_gauss_cur_backward.argtypes = [vp, i64, vp, i64, vp, vp, i32, f64, vp, vp, i32, vp, vp, vp, vp, vp]
        L.orc_jacobi_svd.restype = ct.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


class _Marshalled:
    """Keeps the numpy arrays referenced by a _Problem alive."""

    def __init__(self, p):
        self.keep = []
        s = _Problem()
        s.src, s.m, s.n = int(p.src), int(p.m), int(p.n)
        if p.W is not None:
            W = np.ascontiguousarray(p.W)
            if W.dtype not in (np.float64, np.float32):
                raise TypeError("dense input must be float64 or float32")
            self.keep.append(W)
            s.W, s.ldw = W.ctypes.data, W.shape[1]
            s.dtype = 1 if W.dtype == np.float32 else 0
        if p.W is None:
            s.dtype = {"f64": 0, "f32": 1, "bf16": 2}[getattr(p, "entries", "f64")]
        for name in ("X", "Y"):
            a = getattr(p, name)
            if a is not None:
                a = np.ascontiguousarray(a, dtype=np.float64)
                self.keep.append(a)
                setattr(s, name, a.ctypes.data)
        s.ell = float(p.ell)
        s.mkind = int(p.mkind)
        s.mside = int(getattr(p, "mside", 0))
        order = int(p.m) if s.mside else int(p.n)          # M is order x order
        if p.mkind == 1:
            perm = np.ascontiguousarray(p.perm, dtype=np.int32)
            ds = np.ascontiguousarray(p.dsign, dtype=np.int8)
            self.keep += [perm, ds]
            s.depth, s.perm, s.dsign = int(p.depth), perm.ctypes.data, ds.ctypes.data
        elif p.mkind == 2:
            sr = np.ascontiguousarray(p.srow, dtype=np.int32)
            ss = np.ascontiguousarray(p.ssign, dtype=np.int8)
            self.keep += [sr, ss]
            s.nnz, s.srow, s.ssign = int(p.nnz), sr.ctypes.data, ss.ctypes.data
        elif p.mkind == 3:
            perms = np.ascontiguousarray(p.perm, dtype=np.int32)
            sg = np.ascontiguousarray(p.dsign, dtype=np.int8)
            brow, bval = bidiag_columns(order, p.depth, perms, sg)
            self.keep += [perms, sg, brow, bval]
            s.depth, s.perm, s.dsign = int(p.depth), perms.ctypes.data, sg.ctypes.data
            s.brow, s.bval = brow.ctypes.data, bval.ctypes.data
        elif p.mkind == 4:
            if s.mside:
                raise ValueError("the abridged Fourier multiplier is a right multiplier")
            perm = np.ascontiguousarray(p.perm, dtype=np.int32)
            dre = np.ascontiguousarray(p.dcplx[:, 0], dtype=np.float64)
            dim = np.ascontiguousarray(p.dcplx[:, 1], dtype=np.float64)
            frow, fwt = fourier_columns(p.n, p.depth, perm, dre, dim)
            self.keep += [perm, dre, dim, frow, fwt]
            s.depth, s.perm = int(p.depth), perm.ctypes.data
            s.dre, s.dim, s.frow, s.fwt = dre.ctypes.data, dim.ctypes.data, frow.ctypes.data, fwt.ctypes.data
        self.s = s

    @property
    def ref(self):
        return ct.byref(self.s)


# ------------------------------------------------------------------ strips
def cols(p):
    """Columns of the pre-processed W': 2n for the real-form abridged Fourier
    multiplier, n otherwise."""
    return 2 * p.n if p.mkind == 4 else p.n


def gather_rows(p, I):
    """W'[I,:] with W' = W M (k x cols(p)); multiplier columns as in entry_wp()."""
    I = np.ascontiguousarray(I, dtype=np.int32)
    mp = _Marshalled(p)
    out = np.empty((len(I), cols(p)))
    lib().orc_gather_rows(mp.ref, _ptr(I), len(I), _ptr(out))
    return out


def gather_cols(p, J):
    """W'[:,J] (m x k)."""
    J = np.ascontiguousarray(J, dtype=np.int32)
    mp = _Marshalled(p)
    out = np.empty((len(J), p.m))
    lib().orc_gather_cols_t(mp.ref, _ptr(J), len(J), _ptr(out))
    return np.ascontiguousarray(out.T)


def gather_rows_orig(p, I):
    """W[I,:] without the multiplier (k x n)."""
    I = np.ascontiguousarray(I, dtype=np.int32)
    mp = _Marshalled(p)
    out = np.empty((len(I), p.n))
    lib().orc_gather_rows_orig(mp.ref, _ptr(I), len(I), _ptr(out))
    return out


# ------------------------------------------------------------------ maxvol
def maxvol(A, J_warm=None, h=1.01, max_swaps=1000):
    """Dominant k x k submatrix of the k x n matrix A (Algorithms algdomin and
    alggos).  Returns dict(J, C = B^{-1} A, logdet, nswaps, status)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    k, n = A.shape
    J = np.empty(k, dtype=np.int32)
    C = np.empty((k, n))
    ld = ct.c_double()
    ns = ct.c_int32()
    Jw = None if J_warm is None else np.ascontiguousarray(J_warm, dtype=np.int32)
    st = lib().orc_maxvol(_ptr(A), k, n, _ptr(Jw), h, max_swaps, _ptr(J), _ptr(C), ct.byref(ld), ct.byref(ns))
    return dict(J=J, C=C, logdet=ld.value, nswaps=ns.value, status=st)


def brute_maxvol(A):
    """Exhaustive maximal |det| over all k-subsets of columns (eqvol)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    k, n = A.shape
    J = np.empty(k, dtype=np.int32)
    v = lib().orc_brute_maxvol(_ptr(A), k, n, _ptr(J))
    return J, v


# ------------------------------------------------------------------ nucleus
def nucleus(G, tol=1e-13):
    """U = pinv of the rank-r QRP truncation of G (Algorithm algcnnncl with
    Remark reubsc).  Returns (U, r)."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    k = G.shape[0]
    assert G.shape == (k, k)
    U = np.empty((k, k))
    r = lib().orc_nucleus(_ptr(G), k, tol, _ptr(U))
    return U, r


def jacobi_svd(A):
    """One-sided Jacobi SVD (m >= n): returns (Uo, s, V)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    assert m >= n
    Uo = np.empty((m, n)); s = np.empty(n); V = np.empty((n, n))
    lib().orc_jacobi_svd(_ptr(A), m, n, _ptr(Uo), _ptr(s), _ptr(V))
    return Uo, s, V


# ------------------------------------------------------------------ C-A
def ca_run(p, k, sweeps, I0, h=1.01, max_swaps=1000, rank_tol=1e-13, J0=None):
    """alpha C-A loops then the canonical nucleus.  Returns dict with I, J,
    C (m x k) = W'[:,J], U (k x k), R (k x n) = W[I,:], logvol (2*sweeps),
    rank, swaps, loops, status.  J0: columns warm-starting the first column
    step (resume from a previous run's (I, J)), or None for the cold start."""
    mp = _Marshalled(p)
    I0 = np.ascontiguousarray(I0, dtype=np.int32)
    assert len(I0) == k
    J0 = None if J0 is None else np.ascontiguousarray(J0, dtype=np.int32)
    assert J0 is None or len(J0) == k
    I = np.empty(k, dtype=np.int32); J = np.empty(k, dtype=np.int32)
    C = np.empty((p.m, k)); U = np.empty((k, k)); R = np.empty((k, p.n))
    lv = np.empty(2 * sweeps); info = np.empty(4, dtype=np.int32)
    lib().orc_ca_run_warm(mp.ref, k, sweeps, _ptr(I0), _ptr(J0), h, max_swaps, rank_tol, _ptr(I), _ptr(J), _ptr(C),
                          _ptr(U), _ptr(R), _ptr(lv), _ptr(info))
    return dict(I=I, J=J, C=C, U=U, R=R, logvol=lv, rank=int(info[0]), swaps=int(info[1]),
                loops=int(info[2]), status=int(info[3]))


def rhtcur(p, Hbar, h=1.01, max_swaps=1000, rank_tol=1e-13):
    """CUR LRA with Gaussian sampling (Algorithm algrhtcur, lbar = l = k):
    rows I from the sketch S = W Hbar (Hbar n x k), then columns J from W[I, :]
    (orc_rhtcur).  Returns ca_run's dict (logvol of the second run)."""
    assert p.mkind == 0, "Algorithm algrhtcur samples W itself"
    mp = _Marshalled(p)
    Hbar = np.ascontiguousarray(Hbar, dtype=np.float64)
    assert Hbar.ndim == 2 and Hbar.shape[0] == p.n
    k = Hbar.shape[1]
    I = np.empty(k, dtype=np.int32); J = np.empty(k, dtype=np.int32)
    C = np.zeros((p.m, k)); U = np.zeros((k, k)); R = np.zeros((k, p.n))
    lv = np.empty(2); info = np.zeros(4, dtype=np.int32)
    lib().orc_rhtcur(mp.ref, _ptr(Hbar), k, h, max_swaps, rank_tol, _ptr(I), _ptr(J), _ptr(C), _ptr(U), _ptr(R),
                     _ptr(lv), _ptr(info))
    return dict(I=I, J=J, C=C, U=U, R=R, logvol=lv, rank=int(info[0]), swaps=int(info[1]), loops=int(info[2]),
                status=int(info[3]))


def jacobi_eig(G):
    """Round-robin Jacobi eigen-decomposition (orc_jacobi_eig): returns the
    rotated G (diagonal to rounding) and Q with G_in = Q G Q^T."""
    G = np.array(G, dtype=np.float64, order="C", copy=True)
    k = G.shape[0]
    Q = np.empty((k, k))
    lib().orc_jacobi_eig(_ptr(G), _ptr(Q), k)
    return G, Q


def lev_scores(A, r):
    """SVD-based leverage scores v_j = ||row j of V^(r)||^2 of the columns of a
    k x n sketch (orc_lev_scores); returns (v, eigenpairs used)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    k, n = A.shape
    v = np.empty(n)
    re = lib().orc_lev_scores(_ptr(A), k, n, int(r), _ptr(v))
    return v, int(re)


def lev_sample(v, l, kind, u):
    """Exactly(l) (kind 0) / Expected(l) (kind 1) sampling by the scores v
    (orc_lev_sample); u: the uniform draws.  Returns the picked indices."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(max(int(l), 1), dtype=np.int32)
    cnt = lib().orc_lev_sample(_ptr(v), len(v), int(l), int(kind), _ptr(u), _ptr(out))
    return out[:cnt].copy()


def ca_lev(p, k, r, iters, kind, draws, I0, rank_tol=1e-6):
    """C-A iterations with DMM08 Algorithm 1 on the sketches (orc_ca_lev):
    kind 0 Exactly(k), 1 Expected(k) with SVD-based scores; 2, 3 the same with
    uniform scores; draws (2 iters x max(m, n) uniforms).  Returns I (kI),
    J (kJ), C (m x kJ), U (kJ x kI), R (kI x n), rank, kI, kJ, status."""
    mp = _Marshalled(p)
    L = max(p.m, p.n)
    draws = np.ascontiguousarray(draws, dtype=np.float64).reshape(-1)
    assert draws.size >= 2 * iters * L
    I0 = np.ascontiguousarray(I0, dtype=np.int32)
    assert len(I0) == k
    I = np.zeros(k, dtype=np.int32); J = np.zeros(k, dtype=np.int32)
    C = np.zeros(p.m * k); U = np.zeros(k * k); R = np.zeros(k * p.n)
    info = np.zeros(4, dtype=np.int32)
    lib().orc_ca_lev(mp.ref, int(k), int(r), int(iters), int(kind), _ptr(draws), _ptr(I0), rank_tol, _ptr(I),
                     _ptr(J), _ptr(C), _ptr(U), _ptr(R), _ptr(info))
    kI, kJ = int(info[1]), int(info[2])
    return dict(I=I[:kI].copy(), J=J[:kJ].copy(), C=C[:p.m * kJ].reshape(p.m, kJ).copy(),
                U=U[:kJ * kI].reshape(kJ, kI).copy(), R=R[:kI * p.n].reshape(kI, p.n).copy(), rank=int(info[0]),
                kI=kI, kJ=kJ, status=int(info[3]))


def hmatvec(p, far, near, gens, x):
    """y = M x for M = K(P, P) (M_ii = 0) partitioned into far blocks with
    generators gens[b] = (C, U, R) (far order) and near blocks taken densely
    (the FMM's stage (iii)): plain numpy FP64 products, block by block."""
    P = np.asarray(p.X, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros(p.m)
    for b, (r0, nr, c0, nc) in enumerate(np.asarray(far)[:, :4]):
        C, U, R = gens[b]
        y[r0:r0 + nr] += C @ (U @ (R @ x[c0:c0 + nc]))
    for (r0, nr, c0, nc) in np.asarray(near)[:, :4]:
        d = np.sqrt(((P[r0:r0 + nr, None, :] - P[None, c0:c0 + nc, :]) ** 2).sum(axis=2))
        with np.errstate(divide="ignore"):
            K = np.where(d > 0.0, 1.0 / d, 0.0)
        y[r0:r0 + nr] += K @ x[c0:c0 + nc]
    return y


def ca_run_adaptive(p, stages, margin, sweeps, I0, h=1.01, max_swaps=1000, rank_tol=1e-6):
    """C-A with staged generator sizes (orc_ca_run_adaptive): a run at each size
    k_s of ``stages`` (clipped to min(m, n)) until the nucleus rank r_s < k_s -
    margin or the last size.  I0 holds min(stages[-1], m, n) distinct rows.
    Returns ca_run's dict at the final size plus k (final size) and stages (run)."""
    mp = _Marshalled(p)
    st = np.ascontiguousarray(stages, dtype=np.int32)
    assert len(st) >= 1 and np.all(np.diff(st) > 0) and st[0] >= 1
    kmax = int(min(st[-1], p.m, p.n))
    I0 = np.ascontiguousarray(I0, dtype=np.int32)[:kmax]
    assert len(I0) == kmax
    I = np.empty(kmax, dtype=np.int32); J = np.empty(kmax, dtype=np.int32)
    C = np.empty(p.m * kmax); U = np.empty(kmax * kmax); R = np.empty(kmax * p.n)
    lv = np.empty(2 * sweeps); info = np.empty(6, dtype=np.int32)
    lib().orc_ca_run_adaptive(mp.ref, _ptr(st), len(st), int(margin), sweeps, _ptr(I0), h, max_swaps, rank_tol,
                              _ptr(I), _ptr(J), _ptr(C), _ptr(U), _ptr(R), _ptr(lv), _ptr(info))
    k = int(info[4])
    return dict(I=I[:k].copy(), J=J[:k].copy(), C=C[:p.m * k].reshape(p.m, k), U=U[:k * k].reshape(k, k),
                R=R[:k * p.n].reshape(k, p.n), logvol=lv, rank=int(info[0]), swaps=int(info[1]),
                loops=int(info[2]), status=int(info[3]), k=k, stages=int(info[5]))


def cynical(p, kind, r, q, K, L, I0s, sweeps=3, h=1.01, max_swaps=1000, rank_tol=1e-13):
    """Cynical CUR (orc_cynical): kind 0 = Tests 3 (sketch W'[K, L] from the
    caller's K, L), kind 1 = Tests 4 (one C-A loop with q x q generators from the
    caller's L makes the sketch); then an r x r C-A generator inside the sketch
    from its initial rows I0s (r indices in [0, q)).  Returns ca_run's keys
    (without logvol) plus K, L (the sketch sets used)."""
    mp = _Marshalled(p)
    K = np.ascontiguousarray(np.zeros(q) if K is None else K, dtype=np.int32).copy()
    L = np.ascontiguousarray(L, dtype=np.int32).copy()
    I0s = np.ascontiguousarray(I0s, dtype=np.int32)
    assert len(K) == q and len(L) == q and len(I0s) == r
    I = np.zeros(r, dtype=np.int32); J = np.zeros(r, dtype=np.int32)
    C = np.zeros((p.m, r)); U = np.zeros((r, r)); R = np.zeros((r, p.n))
    info = np.zeros(4, dtype=np.int32)
    lib().orc_cynical(mp.ref, int(kind), int(r), int(q), _ptr(K), _ptr(L), _ptr(I0s), int(sweeps), h, max_swaps,
                      rank_tol, _ptr(I), _ptr(J), _ptr(C), _ptr(U), _ptr(R), _ptr(info))
    return dict(I=I, J=J, C=C, U=U, R=R, K=K, L=L, rank=int(info[0]), swaps=int(info[1]), loops=int(info[2]),
                status=int(info[3]))


def fourier_columns(n, d, perm, dre, dim):
    """Columns of the real form [Re M, Im M] of M = D Omega_{n,d} P before the
    scale 2^(-d/2): (2n, 2^d) rows (ascending) and real weights."""
    w = 1 << int(d)
    rows = np.zeros((2 * n, w), dtype=np.int32)
    wts = np.zeros((2 * n, w), dtype=np.float64)
    lib().orc_fourier_columns(int(n), int(d), _ptr(np.ascontiguousarray(perm, dtype=np.int32)),
                              _ptr(np.ascontiguousarray(dre, dtype=np.float64)),
                              _ptr(np.ascontiguousarray(dim, dtype=np.float64)), _ptr(rows), _ptr(wts))
    return rows, wts


def fourier_abridged(n, d):
    """Dense complex Omega_{n,d} from the decimation-in-frequency recursion eqfd
    with Omega_s = I_s (n = 2^d s)."""
    re = np.empty((n, n))
    im = np.empty((n, n))
    lib().orc_fourier_abridged(int(n), int(d), _ptr(re), _ptr(im))
    return re + 1j * im


def bidiag_columns(n, q, perms, signs):
    """Columns of the product of q quasi-Gaussian factors (I + D_i S) P_i:
    (n, min(2^q, n)) rows and integer values (0 = unused slot), ascending rows."""
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    signs = np.ascontiguousarray(signs, dtype=np.int8)
    w = min(1 << int(q), int(n))
    rows = np.zeros((n, w), dtype=np.int32)
    vals = np.zeros((n, w), dtype=np.int32)
    lib().orc_bidiag_columns(int(n), int(q), _ptr(perms), _ptr(signs), _ptr(rows), _ptr(vals))
    return rows, vals


def nucleus_rect(G, tol):
    """U (l x k) = pinv of the rank-r QRP truncation of the k x l generator G (k <= l); returns (U, r)."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    k, l = G.shape
    assert k <= l
    U = np.empty((l, k))
    r = lib().orc_nucleus_rect(_ptr(G), k, l, tol, _ptr(U))
    return U, int(r)


def oversample(p, I, J, pextra, h=1.01, rank_tol=1e-13, pmax=0, max_cycles=0):
    """Rectangular k x (k + pextra) generator grown from the square one (I, J) by
    greedy volume expansions, then (pmax > 0) expansion/contraction cycles
    until the generator passes the local h-maximality test of Corollary colclmx
    (orc_oversample_cycle).  Returns J (l), C (m x l), U (l x k), R (k x n),
    rank, l, status, cycles (kept), ptried (largest p tried)."""
    mp = _Marshalled(p)
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    k, L = len(I), len(I) + int(pextra)
    Jo = np.zeros(L + max(int(pmax), 0), dtype=np.int32)
    C = np.zeros((p.m, L)); U = np.zeros((L, k)); R = np.zeros((k, p.n))
    info = np.zeros(5, dtype=np.int32)
    lib().orc_oversample_cycle(mp.ref, _ptr(I), _ptr(J), k, int(pextra), int(pmax), int(max_cycles), h, rank_tol,
                               _ptr(Jo), _ptr(C), _ptr(U), _ptr(R), _ptr(info))
    l = int(info[1])
    return dict(J=Jo[:l].copy(), C=np.ascontiguousarray(C.reshape(-1)[:p.m * l].reshape(p.m, l)),
                U=np.ascontiguousarray(U.reshape(-1)[:l * k].reshape(l, k)), R=R, rank=int(info[0]), l=l,
                status=int(info[2]), cycles=int(info[3]), ptried=int(info[4]))


def alg1tor(A, tol=1e-13):
    """Algorithm alg1tor on the k x n matrix A (Householder QR with column
    pivoting, stopped at the numerical rank r at tol; orc_alg1tor).  Returns
    r, the pivots J0 (r), and the reduced matrix (k x n) whose first r rows are
    R' of Algorithm algprjvlm's factorisation A = Q R P, columns in their
    original order."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    k, n = A.shape
    J0 = np.zeros(max(min(k, n), 1), dtype=np.int32)
    r = int(lib().orc_alg1tor(_ptr(A), k, n, float(tol), _ptr(J0)))
    return r, J0[:r].copy(), A


def prjvol(p, I, J, pextra, h=1.01, max_swaps=1000, rank_tol=1e-13):
    """k x l generator (l = min(k + pextra, n)) of maximal r-projective volume in
    the row strip W'[I, :] (Algorithm algprjvlm with Algorithm alg1tor for the
    rank-revealing stage, Algorithm algdomin's swaps on R' and Algorithm algrup
    up to l columns; orc_prjvol).  Returns J (l), C (m x l), U (l x k), R (k x n),
    rank (nucleus), l, status, swaps, srank (the strip's numerical rank r)."""
    mp = _Marshalled(p)
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    k, L = len(I), len(I) + int(pextra)
    Jo = np.zeros(L, dtype=np.int32)
    C = np.zeros((p.m, L)); U = np.zeros((L, k)); R = np.zeros((k, p.n))
    info = np.zeros(5, dtype=np.int32)
    lib().orc_prjvol(mp.ref, _ptr(I), _ptr(J), k, int(pextra), h, int(max_swaps), rank_tol, _ptr(Jo), _ptr(C),
                     _ptr(U), _ptr(R), _ptr(info))
    l = int(info[1])
    return dict(J=Jo[:l].copy(), C=np.ascontiguousarray(C.reshape(-1)[:p.m * l].reshape(p.m, l)),
                U=np.ascontiguousarray(U.reshape(-1)[:l * k].reshape(l, k)), R=R, rank=int(info[0]), l=l,
                status=int(info[2]), swaps=int(info[3]), srank=int(info[4]))


def cur_apply(C, U, R, X):
    """Y = C (U (R X)) in FP64 (FMM stage iii product with the generators)."""
    C = np.ascontiguousarray(C, dtype=np.float64); U = np.ascontiguousarray(U, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64); X = np.ascontiguousarray(X, dtype=np.float64)
    m, k = C.shape
    n = R.shape[1]
    if X.ndim == 1:
        X = X[:, None]
    Y = np.empty((m, X.shape[1]))
    lib().orc_cur_apply(_ptr(C), _ptr(U), _ptr(R), m, n, k, _ptr(X), X.shape[1], _ptr(Y))
    return Y


def residual_sample(p, C, U, R, Q, S, return_E=False):
    """Statistics of the q x s sample E[Q,S] of E = W - C U R (a-posteriori
    estimation from a random submatrix): [mean, var, mean|e|, max|e|, fro ratio].
    C m x l, U l x k, R k x n (l = k for square generators)."""
    mp = _Marshalled(p)
    C = np.ascontiguousarray(C, dtype=np.float64); U = np.ascontiguousarray(U, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.int32); S = np.ascontiguousarray(S, dtype=np.int32)
    l, k = C.shape[1], R.shape[0]
    assert U.shape == (l, k)
    stats = np.empty(5)
    E = np.empty((len(Q), len(S))) if return_E else None
    lib().orc_residual_sample_rect(mp.ref, _ptr(C), _ptr(U), _ptr(R), k, l, _ptr(Q), len(Q), _ptr(S), len(S),
                                   _ptr(stats), _ptr(E))
    return (stats, E) if return_E else stats


# ------------------------------------------------------------------ multipliers
def hadamard_abridged(n, d):
    """Dense H_{n,d} from the recursion eqrfd with H_s = I_s."""
    H = np.empty((n, n))
    lib().orc_hadamard_abridged(n, d, _ptr(H))
    return H


def multiplier_dense(p):
    """Dense multiplier M of the problem (n x n for a right multiplier, m x m for
    a left one), assembled from its definition."""
    mp = _Marshalled(p)
    N = p.m if getattr(p, "mside", 0) else p.n
    M = np.empty((N, cols(p) if p.mkind == 4 else N))
    lib().orc_multiplier_dense(mp.ref, _ptr(M))
    return M


def gauss_cur_apply(X, Y, I, J, ell, x):
    """y = C U R x with C = K(X, Y_J), R = K(X_I, Y), U = K(X_I, Y_J)^{-1},
    K(x, y) = exp(-|x - y|^2 / (2 ell^2)) (FMM stage (iii) product on a
    Gaussian block with fixed pivots).  Returns (y, U, t1 = R x, t2 = U t1)."""
    X = np.ascontiguousarray(X, dtype=np.float64); Y = np.ascontiguousarray(Y, dtype=np.float64)
    I = np.ascontiguousarray(I, dtype=np.int32); J = np.ascontiguousarray(J, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    m, n, k, nrhs = len(X), len(Y), len(I), x.shape[1]
    y = np.empty((m, nrhs)); U = np.empty((k, k)); t1 = np.empty((k, nrhs)); t2 = np.empty((k, nrhs))
    lib().orc_gauss_cur_apply(_ptr(X), m, _ptr(Y), n, _ptr(I), _ptr(J), k, float(ell), _ptr(x), nrhs, _ptr(y),
                              _ptr(U), _ptr(t1), _ptr(t2))
    return y, U, t1, t2


def gauss_cur_backward(X, Y, I, J, ell, x, dy):
    """Backward of gauss_cur_apply at fixed pivots: returns dict(dx, dC, dR, dG, dell)."""
    X = np.ascontiguousarray(X, dtype=np.float64); Y = np.ascontiguousarray(Y, dtype=np.float64)
    I = np.ascontiguousarray(I, dtype=np.int32); J = np.ascontiguousarray(J, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64); dy = np.ascontiguousarray(dy, dtype=np.float64)
    if x.ndim == 1:
        x, dy = x[:, None], dy[:, None]
    m, n, k, nrhs = len(X), len(Y), len(I), x.shape[1]
    dx = np.empty((n, nrhs)); dC = np.empty((m, k)); dR = np.empty((k, n)); dG = np.empty((k, k))
    dl = ct.c_double()
    lib().orc_gauss_cur_backward(_ptr(X), m, _ptr(Y), n, _ptr(I), _ptr(J), k, float(ell), _ptr(x), _ptr(dy), nrhs,
                                 _ptr(dx), _ptr(dC), _ptr(dR), _ptr(dG), ct.byref(dl))
    return dict(dx=dx, dC=dC, dR=dR, dG=dG, dell=dl.value)
