"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's arithmetic: each compares with an
independent route (exhaustive search, a LAPACK routine through numpy, a dense
matrix built by a different recursion, a closed form or a printed table).
"""
import itertools
import math
import os

import numpy as np
import pytest

import lra_inputs as li
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ maxvol
@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("k,n", [(1, 7), (2, 8), (3, 9), (3, 10)])
def test_maxvol_dominant_and_near_global(seed, k, n):
    """Algorithm algdomin output: B = A[:,J] is dominant (Lemma lelcliden:
    max |B^{-1} A| <= h), and by Theorem thlclglb its volume is within
    h^k k^{k/2} of the global maximum found by exhaustive search."""
    g = np.random.default_rng(seed)
    A = g.standard_normal((k, n))
    h = 1.01
    r = oracle.maxvol(A, h=h)
    J = r["J"]
    assert len(set(J.tolist())) == k
    C_ref = np.linalg.solve(A[:, J], A)
    assert np.abs(C_ref).max() <= h * (1 + 1e-12)
    np.testing.assert_allclose(r["C"], C_ref, rtol=0, atol=1e-12 * max(1.0, np.abs(C_ref).max()))
    vol = abs(np.linalg.det(A[:, J]))
    assert math.isclose(r["logdet"], math.log(vol), rel_tol=1e-12, abs_tol=1e-12)
    _, best = oracle.brute_maxvol(A)
    assert best >= vol * (1 - 1e-12)
    assert vol >= best / (h ** k * k ** (k / 2)) * (1 - 1e-12)


def test_maxvol_brute_force_agrees_when_h_is_one():
    """With h = 1 a dominant submatrix is locally maximal; on small random
    inputs the greedy-initialised search reaches the exhaustive optimum in
    the large majority of cases (a weaker sub-check of the same theorem)."""
    hits = 0
    for seed in range(40):
        A = np.random.default_rng(100 + seed).standard_normal((3, 8))
        r = oracle.maxvol(A, h=1.0)
        Jb, best = oracle.brute_maxvol(A)
        vol = abs(np.linalg.det(A[:, r["J"]]))
        hits += vol >= best * (1 - 1e-12)
    assert hits >= 30


def test_maxvol_brute_force_square_identity():
    """k = n: the only choice is all columns, no swap."""
    A = np.random.default_rng(3).standard_normal((4, 4))
    r = oracle.maxvol(A)
    assert sorted(r["J"].tolist()) == [0, 1, 2, 3]
    assert r["nswaps"] == 0


def test_maxvol_warm_start_never_decreases_volume():
    """Each swap strictly increases |det| (Algorithm algdomin, stage 2)."""
    g = np.random.default_rng(7)
    A = g.standard_normal((5, 60))
    J0 = np.arange(5, dtype=np.int32)
    v0 = abs(np.linalg.det(A[:, J0]))
    r = oracle.maxvol(A, J_warm=J0)
    v1 = abs(np.linalg.det(A[:, r["J"]]))
    assert v1 >= v0 * (1 - 1e-12)
    if r["nswaps"]:
        assert v1 > v0
    assert np.abs(np.linalg.solve(A[:, r["J"]], A)).max() <= 1.01 * (1 + 1e-12)


def test_maxvol_rank_deficient_strip_flags():
    """An exactly singular strip (a zero row) meets a zero pivot."""
    g = np.random.default_rng(1)
    A = g.standard_normal((3, 12))
    A[1] = 0.0
    r = oracle.maxvol(A)
    assert r["status"] == 16 and r["nswaps"] == 0


def test_maxvol_lowest_index_tie_break():
    """Equal magnitudes: the lowest column index wins (the paper is silent;
    the tie rule is part of the specification of the pivots)."""
    A = np.array([[1.0, -1.0, 1.0, 0.5], [0.0, 1.0, 1.0, 1.0]])
    r = oracle.maxvol(A, h=10.0)
    assert r["J"][0] == 0


# ------------------------------------------------------------------ nucleus
@pytest.mark.parametrize("k", [1, 2, 5, 16, 48])
def test_nucleus_full_rank_is_inverse(k):
    """r = k: the canonical nucleus is G^{-1} (Remark reklr_kl, eq. eqnucinv)."""
    G = np.random.default_rng(k).standard_normal((k, k))
    U, r = oracle.nucleus(G)
    assert r == k
    np.testing.assert_allclose(U @ G, np.eye(k), atol=1e-10 * np.linalg.cond(G))


@pytest.mark.parametrize("k,r", [(6, 1), (7, 3), (16, 9), (33, 20)])
def test_nucleus_exact_low_rank_equals_library_pinv(k, r):
    """An exactly rank-r generator: its truncation is itself, so the nucleus
    must equal the Moore-Penrose inverse (eq. eqnuc+svd) computed by LAPACK's SVD."""
    g = np.random.default_rng(10 * k + r)
    G = g.standard_normal((k, r)) @ g.standard_normal((r, k))
    U, rr = oracle.nucleus(G, tol=1e-9)
    assert rr == r
    P = np.linalg.pinv(G, rcond=1e-9)
    np.testing.assert_allclose(U, P, atol=1e-9 * np.abs(P).max())


def test_nucleus_penrose_conditions_on_truncation():
    """Numerically rank-deficient G (singular values 1..1e-12): the nucleus is
    a Moore-Penrose inverse of a rank-r approximation G_r with ||G - G_r|| of the
    order of the dropped singular values."""
    g = np.random.default_rng(5)
    Uo, _ = np.linalg.qr(g.standard_normal((12, 12)))
    Vo, _ = np.linalg.qr(g.standard_normal((12, 12)))
    s = np.array([1, .5, .2, .1, 1e-2, 1e-3, 1e-8, 1e-9, 1e-10, 1e-11, 1e-12, 1e-12])
    G = (Uo * s) @ Vo.T
    U, r = oracle.nucleus(G, tol=1e-6)
    assert r == 6
    Gr = np.linalg.pinv(U, rcond=1e-12)             # pinv(pinv(G_r)) = G_r
    assert np.linalg.matrix_rank(U, tol=1e-6 * np.abs(U).max()) == 6
    assert np.linalg.norm(G - Gr, 2) < 1e-6
    np.testing.assert_allclose(U @ Gr @ U, U, atol=1e-8 * np.abs(U).max())
    np.testing.assert_allclose(Gr @ U @ Gr, Gr, atol=1e-12)


def test_jacobi_svd_matches_lapack():
    A = np.random.default_rng(2).standard_normal((9, 6))
    Uo, s, V = oracle.jacobi_svd(A)
    np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-13)
    np.testing.assert_allclose((Uo * s) @ V.T, A, atol=1e-13)


def test_nucleus_agrees_with_jacobi_svd_truncation_when_gap_is_large():
    """Remark reubsc: the QRP truncation and the SVD truncation give about the
    same nucleus when sigma_r >> sigma_{r+1}."""
    g = np.random.default_rng(11)
    Uo, _ = np.linalg.qr(g.standard_normal((10, 10)))
    Vo, _ = np.linalg.qr(g.standard_normal((10, 10)))
    s = np.array([3, 2, 1, .5, .3, 1e-11, 1e-12, 1e-12, 1e-13, 1e-14])
    G = (Uo * s) @ Vo.T
    U, r = oracle.nucleus(G, tol=1e-8)
    Ju, js, Jv = oracle.jacobi_svd(G)
    P = (Jv[:, :r] / js[:r]) @ Ju[:, :r].T
    np.testing.assert_allclose(U, P, atol=1e-8 * np.abs(P).max())


# ------------------------------------------------------------------ C-A / CUR
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("mult", ["none", "arht", "sparse", "bidiag"])
def test_exact_recovery_rank_r(seed, mult):
    """Theorem thdcmp: for rank-r W with a nonsingular r x r generator,
    W = C W_{I,J}^{-1} R exactly; with a multiplier M the back-transformed CUR
    (W M)[:,J] ((W M)[I,J])^+ W[I,:] is still exact (Algorithm alglratpsvd1 stage 4)."""
    p = li.dense_lowrank(128, 128, r=6, noise=0.0, seed=seed)
    if mult == "arht":
        li.with_arht(p, 2, seed + 50)
    elif mult == "sparse":
        li.with_sparse(p, 4, seed + 50)
    elif mult == "bidiag":
        li.with_bidiag(p, 3, seed + 50)
    I0 = li.initial_rows(128, 6, seed + 99)
    o = oracle.ca_run(p, 6, 3, I0)
    W = p.W
    err = np.linalg.norm(W - o["C"] @ o["U"] @ o["R"]) / np.linalg.norm(W)
    assert err < 1e-11, err
    assert o["rank"] == 6
    # the outputs are the submatrices they claim to be
    M = oracle.multiplier_dense(p) if mult != "none" else np.eye(128)
    WM = W @ M
    np.testing.assert_allclose(o["C"], WM[:, o["J"]], atol=1e-14)
    np.testing.assert_array_equal(o["R"], W[o["I"], :])


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("mult", ["arht", "sparse", "bidiag"])
def test_exact_recovery_rank_r_left_multiplier(seed, mult):
    """Remark re2orddmn (m > n: pre-multiply): with W' = M^T W the CUR of W from
    the generator (I, J) of W' is W[:, J] pinv(W'[I, J]) W'[I, :] (the
    right-multiplier back-transform applied to W^T), exact for rank-r W with a
    nonsingular core; C and R are the submatrices they claim to be, with M built
    densely from its definition."""
    p = li.dense_lowrank(160, 96, r=5, noise=0.0, seed=seed)
    if mult == "arht":
        li.with_arht(p, 3, seed + 60, side="left")
    elif mult == "sparse":
        li.with_sparse(p, 4, seed + 60, side="left")
    else:
        li.with_bidiag(p, 3, seed + 60, side="left")
    o = oracle.ca_run(p, 5, 3, li.initial_rows(160, 5, seed + 7))
    W = p.W
    err = np.linalg.norm(W - o["C"] @ o["U"] @ o["R"]) / np.linalg.norm(W)
    assert err < 1e-11, err
    assert o["rank"] == 5
    M = oracle.multiplier_dense(p)
    assert M.shape == (160, 160)
    MtW = M.T @ W
    np.testing.assert_array_equal(o["C"], W[:, o["J"]])
    np.testing.assert_allclose(o["R"], MtW[o["I"], :], atol=1e-14)
    # the nucleus is the (pseudo-)inverse of the pre-processed core
    np.testing.assert_allclose(o["U"] @ MtW[np.ix_(o["I"], o["J"])], np.eye(5), atol=1e-9)


@pytest.mark.parametrize("mult", ["arht2", "sparse", "bidiag3"])
def test_left_multiplier_gathers_equal_dense_product(mult):
    """With a left multiplier the gathers are rows / columns of M^T W, M m x m
    assembled from its definition (the transpose of the right-side case)."""
    g = np.random.default_rng(14)
    W = g.standard_normal((48, 20))
    p = li.Problem(li.SRC_DENSE, 48, 20, W=W)
    if mult.startswith("arht"):
        li.with_arht(p, int(mult[-1]), 9, side="left")
    elif mult.startswith("bidiag"):
        li.with_bidiag(p, int(mult[-1]), 9, side="left")
    else:
        li.with_sparse(p, 4, 9, side="left")
    MtW = oracle.multiplier_dense(p).T @ W
    I = np.array([3, 0, 47, 17], dtype=np.int32)
    J = np.array([19, 5, 6, 0], dtype=np.int32)
    np.testing.assert_allclose(oracle.gather_rows(p, I), MtW[I], atol=1e-14)
    np.testing.assert_allclose(oracle.gather_cols(p, J), MtW[:, J], atol=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_volume_non_decreasing_across_steps(seed):
    """C-A steps warm-started from the current sets never decrease the volume
    of the generator (the C-A volume argument; each swap of Algorithm algdomin
    increases |det|)."""
    p = li.factor_gaussian(200, 10, 1e-3, seed)
    o = oracle.ca_run(p, 10, 4, li.initial_rows(200, 10, seed))
    lv = o["logvol"][~np.isnan(o["logvol"])]
    assert np.all(np.diff(lv) >= -1e-10 * np.abs(lv[:-1]))
    # final logvol is log|det W[I,J]| computed independently
    assert math.isclose(lv[-1], math.log(abs(np.linalg.det(p.W[np.ix_(o["I"], o["J"])]))), rel_tol=1e-10)


def test_chebyshev_error_bound_theorem_th12():
    """Theorem th12 with k = l = r: ||W - CUR||_C <= h (r+1) sigma_{r+1}(W),
    h = (max volume over all r x r submatrices) / (volume of the generator),
    both measured by exhaustive search on a tiny matrix."""
    for seed in range(6):
        g = np.random.default_rng(seed)
        W = g.standard_normal((7, 2)) @ g.standard_normal((2, 7)) + 1e-3 * g.standard_normal((7, 7))
        p = li.Problem(li.SRC_DENSE, 7, 7, W=W)
        o = oracle.ca_run(p, 2, 3, li.initial_rows(7, 2, seed))
        best = max(abs(np.linalg.det(W[np.ix_(I, J)]))
                   for I in itertools.combinations(range(7), 2) for J in itertools.combinations(range(7), 2))
        h = best / abs(np.linalg.det(W[np.ix_(o["I"], o["J"])]))
        sig = np.linalg.svd(W, compute_uv=False)
        E = W - o["C"] @ o["U"] @ o["R"]
        assert np.abs(E).max() <= h * 3 * sig[2] * (1 + 1e-9)


def test_tests2_error_band_from_paper_table():
    """Table tb_ranrc (Tests 2, n = 256): our C-A with dominance swaps must do
    at least as well on average as the paper's reported mean error."""
    table = {}
    with open(os.path.join(GOLDEN, "tests2_error_table.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, r, mean, std = line.split()
                table[(int(n), int(r))] = float(mean)
    for (n, r), paper_mean in table.items():
        errs = []
        for seed in range(8):
            p = li.factor_gaussian(n, r, 1e-10, seed)
            o = oracle.ca_run(p, r, 5, li.initial_rows(n, r, 1000 + seed))
            E = p.W - o["C"] @ o["U"] @ o["R"]
            errs.append(np.linalg.norm(E, 2) / np.linalg.norm(p.W, 2))
        assert np.mean(errs) <= paper_mean
        # and not below the noise floor 1e-10 ||G3|| / ||W||
        assert np.min(errs) > 1e-13


def test_early_stop_when_no_swap():
    p = li.dense_lowrank(64, 64, r=4, noise=0.0, seed=3)
    o = oracle.ca_run(p, 4, 6, li.initial_rows(64, 4, 1))
    assert o["loops"] < 6


# ------------------------------------------------------------------ multipliers
def _read_blocks():
    out, cur = {}, None
    with open(os.path.join(GOLDEN, "abridged_hadamard_blocks.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("d="):
                cur = int(line[2:]); out[cur] = []
            else:
                out[cur].append([int(v) for v in line.split()])
    return {d: np.array(v) for d, v in out.items()}


@pytest.mark.parametrize("s", [1, 3, 8])
def test_abridged_hadamard_matches_printed_blocks(s):
    """H_{n,1} and H_{n,2} printed in equation eqbschf."""
    for d, B in _read_blocks().items():
        H = oracle.hadamard_abridged(s * (1 << d), d)
        np.testing.assert_array_equal(H, np.kron(B, np.eye(s)))


@pytest.mark.parametrize("n,d", [(16, 1), (24, 2), (64, 3)])
def test_arht_orthogonal_and_sparse(n, d):
    """D H_{n,d} P scaled by 2^{-d/2} is orthogonal and has 2^d nonzeros per
    row and column (appendix on abridged multipliers)."""
    p = li.Problem(li.SRC_DENSE, 4, n, W=np.zeros((4, n)))
    li.with_arht(p, d, 5)
    M = oracle.multiplier_dense(p)
    np.testing.assert_allclose(M @ M.T, np.eye(n), atol=1e-15)
    assert np.all((M != 0).sum(0) == 2 ** d) and np.all((M != 0).sum(1) == 2 ** d)


@pytest.mark.parametrize("mult", ["arht1", "arht2", "arht3", "sparse", "bidiag1", "bidiag3", "bidiag5"])
def test_multiplier_gathers_equal_dense_product(mult):
    """The strip gathers (closed-form column combinations) equal rows / columns
    of W M with M assembled densely from its recursive definition."""
    g = np.random.default_rng(4)
    W = g.standard_normal((40, 48))
    p = li.Problem(li.SRC_DENSE, 40, 48, W=W)
    if mult.startswith("arht"):
        li.with_arht(p, int(mult[-1]), 8)
    elif mult.startswith("bidiag"):
        li.with_bidiag(p, int(mult[-1]), 8)
    else:
        li.with_sparse(p, 4, 8)
    WM = W @ oracle.multiplier_dense(p)
    I = np.array([3, 0, 39, 17], dtype=np.int32)
    J = np.array([47, 5, 6, 0, 22], dtype=np.int32)
    np.testing.assert_allclose(oracle.gather_rows(p, I), WM[I], atol=1e-14)
    np.testing.assert_allclose(oracle.gather_cols(p, J), WM[:, J], atol=1e-14)
    np.testing.assert_array_equal(oracle.gather_rows_orig(p, I), W[I])


def test_bf16_laplace_entries_are_the_rounded_fp32_entries():
    """BF16 entries: the FP32 entry rounded to bfloat16 to nearest, ties to even,
    equal to PyTorch's float32 -> bfloat16 conversion on a million entries (with
    ties among them), within 2^-8 of the FP32 entry."""
    torch = pytest.importorskip("torch")
    p = li.laplace_clusters(1000, 1000, seed=8)
    I = np.arange(1000, dtype=np.int32)
    f32 = oracle.gather_rows(li.Problem(li.SRC_LAPLACE, 1000, 1000, X=p.X, Y=p.Y, entries="f32"), I)
    b16 = oracle.gather_rows(li.Problem(li.SRC_LAPLACE, 1000, 1000, X=p.X, Y=p.Y, entries="bf16"), I)
    ref = torch.from_numpy(f32.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(b16, ref)
    bits = f32.astype(np.float32).view(np.uint32)
    assert ((bits & 0xFFFF) == 0x8000).sum() > 0           # ties were exercised
    assert np.all(np.abs(b16 / f32 - 1) <= 2.0 ** -8)


# ------------------------------------------------------------------ abridged Fourier (ARFT)
@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_fourier_recursion_at_full_depth_is_the_dft(k):
    """Equation eqfd run to the bottom (d = k, Omega_1 = 1) gives the DFT matrix of
    equation eqdft, (w_n^{ij}) with w_n = exp(2 pi sqrt(-1) / n): this fixes the
    reading of the odd/even permutation and of Dhat_q = diag(w_{2q}^j), j < q."""
    n = 1 << k
    i = np.arange(n)
    F = np.exp(2j * np.pi * np.outer(i, i) / n)
    np.testing.assert_allclose(oracle.fourier_abridged(n, k), F, atol=1e-13)


@pytest.mark.parametrize("s", [1, 3, 8])
def test_fourier_abridged_depth_one_closed_form(s):
    """Omega_{2s,1} from Omega_s = I_s: row 2j holds 1 at columns j and j + s, row
    2j + 1 holds w_{2s}^j and -w_{2s}^j there."""
    n = 2 * s
    W = np.zeros((n, n), dtype=complex)
    for j in range(s):
        w = np.exp(2j * np.pi * j / n)
        W[2 * j, j] = W[2 * j, j + s] = 1.0
        W[2 * j + 1, j], W[2 * j + 1, j + s] = w, -w
    np.testing.assert_allclose(oracle.fourier_abridged(n, 1), W, atol=1e-15)


@pytest.mark.parametrize("n,d", [(24, 2), (40, 3), (64, 4), (96, 1)])
def test_fourier_abridged_unitary_up_to_scale_and_sparse(n, d):
    """Omega_{n,d} is unitary up to scaling (Omega^H Omega = 2^d I) with 2^d
    nonzeros, all of modulus 1, in every row and column."""
    F = oracle.fourier_abridged(n, d)
    np.testing.assert_allclose(F.conj().T @ F, (1 << d) * np.eye(n), atol=1e-12)
    nz = np.abs(F) > 1e-12
    assert np.all(nz.sum(0) == 1 << d) and np.all(nz.sum(1) == 1 << d)
    np.testing.assert_allclose(np.abs(F[nz]), 1.0, atol=1e-14)


@pytest.mark.parametrize("n,d", [(48, 1), (48, 2), (64, 3)])
def test_arft_real_form_gathers_equal_dense_product(n, d):
    """The real form [Re M, Im M] of M = 2^{-d/2} D Omega_{n,d} P has orthonormal
    rows, and the strip gathers (column lists with 2^d real weights) equal rows and
    columns of W [Re M, Im M] with the multiplier built densely by the recursion."""
    g = np.random.default_rng(21)
    W = g.standard_normal((30, n))
    p = li.Problem(li.SRC_DENSE, 30, n, W=W)
    li.with_arft(p, d, 3)
    Mr = oracle.multiplier_dense(p)
    assert Mr.shape == (n, 2 * n)
    np.testing.assert_allclose(Mr @ Mr.T, np.eye(n), atol=1e-14)
    # the complex M itself: D Omega P scaled, from numpy on the dense recursion
    D = p.dcplx[:, 0] + 1j * p.dcplx[:, 1]
    M = (D[:, None] * oracle.fourier_abridged(n, d)[:, p.perm]) * 2.0 ** (-d / 2)
    np.testing.assert_allclose(Mr, np.hstack([M.real, M.imag]), atol=1e-15)
    WM = W @ Mr
    I = np.array([3, 0, 29, 17], dtype=np.int32)
    J = np.array([2 * n - 1, 5, n, 0, n - 1], dtype=np.int32)
    np.testing.assert_allclose(oracle.gather_rows(p, I), WM[I], atol=1e-13)
    np.testing.assert_allclose(oracle.gather_cols(p, J), WM[:, J], atol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_exact_recovery_rank_r_arft(seed):
    """Algorithm alglratpsvd1 with the real-form ARFT as the n x 2n multiplier H
    (orthonormal rows): W = (W H)[:, J] ((W H)[I, J])^+ W[I, :] for rank-r W."""
    p = li.dense_lowrank(96, 64, r=6, noise=0.0, seed=seed)
    li.with_arft(p, 2, seed + 40)
    o = oracle.ca_run(p, 6, 3, li.initial_rows(96, 6, seed + 3))
    W = p.W
    assert np.all(o["J"] < 128) and o["rank"] == 6
    err = np.linalg.norm(W - o["C"] @ o["U"] @ o["R"]) / np.linalg.norm(W)
    assert err < 1e-11, err
    WM = W @ oracle.multiplier_dense(p)
    np.testing.assert_allclose(o["C"], WM[:, o["J"]], atol=1e-13)
    np.testing.assert_array_equal(o["R"], W[o["I"], :])


def test_sparse_multiplier_structure():
    p = li.Problem(li.SRC_DENSE, 4, 50, W=np.zeros((4, 50)))
    li.with_sparse(p, 4, 2)
    M = oracle.multiplier_dense(p)
    assert np.all((M != 0).sum(0) == 4)
    np.testing.assert_allclose(np.linalg.norm(M, axis=0), 1.0, rtol=1e-15)


def test_bidiag_single_factor_closed_form():
    """q = 1: M = 2^{-1/2} (I + D S) P of eq. def11, built entry by entry with numpy
    (column a: 1 at row b = perm[a], the sign of row b+1 at row (b+1) mod n)."""
    n = 37
    p = li.Problem(li.SRC_DENSE, 3, n, W=np.zeros((3, n)))
    li.with_bidiag(p, 1, 4)
    F = np.zeros((n, n))
    for a in range(n):
        b = p.perm[0, a]
        F[b, a] += 1.0
        F[(b + 1) % n, a] += float(p.dsign[0, (b + 1) % n])
    np.testing.assert_array_equal(oracle.multiplier_dense(p), F / np.sqrt(2.0))


def test_bidiag_product_structure():
    """The product of q factors: at most 2^q nonzeros per column, integer multiples
    of 2^{-q/2}, E[M^T M] = I (each factor has E[F^T F] = 2 I): the mean squared
    column norm over many columns is close to 1."""
    n, q = 400, 4
    p = li.Problem(li.SRC_DENSE, 3, n, W=np.zeros((3, n)))
    li.with_bidiag(p, q, 11)
    M = oracle.multiplier_dense(p) * 2.0 ** (q / 2)
    assert (M != 0).sum(0).max() <= 2 ** q
    np.testing.assert_array_equal(M, np.round(M))
    assert abs(np.mean((M ** 2).sum(0)) / 2 ** q - 1.0) < 0.05


def test_bidiag_twenty_factors_dense_columns():
    """The paper's 20-factor products (n = 48 < 2^20): every column fills at
    most n slots; the slot list equals the left-to-right dense product exactly
    (integers), and the gathered strip W M agrees with numpy's product."""
    n, q = 48, 20
    g = np.random.default_rng(3)
    W = g.standard_normal((6, n))
    p = li.Problem(li.SRC_DENSE, 6, n, W=W)
    li.with_bidiag(p, q, 13)
    rows, vals = oracle.bidiag_columns(n, q, p.perm, p.dsign)
    assert rows.shape == (n, n)
    M = oracle.multiplier_dense(p) * 2.0 ** (q / 2)
    np.testing.assert_array_equal(M, np.round(M))
    assert np.abs(M).max() <= 2.0 ** q
    S = np.zeros((n, n))
    for j in range(n):
        nz = vals[j] != 0
        assert np.all(np.diff(rows[j][nz]) > 0)
        S[rows[j][nz], j] = vals[j][nz]
    np.testing.assert_array_equal(S, M)
    R = oracle.gather_rows(p, np.arange(6, dtype=np.int32))
    ref = W @ (M * 2.0 ** (-q / 2))
    np.testing.assert_allclose(R, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_hmt11_laplacian_spectrum_closed_form():
    """The single-layer Laplacian input (bidiagonal pre-processing tests, inputs
    (i)) is circulant: log|2 e^{it} - e^{if}| = ln 2 - sum_m 2^-m cos(m(t-f)) / m,
    so its singular values are psi * 2 pi ln 2 = 1 once and
    psi * pi 2^-m / m * sinc(pi m / n) twice for m = 1, 2, ... (the sinc from
    averaging e^{imf} over an arc), up to aliasing terms of size 2^-(n-m)."""
    n = 256
    p = li.hmt11_laplacian(n)
    psi = 1.0 / (2.0 * np.pi * np.log(2.0))
    sv = np.linalg.svd(p.W, compute_uv=False)
    m = np.arange(1, 40)
    lam = psi * np.pi * 2.0 ** -m / m * np.sin(np.pi * m / n) / (np.pi * m / n)
    expected = np.sort(np.concatenate([[1.0], lam, lam]))[::-1][:40]
    np.testing.assert_allclose(sv[:40], expected, rtol=1e-8)
    np.testing.assert_allclose(p.W.sum(axis=1), 1.0, rtol=1e-13)


def test_hmt11_laplacian_entries_by_adaptive_quadrature():
    """Entries against scipy's adaptive quadrature of psi * log|2 w^i - y| over arc j."""
    from scipy.integrate import quad
    n = 64
    p = li.hmt11_laplacian(n)
    psi = 1.0 / (2.0 * np.pi * np.log(2.0))
    for i, j in [(0, 0), (5, 9), (63, 1), (17, 40), (32, 0)]:
        z = 2.0 * np.exp(2j * np.pi * i / n)
        v, _ = quad(lambda f: np.log(abs(z - np.exp(1j * f))), 2 * np.pi * j / n, 2 * np.pi * (j + 1) / n,
                    epsabs=1e-15, epsrel=1e-13)
        assert abs(p.W[i, j] - psi * v) <= 1e-14 * max(abs(psi * v), 1e-3), (i, j)


def test_hmt11_laplacian_ca_with_twenty_bidiagonal_factors():
    """C-A (five loops, as in Tests 2) on the 20-factor pre-processed input: the
    spectral error stays within a small factor of sigma_{k+1}."""
    n = 256
    for k, seed in [(31, 0), (39, 1), (35, 2)]:
        p = li.hmt11_laplacian(n)
        li.with_bidiag(p, 20, 100 + seed)
        o = oracle.ca_run(p, k, 5, li.initial_rows(n, k, seed))
        sv = np.linalg.svd(p.W, compute_uv=False)
        err = np.linalg.norm(p.W - o["C"] @ o["U"] @ o["R"], 2)
        assert sv[k] <= err <= 10 * sv[k], (k, err, sv[k])


def test_float32_input_is_widened_exactly():
    W = np.random.default_rng(0).standard_normal((10, 12)).astype(np.float32)
    p = li.Problem(li.SRC_DENSE, 10, 12, W=W)
    np.testing.assert_array_equal(oracle.gather_rows(p, np.array([2, 5], np.int32)), W[[2, 5]].astype(np.float64))


# ------------------------------------------------------------------ kernels
def test_laplace_entries_closed_form_values():
    """1/|x - y| at points with known distances (3-4-12 -> 13)."""
    X = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 3.0]])
    Y = np.array([[3.0, 4.0, 12.0], [1.0, 2.0, 5.0]])
    p = li.Problem(li.SRC_LAPLACE, 2, 2, X=X, Y=Y)
    R = oracle.gather_rows(p, np.array([0, 1], np.int32))
    assert R[0, 0] == 1.0 / 13.0 and R[1, 1] == 0.5


def test_gaussian_entries_closed_form_values():
    X = np.array([[0.0, 0.0, 0.0]])
    Y = np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 0.0]])
    p = li.Problem(li.SRC_GAUSSIAN, 1, 2, X=X, Y=Y, ell=0.3)
    R = oracle.gather_rows(p, np.array([0], np.int32))
    assert R[0, 0] == 1.0 and abs(R[0, 1] - math.exp(-0.5)) < 1e-16


def test_separated_laplace_block_error_decays_with_rank():
    """Interactions of well-separated clusters have low numerical rank: the
    C-A CUR error falls fast as k grows."""
    p = li.laplace_clusters(300, 280, seed=1)
    X, Y = p.X, p.Y
    K = 1.0 / np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=2)
    errs = []
    sig = np.linalg.svd(K, compute_uv=False)
    for k in (2, 4, 8, 12, 16):
        o = oracle.ca_run(p, k, 3, li.initial_rows(300, k, 2))
        err = np.linalg.norm(K - o["C"] @ o["U"] @ o["R"]) / np.linalg.norm(K)
        best = np.sqrt(np.sum(sig[k:] ** 2)) / np.linalg.norm(K)     # Eckart-Young optimum
        assert best <= err < 30 * best
        errs.append(err)
    assert errs[-1] < 1e-5 and all(b < a for a, b in zip(errs, errs[1:]))


def _fl64(q):
    """Round an exact rational to the nearest double (CPython int / int is correctly rounded)."""
    return float(q.numerator / q.denominator) if q.denominator != 1 else float(q.numerator)


def _laplace_f32_exact(x, y):
    """The FP32 Laplace entry from its definition, with exact rational arithmetic for
    the FP64 squared distance r2 = fma(dz, dz, fma(dy, dy, dx*dx)) and numpy's IEEE
    single-precision square root and quotient."""
    from fractions import Fraction as F
    dx, dy, dz = (float(np.float64(a) - np.float64(b)) for a, b in zip(x, y))
    dxx = float(np.float64(dx) * np.float64(dx))
    t = _fl64(F(dy) * F(dy) + F(dxx))
    r2 = _fl64(F(dz) * F(dz) + F(t))
    s = np.sqrt(np.float32(r2))
    return float(np.float32(1.0) / s)


def test_laplace_f32_entries_follow_their_definition():
    """Kernel entries in FP32: fl32(1 / fl32(sqrt(fl32(r2)))), r2 the fused FP64
    squared distance; checked entry by entry against exact rational r2 and numpy's
    single-precision operations, including nearly coincident and far points."""
    g = np.random.default_rng(11)
    X = g.random((24, 3))
    Y = np.concatenate([g.random((20, 3)) + [3.0, 0.0, 0.0], X[:4] + 1e-9 * g.standard_normal((4, 3))])
    p = li.Problem(li.SRC_LAPLACE, 24, 24, X=X, Y=Y, entries="f32")
    R = oracle.gather_rows(p, np.arange(24, dtype=np.int32))
    for i in range(24):
        for j in range(24):
            assert R[i, j] == _laplace_f32_exact(X[i], Y[j]), (i, j)


def test_laplace_f32_entries_relative_error_bound():
    """Three correctly rounded FP32 operations: |w32 / w64 - 1| <= (1/2 + 1 + 1) 2^-24 + O(2^-48)."""
    p = li.laplace_clusters(300, 280, seed=5)
    q = li.Problem(li.SRC_LAPLACE, 300, 280, X=p.X, Y=p.Y, entries="f32")
    rows = np.arange(300, dtype=np.int32)
    W64, W32 = oracle.gather_rows(p, rows), oracle.gather_rows(q, rows)
    rel = np.abs(W32 / W64 - 1.0)
    assert rel.max() <= 2.5 * 2.0 ** -24 * (1 + 1e-6)
    assert np.all(W32 == W32.astype(np.float32))      # every entry is an FP32 number
    assert rel.max() > 0                               # and they differ from the FP64 entries


def test_laplace_f32_kernel_run_equals_dense_f32_run():
    """A C-A run that evaluates the FP32 kernel entries on demand equals the run on the
    dense FP32 matrix of the same entries (gathers, core and outputs use one definition)."""
    p = li.laplace_clusters(260, 230, seed=6)
    q = li.Problem(li.SRC_LAPLACE, 260, 230, X=p.X, Y=p.Y, entries="f32")
    W32 = oracle.gather_rows(q, np.arange(260, dtype=np.int32)).astype(np.float32)
    d = li.Problem(li.SRC_DENSE, 260, 230, W=W32)
    I0 = li.initial_rows(260, 12, 4)
    a, b = oracle.ca_run(q, 12, 3, I0), oracle.ca_run(d, 12, 3, I0)
    for key in ("I", "J", "C", "U", "R", "logvol"):
        np.testing.assert_array_equal(a[key], b[key])
    assert (a["swaps"], a["loops"], a["status"]) == (b["swaps"], b["loops"], b["status"])


def test_laplace_f32_entries_error_against_fp64_matrix():
    """With FP32 entries the CUR of the separated clusters still approximates the FP64
    matrix to <= 1e-6 relative Frobenius error at k = 24 (the FP32 perturbation adds at
    most 1.25 * 2^-23 relative per entry, about 1.5e-7 in the Frobenius ratio)."""
    p = li.laplace_clusters(400, 350, seed=7)
    q = li.Problem(li.SRC_LAPLACE, 400, 350, X=p.X, Y=p.Y, entries="f32")
    K = oracle.gather_rows(p, np.arange(400, dtype=np.int32))
    I0 = li.initial_rows(400, 24, 1)
    o64, o32 = oracle.ca_run(p, 24, 3, I0), oracle.ca_run(q, 24, 3, I0)
    e64 = np.linalg.norm(K - o64["C"] @ o64["U"] @ o64["R"]) / np.linalg.norm(K)
    e32 = np.linalg.norm(K - o32["C"] @ o32["U"] @ o32["R"]) / np.linalg.norm(K)
    assert e64 < 1e-6 and e32 < 1e-6, (e64, e32)
    assert e32 <= 1.5 * e64 + 1.25 * 2.0 ** -23


# ------------------------------------------------------------------ adaptive generator size
def test_adaptive_single_stage_is_the_fixed_run():
    p = li.laplace_clusters(300, 280, seed=3)
    I0 = li.initial_rows(300, 20, 2)
    a = oracle.ca_run_adaptive(p, (20,), 2, 3, I0)
    b = oracle.ca_run(p, 20, 3, I0, rank_tol=1e-6)
    for key in ("I", "J", "C", "U", "R", "logvol"):
        np.testing.assert_array_equal(a[key], b[key])
    assert (a["k"], a["stages"], a["swaps"], a["loops"]) == (20, 1, b["swaps"], b["loops"])


@pytest.mark.parametrize("r, kf, nst", [(5, 8, 1), (13, 16, 2), (20, 32, 3)])
def test_adaptive_exact_low_rank_recovery(r, kf, nst):
    """Rank-r W = A B (Theorem thdcmp: W = CUR once the core has rank r): the
    stages 8, 16, 32 with margin 2 grow until the core rank r < k - 2."""
    g = np.random.default_rng(r)
    W = g.standard_normal((90, r)) @ g.standard_normal((r, 70))
    p = li.Problem(li.SRC_DENSE, 90, 70, W=W)
    o = oracle.ca_run_adaptive(p, (8, 16, 32), 2, 3, li.initial_rows(90, 32, 4), rank_tol=1e-9)
    assert (o["k"], o["stages"], o["rank"]) == (kf, nst, r)
    assert np.linalg.norm(W - o["C"] @ o["U"] @ o["R"]) <= 1e-9 * np.linalg.norm(W)


def test_adaptive_next_stage_starts_from_current_rows():
    """Stage 2 is the fixed run of size k_2 from the stage-1 rows followed by the
    caller's rows not among them, in order."""
    p = li.laplace_clusters(500, 450, seed=8)
    I0 = li.initial_rows(500, 40, 6)
    a = oracle.ca_run_adaptive(p, (12, 40), 0, 3, I0)
    s1 = oracle.ca_run(p, 12, 3, I0[:12], rank_tol=1e-6)
    assert s1["rank"] >= 12 and a["stages"] == 2
    rest = [i for i in I0 if i not in set(s1["I"].tolist())]
    I2 = np.concatenate([s1["I"], np.array(rest[:28], np.int32)])
    b = oracle.ca_run(p, 40, 3, I2, rank_tol=1e-6)
    for key in ("I", "J", "C", "U", "R"):
        np.testing.assert_array_equal(a[key], b[key])
    assert a["swaps"] == s1["swaps"] + b["swaps"] and a["loops"] == s1["loops"] + b["loops"]


def test_adaptive_fmm_blocks_accuracy_and_size():
    """Octree interaction blocks of the Laplace kernel: with stages 28, 40, 64 and
    margin 2 every block ends within 1e-6 relative Frobenius error, with a final
    size at least the numerical rank at 1e-6 (the paper's rank(., 1e-6)) and the
    stop rule met."""
    p, blocks, lev = li.fmm_blocks(npts=1 << 16, nblocks=256, seed=4)
    I0s = li.block_initial_rows(blocks, 64, 3)
    for b in np.random.default_rng(0).choice(len(blocks), 10, replace=False):
        r0, nr, c0, nc = blocks[b]
        s = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=p.X[r0:r0 + nr], Y=p.Y[c0:c0 + nc])
        o = oracle.ca_run_adaptive(s, (28, 40, 64), 2, 3, I0s[b])
        K = oracle.gather_rows(s, np.arange(s.m, dtype=np.int32))
        sv = np.linalg.svd(K, compute_uv=False)
        err = np.linalg.norm(K - o["C"] @ o["U"] @ o["R"]) / np.linalg.norm(K)
        assert err <= 1e-6 and o["k"] >= int((sv > 1e-6 * sv[0]).sum())
        assert o["rank"] < o["k"] - 2 or o["k"] == min(64, nr, nc)


# ------------------------------------------------------------------ cynical algorithms (Tests 3, 4)
def _sketch_sets(n, r, seed):
    g = np.random.default_rng(seed)
    q = 4 * r
    return q, g.choice(n, q, replace=False), g.choice(n, q, replace=False), g.choice(q, r, replace=False)


def test_cynical_error_band_from_paper_table():
    """Table tb_ranrc (Tests 3 and 4, n = 256..1024, r = 8, 16): our mean relative
    spectral error is at most the paper's printed mean, and above the 1e-10 noise
    floor's order."""
    with open(os.path.join(GOLDEN, "tests34_error_table.txt")) as f:
        rows = [line.split() for line in f if line.strip() and not line.startswith("#")]
    for test, n, r, mean, _ in rows:
        test, n, r, mean = int(test), int(n), int(r), float(mean)
        errs = []
        for seed in range(6):
            p = li.factor_gaussian(n, r, 1e-10, seed)
            q, K, L, I0s = _sketch_sets(n, r, 700 + seed)
            o = oracle.cynical(p, test - 3, r, q, K if test == 3 else None, L, I0s, sweeps=5)
            E = p.W - o["C"] @ o["U"] @ o["R"]
            errs.append(np.linalg.norm(E, 2) / np.linalg.norm(p.W, 2))
        assert np.mean(errs) <= mean, (test, n, r, np.mean(errs))
        assert np.min(errs) > 1e-13


@pytest.mark.parametrize("kind", [0, 1])
def test_cynical_exact_recovery_rank_r(kind):
    """Theorem thdcmp: W = CUR once the r x r generator of a rank-r W is nonsingular."""
    g = np.random.default_rng(40 + kind)
    W = g.standard_normal((300, 6)) @ g.standard_normal((6, 250))
    p = li.Problem(li.SRC_DENSE, 300, 250, W=W)
    q, K, L, I0s = _sketch_sets(250, 6, 9)
    o = oracle.cynical(p, kind, 6, q, K, L, I0s)
    assert o["rank"] == 6 and o["status"] in (0, 16)
    assert np.linalg.norm(W - o["C"] @ o["U"] @ o["R"]) <= 1e-10 * np.linalg.norm(W)
    assert set(o["I"]) <= set(o["K"]) and set(o["J"]) <= set(o["L"])


def test_cynical_generator_dominant_in_sketch():
    """Tests 3: when the sketch C-A converged, the generator B = S[I', J'] is dominant
    in the sketch S = W[K, L] both ways: max |S[:, J'] B^-1| <= h and max |B^-1 S[I', :]| <= h
    (Lemma lelcliden's condition, checked with numpy.linalg.solve)."""
    for seed in range(4):
        p = li.factor_gaussian(256, 8, 1e-6, seed)
        q, K, L, I0s = _sketch_sets(256, 8, 900 + seed)
        o = oracle.cynical(p, 0, 8, q, K, L, I0s, sweeps=8)
        if o["loops"] >= 8:
            continue
        S = p.W[np.ix_(K, L)]
        Ip = [list(K).index(i) for i in o["I"]]
        Jp = [list(L).index(j) for j in o["J"]]
        B = S[np.ix_(Ip, Jp)]
        assert np.abs(np.linalg.solve(B, S[Ip, :])).max() <= 1.01 + 1e-9
        assert np.abs(np.linalg.solve(B.T, S[:, Jp].T)).max() <= 1.01 + 1e-9


def test_cynical_one_loop_sketch_sets_are_dominant():
    """Tests 4: K is a dominant row set of the column strip W[:, L0] (L0 the caller's
    columns) and the final L a dominant column set of the row strip W[K, :]."""
    p = li.factor_gaussian(512, 8, 1e-8, 3)
    q, _, L0, I0s = _sketch_sets(512, 8, 77)
    o = oracle.cynical(p, 1, 8, q, None, L0, I0s)
    K, L = o["K"], o["L"]
    A = p.W[:, L0]
    assert np.abs(np.linalg.solve(A[K, :].T, A.T)).max() <= 1.01 + 1e-9
    Rk = p.W[K, :]
    assert np.abs(np.linalg.solve(Rk[:, L], Rk)).max() <= 1.01 + 1e-9


def test_cynical_sketch_of_generator_size_keeps_it():
    """q = r: the sketch is the generator itself, so I, J are K, L reordered."""
    p = li.factor_gaussian(200, 5, 1e-6, 1)
    g = np.random.default_rng(2)
    K, L = g.choice(200, 5, replace=False), g.choice(200, 5, replace=False)
    o = oracle.cynical(p, 0, 5, 5, K, L, np.arange(5))
    assert sorted(o["I"]) == sorted(K) and sorted(o["J"]) == sorted(L)


# ------------------------------------------------------------------ rectangular generators
@pytest.mark.parametrize("k,l", [(1, 5), (4, 9), (6, 6), (8, 20)])
def test_nucleus_rect_full_rank_is_pinv(k, l):
    G = np.random.default_rng(k * l).standard_normal((k, l))
    U, r = oracle.nucleus_rect(G, 1e-13)
    assert r == k
    np.testing.assert_allclose(U, np.linalg.pinv(G), atol=1e-12 * np.abs(np.linalg.pinv(G)).max())


def test_nucleus_rect_exact_low_rank_is_pinv():
    """G = A B of exact rank 3 (k = 6, l = 11): the truncated nucleus is its pseudo-inverse."""
    g = np.random.default_rng(3)
    G = g.standard_normal((6, 3)) @ g.standard_normal((3, 11))
    U, r = oracle.nucleus_rect(G, 1e-10)
    assert r == 3
    np.testing.assert_allclose(U, np.linalg.pinv(G, rcond=1e-10), atol=1e-11 * np.abs(U).max())


def test_oversample_each_step_maximises_the_volume():
    """Algorithm algrup: every added column maximises det(C_{g+1} C_{g+1}^T) over all
    columns outside the generator (brute force with numpy determinants)."""
    p = li.dense_lowrank(50, 60, r=10, noise=1e-6, seed=2)
    o = oracle.ca_run(p, 4, 3, li.initial_rows(50, 4, 1))
    ov = oracle.oversample(p, o["I"], o["J"], 5)
    assert ov["l"] == 9
    W = p.W
    Jp = list(ov["J"])
    for g in range(4, 9):
        base = Jp[:g]
        dets = []
        for q in range(60):
            if q in base:
                dets.append(-1.0)
                continue
            Cg = W[np.ix_(o["I"], base + [q])]
            dets.append(np.linalg.det(Cg @ Cg.T))
        best = int(np.argmax(dets))
        assert dets[Jp[g]] >= dets[best] * (1 - 1e-9), (g, Jp[g], best)


def test_oversample_zero_is_the_square_generator():
    p = li.dense_lowrank(80, 70, r=6, noise=1e-7, seed=4)
    o = oracle.ca_run(p, 6, 3, li.initial_rows(80, 6, 2))
    ov = oracle.oversample(p, o["I"], o["J"], 0)
    assert ov["l"] == 6
    np.testing.assert_array_equal(ov["J"], o["J"])
    np.testing.assert_array_equal(ov["C"], o["C"])
    U, _ = oracle.nucleus_rect(p.W[np.ix_(o["I"], o["J"])], 1e-13)
    np.testing.assert_array_equal(ov["U"], U)


def test_oversampled_generators_reduce_the_error():
    """Theorem th3: wider generators (k x l, l > k) lower the CUR error bound; on
    inputs with a decaying spectrum the mean error falls as columns are added and
    stays above the Eckart-Young optimum of rank k."""
    means = []
    for pe in (0, 4, 12):
        errs = []
        for seed in range(6):
            p = li.dense_lowrank(200, 180, r=20, noise=1e-9, seed=seed)
            o = oracle.ca_run(p, 8, 3, li.initial_rows(200, 8, seed))
            ov = oracle.oversample(p, o["I"], o["J"], pe)
            E = p.W - ov["C"] @ ov["U"] @ ov["R"]
            sv = np.linalg.svd(p.W, compute_uv=False)
            errs.append(np.linalg.norm(E, 2) / sv[8])
            assert errs[-1] >= 1 - 1e-9
        means.append(np.mean(errs))
    assert means[0] > means[1] > means[2], means


# ------------------------------------------------------------------ Gaussian-sampling CUR
def test_rhtcur_recovers_exact_low_rank():
    """Algorithm algrhtcur: on an exact rank-k input with a Gaussian Hbar (n x k)
    the CUR reproduces W to rounding."""
    for seed in range(3):
        p = li.factor_gaussian(300, 10, 0.0, seed=seed)
        H = np.random.default_rng(seed).standard_normal((300, 10))
        o = oracle.rhtcur(p, H)
        assert o["status"] == 0 and o["rank"] == 10 and o["loops"] == 2
        assert np.linalg.norm(p.W - o["C"] @ o["U"] @ o["R"]) <= 1e-12 * np.linalg.norm(p.W)


def test_rhtcur_selections_are_dominant():
    """Step 2 picks rows I whose k x k submatrix of S = W Hbar is h-dominant in S
    (|S S_I^{-1}| <= h), step 3 columns J with W[I, J] h-dominant in W[I, :];
    C, R are the gathered W[:, J], W[I, :] and U the inverse of W[I, J]."""
    h = 1.05
    for seed in range(4):
        p = li.dense_lowrank(200, 180, r=20, noise=1e-6, seed=seed)
        H = np.random.default_rng(10 + seed).standard_normal((180, 8))
        o = oracle.rhtcur(p, H, h=h)
        S = p.W @ H
        assert np.abs(S @ np.linalg.inv(S[o["I"], :])).max() <= h * (1 + 1e-9)
        B = p.W[np.ix_(o["I"], o["J"])]
        assert np.abs(np.linalg.solve(B, p.W[o["I"], :])).max() <= h * (1 + 1e-9)
        np.testing.assert_array_equal(o["C"], p.W[:, o["J"]])
        np.testing.assert_array_equal(o["R"], p.W[o["I"], :])
        np.testing.assert_allclose(o["U"] @ B, np.eye(8), atol=1e-8)


def test_rhtcur_with_a_selection_matrix_samples_columns():
    """Hbar = the first k columns of the identity makes S = W[:, :k] exactly
    (every fma adds an exact zero or the entry itself): the rows are those of a
    dominant submatrix of W[:, :k]."""
    p = li.dense_lowrank(120, 90, r=6, noise=1e-7, seed=5)
    H = np.eye(90)[:, :6]
    o = oracle.rhtcur(p, H, h=1.01)
    S = p.W[:, :6]
    assert np.abs(S @ np.linalg.inv(S[o["I"], :])).max() <= 1.01 * (1 + 1e-12)


def test_rhtcur_error_near_optimal_on_decaying_spectra():
    p = li.dense_lowrank(400, 350, r=20, noise=1e-9, seed=3)
    sv = np.linalg.svd(p.W, compute_uv=False)
    for k, seed in [(8, 0), (12, 1)]:
        H = np.random.default_rng(seed).standard_normal((350, k))
        o = oracle.rhtcur(p, H)
        err = np.linalg.norm(p.W - o["C"] @ o["U"] @ o["R"], 2)
        assert sv[k] <= err <= 20 * sv[k], (k, err / sv[k])


# ------------------------------------------------------------------ leverage-score sampling inside C-A
def test_jacobi_eigendecomposition():
    """The round-robin Jacobi sweeps diagonalise a symmetric matrix: eigenvalues
    equal LAPACK's, G = Q diag Q^T, Q orthogonal."""
    g = np.random.default_rng(1)
    for k in (1, 2, 7, 16, 33):
        A = g.standard_normal((k, 3 * k + 5))
        G0 = A @ A.T
        D, Q = oracle.jacobi_eig(G0)
        off = D - np.diag(np.diag(D))
        assert np.abs(off).max() <= 1e-14 * np.abs(G0).max()
        np.testing.assert_allclose(np.sort(np.diag(D)), np.linalg.eigvalsh(G0), rtol=1e-11, atol=1e-13)
        assert np.abs(Q @ np.diag(np.diag(D)) @ Q.T - G0).max() <= 1e-13 * np.abs(G0).max()
        assert np.abs(Q.T @ Q - np.eye(k)).max() <= 1e-13


def test_leverage_scores_are_the_row_norms_of_the_top_singular_vectors():
    """Eq. eqlevsc with beta = 1: v_j = ||V^(r)[j, :]||^2 for the top-r right
    singular vectors (numpy's SVD), summing to r; eigenvalues below 1e-12 of the
    largest (sigma below 1e-6 sigma_max) are left out."""
    g = np.random.default_rng(2)
    A = g.standard_normal((12, 5)) @ np.diag(2.0 ** -np.arange(5)) @ g.standard_normal((5, 200))
    A += 1e-9 * g.standard_normal(A.shape)
    _, sv, Vt = np.linalg.svd(A, full_matrices=False)
    for r in (1, 3, 5):
        v, used = oracle.lev_scores(A, r)
        assert used == r
        np.testing.assert_allclose(v, (Vt[:r] ** 2).sum(axis=0), atol=1e-11)
        assert abs(v.sum() - r) <= 1e-10
    v, used = oracle.lev_scores(A, 9)            # sigma_6.. ~ 1e-9 sigma_1: left out
    assert used == 5


def test_exactly_sampling_is_the_inverse_cdf():
    """Algorithm algsmplex: draw t picks the smallest j with cum_j > u_t total;
    zero-score indices are never picked; u near 1 falls back to the last
    positive score."""
    v = np.array([0.0, 1.0, 0.0, 2.0, 3.0, 0.0, 4.0, 0.0])
    cum, tot = np.cumsum(v), v.sum()
    u = np.array([0.0, 0.05, 0.1 - 1e-12, 0.1, 0.35, 0.6, 0.999999, 1.0 - 2.0 ** -53])
    got = oracle.lev_sample(v, len(u), 0, u)
    ref = [int(np.argmax(cum > x * tot)) if (cum > x * tot).any() else 6 for x in u]
    np.testing.assert_array_equal(got, ref)
    assert not set(got) & {0, 2, 5, 7}


def test_exactly_sampling_frequencies_follow_the_scores():
    g = np.random.default_rng(3)
    v = g.random(20) ** 2
    u = g.random(200000)
    got = oracle.lev_sample(v, len(u), 0, u)
    freq = np.bincount(got, minlength=20) / len(u)
    p = v / v.sum()
    assert np.abs(freq - p).max() <= 5 * np.sqrt(p.max() / len(u))


def test_expected_sampling_keeps_each_index_with_its_probability():
    """Algorithm algsmplexp: j (ascending) is kept when u_j < min(1, l p_j), at
    most l of them; nothing kept -> the largest score."""
    v = np.array([4.0, 1.0, 0.0, 3.0, 2.0])
    l, tot = 2, v.sum()
    u = np.array([0.79, 0.21, 0.0, 0.59, 0.3])
    pr = np.minimum(1.0, l * v / tot)               # 0.8 0.2 0 0.6 0.4
    ref = [j for j in range(5) if u[j] < pr[j]][:l]
    np.testing.assert_array_equal(oracle.lev_sample(v, l, 1, u), ref)
    np.testing.assert_array_equal(oracle.lev_sample(v, l, 1, np.full(5, 0.9999)), [0])


@pytest.mark.parametrize("kind", [0, 1])
def test_ca_with_leverage_sampling_recovers_low_rank(kind):
    """C-A iterations with DMM08 Algorithm 1 on the sketches (k = 2r, 4r samples
    per step) reproduce an exact rank-r input."""
    g = np.random.default_rng(4)
    for k, seed in [(16, 0), (32, 1)]:
        p = li.factor_gaussian(300, 8, 0.0, seed=seed)
        o = oracle.ca_lev(p, k, 8, 8, kind, g.random(2 * 8 * 300), li.initial_rows(300, k, seed))
        assert o["rank"] == 8 and o["kI"] <= k and o["kJ"] <= k
        assert np.linalg.norm(p.W - o["C"] @ o["U"] @ o["R"]) <= 1e-10 * np.linalg.norm(p.W)


def test_uniform_scores_sample_by_the_uniform_cdf():
    """Uniform scores (kind 2, 3) make the sampling independent of the sketch:
    Exactly(k) takes floor(u n) for each draw (the inverse CDF of 1/n), and
    Expected(k) keeps j ascending with u_j < k / n, at most k of them; the final
    sets come from the last iteration's draws."""
    p = li.dense_lowrank(90, 70, r=6, noise=1e-9, seed=1)
    it, k = 3, 10
    d = np.random.default_rng(5).random((2 * it, 90))
    I0 = li.initial_rows(90, k, 3)
    o = oracle.ca_lev(p, k, 6, it, 2, d, I0)
    np.testing.assert_array_equal(o["J"], np.floor(d[2 * it - 2][:k] * 70).astype(int))
    np.testing.assert_array_equal(o["I"], np.floor(d[2 * it - 1][:k] * 90).astype(int))
    o = oracle.ca_lev(p, k, 6, it, 3, d, I0)
    np.testing.assert_array_equal(o["J"], np.flatnonzero(d[2 * it - 2][:70] < k / 70)[:k])
    np.testing.assert_array_equal(o["I"], np.flatnonzero(d[2 * it - 1][:90] < k / 90)[:k])


@pytest.mark.parametrize("kind", [2, 3])
def test_uniform_scores_suffice_for_factor_gaussian_inputs(kind):
    """The section on superfast leverage scores: for a perturbed factor-Gaussian
    input with r << n the leverage scores are nearly uniform (chi-square
    concentration, Lemma lmchitail), so sampling 4r rows and columns uniformly
    gives a CUR within a small factor of the perturbation, as the SVD-based
    scores do."""
    g = np.random.default_rng(9)
    for seed in range(4):
        p = li.factor_gaussian(400, 8, 1e-10, seed=seed)
        d = g.random(2 * 3 * 400)
        I0 = li.initial_rows(400, 32, seed)
        u = oracle.ca_lev(p, 32, 8, 3, kind, d, I0)
        s = oracle.ca_lev(p, 32, 8, 3, kind - 2, d, I0)
        eu = np.linalg.norm(p.W - u["C"] @ u["U"] @ u["R"]) / np.linalg.norm(p.W)
        es = np.linalg.norm(p.W - s["C"] @ s["U"] @ s["R"]) / np.linalg.norm(p.W)
        assert u["rank"] == 8 and eu <= 1e-8 and eu <= 10 * es, (seed, eu, es)


def _bidiag_dense(n, q, seed):
    """The oracle's product of q bidiagonal factors, as a dense integer matrix."""
    perms, signs = li.bidiag_descriptor(n, q, seed)
    rows, vals = oracle.bidiag_columns(n, q, perms, signs)
    cols = np.broadcast_to(np.arange(n)[:, None], rows.shape)
    m = vals != 0
    M = np.zeros((n, n))
    M[rows[m], cols[m]] = vals[m]
    return M


def test_bidiag_products_are_nearly_gaussian():
    """Theorem thm1 and the experiment of Figure LowRkTest1 (n = 1024, 20 random
    permuted cyclic bidiagonal factors).  Every factor doubles the expected
    squared norm of a column and the rows are exchangeable, so each entry has
    mean 0 and variance exactly 2^q / n.  After that scaling, one fixed entry
    taken over independent products passes the Kolmogorov-Smirnov test for
    N(0, 1), and two such entries are uncorrelated.  Over all 2^20 entries of
    one product the first four moments are Gaussian's and the KS distance is
    below 0.005."""
    st = pytest.importorskip("scipy.stats")
    n, q, reps = 1024, 20, 120
    sd = np.sqrt(2.0 ** q / n)
    a, b = [], []
    for rep in range(reps):
        M = _bidiag_dense(n, q, 3000 + rep)
        a.append(M[17, 400] / sd)
        b.append(M[900, 33] / sd)
        if rep < 2:
            x = M.ravel() / sd
            assert abs(x.mean()) < 0.01 and abs(x.var() - 1.0) < 0.03 and abs(st.kurtosis(x)) < 0.1
            jit = (M.ravel() + np.random.default_rng(rep).random(n * n) - 0.5) / sd   # continuous version
            assert st.kstest(jit, "norm").statistic < 0.005
    assert st.kstest(np.array(a), "norm").pvalue > 0.01
    assert st.kstest(np.array(b), "norm").pvalue > 0.01
    assert abs(np.corrcoef(a, b)[0, 1]) < 4.0 / np.sqrt(reps)


# ------------------------------------------------------------------ FMM partition and matvec
def test_fmm_partition_covers_every_entry_once_and_far_blocks_are_separated():
    """Far blocks (interaction lists of every level) and near blocks (touching
    leaves) cover each (i, j) exactly once; the boxes of a far block at level l
    are at least one box side (2^-l) apart."""
    p, far, near, L = li.fmm_partition(1 << 12, leaf=32, seed=1)
    cov = np.zeros((p.m, p.m), dtype=np.int32)
    for r0, nr, c0, nc, lev, tb in far:
        cov[r0:r0 + nr, c0:c0 + nc] += 1
        A, B = p.X[r0:r0 + nr], p.X[c0:c0 + nc]
        gap = np.max(np.maximum(A.min(0) - B.max(0), B.min(0) - A.max(0)))
        assert gap >= 2.0 ** -lev - 1e-12
    for r0, nr, c0, nc, tb in near:
        cov[r0:r0 + nr, c0:c0 + nc] += 1
    assert cov.min() == 1 and cov.max() == 1
    assert set(far[:, 4]) == set(range(2, L + 1))


def test_fmm_partition_with_cut_far_blocks_still_covers_once():
    """Far blocks cut into row and column pieces of at most max_block keep the
    exact cover, each piece stays well separated, and a row piece is a target
    group of its own (consecutive blocks, one row range per (level, target))."""
    p, far, near, L = li.fmm_partition(1 << 12, leaf=32, seed=1, max_block=40)
    assert far[:, 1].max() <= 40 and far[:, 3].max() <= 40
    cov = np.zeros((p.m, p.m), dtype=np.int32)
    for r0, nr, c0, nc, lev, tb in far:
        cov[r0:r0 + nr, c0:c0 + nc] += 1
        A, B = p.X[r0:r0 + nr], p.X[c0:c0 + nc]
        assert np.max(np.maximum(A.min(0) - B.max(0), B.min(0) - A.max(0))) >= 2.0 ** -lev - 1e-12
    for r0, nr, c0, nc, tb in near:
        cov[r0:r0 + nr, c0:c0 + nc] += 1
    assert cov.min() == 1 and cov.max() == 1
    keys = [(int(a), int(b)) for a, b in far[:, 4:6]]
    starts = [i for i in range(len(keys)) if i == 0 or keys[i] != keys[i - 1]]
    assert len(starts) == len(set(keys))                     # every group contiguous
    for i0, i1 in zip(starts, starts[1:] + [len(far)]):
        assert len({(int(r0), int(nr)) for r0, nr in far[i0:i1, :2]}) == 1


def _direct(P, x):
    d = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(axis=2))
    with np.errstate(divide="ignore"):
        K = np.where(d > 0.0, 1.0 / d, 0.0)
    return K @ x, K


def test_hmatvec_with_exact_generators_is_the_dense_product():
    p, far, near, L = li.fmm_partition(1 << 11, leaf=32, seed=2)
    x = li.rhs(p.m, 1, 3)[:, 0]
    y_ref, K = _direct(p.X, x)
    gens = [(K[r0:r0 + nr, c0:c0 + nc], np.eye(nc), np.eye(nc)) for r0, nr, c0, nc, _, _ in far]
    y = oracle.hmatvec(p, far, near, gens, x)
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()


def test_hmatvec_with_ca_generators_meets_the_tolerance():
    """Generators from staged C-A runs at tol 1e-6 (the FMM recipe): the
    matvec's relative error stays below 1e-5."""
    p, far, near, L = li.fmm_partition(1 << 12, leaf=64, seed=3)
    I0 = li.block_initial_rows(far[:, :4], 32, 4)
    gens = []
    for b, (r0, nr, c0, nc, lev, tb) in enumerate(far):
        sub = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=p.X[r0:r0 + nr], Y=p.X[c0:c0 + nc])
        o = oracle.ca_run_adaptive(sub, (16, 24, 32), 2, 3, I0[b], h=1.05, rank_tol=1e-6)
        gens.append((o["C"], o["U"], o["R"]))
    x = li.rhs(p.m, 1, 5)[:, 0]
    y_ref, _ = _direct(p.X, x)
    y = oracle.hmatvec(p, far, near, gens, x)
    assert np.linalg.norm(y - y_ref) <= 1e-5 * np.linalg.norm(y_ref)


# ------------------------------------------------------------------ expansion/contraction cycles
def _leverages(Rs, J):
    """s_q = b_q^T (A A^T)^{-1} b_q for every column b_q of Rs, A = Rs[:, J] (Theorem th2)."""
    A = Rs[:, list(J)]
    Gi = np.linalg.inv(A @ A.T)
    return np.einsum("ij,ik,kj->j", Rs, Gi, Rs)


def _greedy_expand(Rs, J, p):
    J = list(J)
    for _ in range(p):
        s = _leverages(Rs, J)
        s[J] = -np.inf
        js = int(np.argmax(s))
        if not s[js] > 0:
            break
        J.append(js)
    return J


def _cycles_by_definition(Rs, J0, pextra, pmax, max_cycles, h):
    """Section scrsorth's recipe from scratch: leverages and volumes recomputed
    from their definitions at every step (no Sherman-Morrison updates)."""
    n = Rs.shape[1]
    vol = lambda JJ: np.linalg.slogdet(Rs[:, JJ] @ Rs[:, JJ].T)[1]
    J = _greedy_expand(Rs, J0, pextra)
    cycles = ptried = 0
    pc, converged = 1, False
    while True:
        s = _leverages(Rs, J)
        out = np.ones(n, bool)
        out[J] = False
        if 1 + (s[out].max() if out.any() else 0.0) <= h:
            converged = True
            break
        if pc > pmax or cycles >= max_cycles:
            break
        ptried = max(ptried, pc)
        Jn = _greedy_expand(Rs, J, pc)
        added = len(Jn) - len(J)
        ok = added > 0
        for _ in range(added if ok else 0):
            s = _leverages(Rs, Jn)
            jr = min(Jn, key=lambda j: (s[j], j))
            if not s[jr] < 1:
                ok = False
                break
            Jn.remove(jr)
        if ok and set(Jn) != set(J) and vol(Jn) > vol(J):
            J, cycles, pc = Jn, cycles + 1, 1
        else:
            pc += 1
    return J, cycles, ptried, converged


def test_cycles_follow_the_definition():
    """The oracle's cycles (whitening updates of Theorem th2) take the same
    decisions as the recipe evaluated from the definitions of the leverages and
    volumes: the same final column list, kept cycles, largest p and outcome."""
    kept = 0
    for seed in range(16):
        p = li.dense_lowrank(60, 80, r=12, noise=1e-4, seed=seed)
        o = oracle.ca_run(p, 5, 3, li.initial_rows(60, 5, seed))
        ov = oracle.oversample(p, o["I"], o["J"], 3, h=1.05, pmax=3, max_cycles=20)
        J, cycles, ptried, converged = _cycles_by_definition(p.W[o["I"], :], o["J"], 3, 3, 20, 1.05)
        assert list(ov["J"]) == J, seed
        assert (ov["cycles"], ov["ptried"]) == (cycles, ptried), seed
        assert (ov["status"] == 0) == converged, seed
        kept += cycles
    assert kept > 5


def test_cycles_reach_the_colclmx_test():
    """A generator that fails Corollary colclmx's test after the greedy
    expansion (1 + max outside leverage > h) passes it after a kept cycle; the
    status says which (0, or LRA_WARN_NOT_CONVERGED)."""
    p = li.dense_lowrank(60, 80, r=6, noise=1e-3, seed=3)
    o = oracle.ca_run(p, 4, 3, li.initial_rows(60, 4, 3))
    Rs = p.W[o["I"], :]
    h = 1.25
    plain = oracle.oversample(p, o["I"], o["J"], 8, h=h)
    cyc = oracle.oversample(p, o["I"], o["J"], 8, h=h, pmax=4, max_cycles=20)
    smax = lambda J: np.delete(_leverages(Rs, J), list(J)).max()
    assert 1 + smax(plain["J"]) > h
    assert cyc["status"] == 0 and cyc["cycles"] >= 1
    assert 1 + smax(cyc["J"]) <= h
    stuck = oracle.oversample(p, o["I"], o["J"], 8, h=1.0001, pmax=4, max_cycles=20)
    assert stuck["status"] == 17 and stuck["ptried"] == 4


def test_cycles_never_lower_the_volume():
    """Each kept cycle raises det(C_l C_l^T); a large h keeps the plain greedy
    expansion (the test passes at once, no cycle)."""
    gains = []
    for seed in range(10):
        p = li.dense_lowrank(120, 150, r=16, noise=1e-5, seed=seed)
        o = oracle.ca_run(p, 6, 3, li.initial_rows(120, 6, seed))
        Rs = p.W[o["I"], :]
        plain = oracle.oversample(p, o["I"], o["J"], 6, h=1.05)
        cyc = oracle.oversample(p, o["I"], o["J"], 6, h=1.05, pmax=4, max_cycles=50)
        v = lambda J: np.linalg.slogdet(Rs[:, list(J)] @ Rs[:, list(J)].T)[1]
        gains.append(v(cyc["J"]) - v(plain["J"]))
        assert gains[-1] >= -1e-12, seed
        assert (gains[-1] > 0) == (cyc["cycles"] > 0), seed
        big = oracle.oversample(p, o["I"], o["J"], 6, h=1e6, pmax=4, max_cycles=50)
        assert big["status"] == 0 and big["cycles"] == 0 and big["ptried"] == 0
        np.testing.assert_array_equal(big["J"], plain["J"])
        np.testing.assert_array_equal(big["U"], plain["U"])
    assert max(gains) > 0


# ------------------------------------------------------------------ limits of superfast LRA
def test_delta_matrices_defeat_superfast_approximation():
    """Example exdlt: of the 2mn +-delta matrices (one entry +-1, the rest 0) a superfast
    algorithm approximates nearly half as poorly as the zero matrix, since it never
    reads most entries.  C-A with k = 2 on 12 x 12: at least 45% end with relative
    error >= 1."""
    m = n = 12
    I0 = np.array([3, 7], np.int32)
    fail = tot = 0
    for i in range(m):
        for j in range(n):
            for sgn in (1.0, -1.0):
                W = np.zeros((m, n))
                W[i, j] = sgn
                o = oracle.ca_run(li.Problem(li.SRC_DENSE, m, n, W=W), 2, 3, I0)
                err = np.linalg.norm(W - o["C"] @ o["U"] @ o["R"]) / np.linalg.norm(W)
                tot += 1
                fail += err >= 1 - 1e-12
    assert fail / tot >= 0.45, fail / tot


def test_residual_sample_sees_a_missed_delta_only_inside_its_sample():
    """Remark reerrdlt and the superfast a-posteriori estimate: on a +-delta matrix whose
    spike the CUR missed, the sampled residual is exactly 1 at the spike when the sample
    covers it and exactly 0 otherwise (a superfast check cannot verify such an output)."""
    m = n = 20
    W = np.zeros((m, n))
    W[13, 5] = -1.0
    p = li.Problem(li.SRC_DENSE, m, n, W=W)
    o = oracle.ca_run(p, 2, 3, np.array([0, 1], np.int32))
    assert np.abs(o["C"] @ o["U"] @ o["R"]).max() == 0.0            # the spike was never read
    hit = oracle.residual_sample(p, o["C"], o["U"], o["R"], np.array([2, 13, 17], np.int32),
                                 np.array([5, 9], np.int32))
    miss = oracle.residual_sample(p, o["C"], o["U"], o["R"], np.array([2, 12, 17], np.int32),
                                  np.array([5, 9], np.int32))
    assert hit[3] == 1.0 and hit[4] == 1.0 and miss[3] == 0.0 and miss[4] == 0.0


def test_log_volume_equals_log_det_of_the_final_core():
    """eq. eqb: every swap multiplies the volume by |c_ij|, every LUP pivot contributes
    its modulus, so the tracked log-volume of the last step is log|det W'[I, J]|."""
    for seed in range(4):
        p = li.factor_gaussian(150, 10, 1e-3, seed)
        o = oracle.ca_run(p, 8, 3, li.initial_rows(150, 8, seed))
        lv = o["logvol"][np.isfinite(o["logvol"])][-1]
        sign, ld = np.linalg.slogdet(p.W[np.ix_(o["I"], o["J"])])
        assert abs(lv - ld) <= 1e-9 * max(1.0, abs(ld)), (lv, ld)


def test_resuming_from_the_output_sets_keeps_the_volume():
    """Checkpoint / resume: a run restarted warm from the (I, J) of a finished run reaches
    a core of at least the same volume (the C-A volume never decreases); restarting cold
    from I alone does not guarantee it (a cold LUP may pick a smaller core)."""
    for seed in range(4):
        p = li.factor_gaussian(200, 12, 1e-4, seed)
        a = oracle.ca_run(p, 10, 1, li.initial_rows(200, 10, seed))
        b = oracle.ca_run(p, 10, 3, a["I"], J0=a["J"])
        va = np.linalg.slogdet(p.W[np.ix_(a["I"], a["J"])])[1]
        vb = np.linalg.slogdet(p.W[np.ix_(b["I"], b["J"])])[1]
        assert vb >= va - 1e-9


# ------------------------------------------------------------------ apply / residual
def test_cur_apply_matches_matmul():
    g = np.random.default_rng(0)
    C, U, R, X = g.standard_normal((30, 5)), g.standard_normal((5, 5)), g.standard_normal((5, 40)), g.standard_normal((40, 3))
    np.testing.assert_allclose(oracle.cur_apply(C, U, R, X), C @ (U @ (R @ X)), rtol=1e-13, atol=1e-13)


def test_residual_sample_full_equals_full_residual():
    """With Q = all rows and S = all columns the sample is the whole error matrix."""
    p = li.dense_lowrank(40, 30, r=3, noise=1e-4, seed=2)
    o = oracle.ca_run(p, 3, 2, li.initial_rows(40, 3, 0))
    Q = np.arange(40, dtype=np.int32); S = np.arange(30, dtype=np.int32)
    st, E = oracle.residual_sample(p, o["C"], o["U"], o["R"], Q, S, return_E=True)
    Eref = p.W - o["C"] @ o["U"] @ o["R"]
    np.testing.assert_allclose(E, Eref, atol=1e-15)
    assert math.isclose(st[0], Eref.mean(), rel_tol=1e-9, abs_tol=1e-18)
    assert math.isclose(st[1], Eref.var(), rel_tol=1e-9)
    assert math.isclose(st[2], np.abs(Eref).mean(), rel_tol=1e-12)
    assert st[3] == np.abs(Eref).max()
    assert math.isclose(st[4], np.linalg.norm(Eref) / np.linalg.norm(p.W), rel_tol=1e-12)


# ------------------------------------------------------------------ differentiable apply
def _gauss_case(seed=0, m=60, n=50, k=6, nrhs=3):
    g = np.random.default_rng(seed)
    X = g.random((m, 3)); Y = g.random((n, 3)); Y[:, 0] += 1.0
    I = np.sort(g.choice(m, k, replace=False)).astype(np.int32)
    J = np.sort(g.choice(n, k, replace=False)).astype(np.int32)
    return X, Y, I, J, g.standard_normal((n, nrhs)), g.standard_normal((m, nrhs))


def test_gauss_cur_apply_matches_dense_formula():
    """y = C G^{-1} R x with the sampled entries (closed-form kernel, LAPACK inverse)."""
    X, Y, I, J, x, _ = _gauss_case()
    ell = 0.4
    K = np.exp(-np.sum((X[:, None] - Y[None]) ** 2, axis=2) / (2 * ell ** 2))
    y, U, t1, t2 = oracle.gauss_cur_apply(X, Y, I, J, ell, x)
    yref = K[:, J] @ np.linalg.solve(K[np.ix_(I, J)], K[I] @ x)
    np.testing.assert_allclose(y, yref, rtol=1e-9, atol=1e-12 * np.abs(yref).max())


@pytest.mark.parametrize("seed", range(3))
def test_gauss_cur_backward_finite_differences(seed):
    """dL/dx, dL/dl and the entry gradients of L = <dy, y> against central
    finite differences of the forward in FP64."""
    X, Y, I, J, x, dy = _gauss_case(seed)
    ell = 0.45
    b = oracle.gauss_cur_backward(X, Y, I, J, ell, x, dy)
    L = lambda e, xx: float(np.sum(dy * oracle.gauss_cur_apply(X, Y, I, J, e, xx)[0]))
    h = 1e-6
    fd = (L(ell + h, x) - L(ell - h, x)) / (2 * h)
    assert abs(fd - b["dell"]) <= 1e-6 * max(1.0, abs(fd))
    xp = x.copy(); xp[3, 1] += h; xm = x.copy(); xm[3, 1] -= h
    fdx = (L(ell, xp) - L(ell, xm)) / (2 * h)
    assert abs(fdx - b["dx"][3, 1]) <= 1e-6 * max(1.0, abs(fdx))
    # entry gradients: perturb one entry of C, R, G through a dense re-evaluation
    K = np.exp(-np.sum((X[:, None] - Y[None]) ** 2, axis=2) / (2 * ell ** 2))
    C, R, G = K[:, J].copy(), K[I].copy(), K[np.ix_(I, J)].copy()
    f = lambda C_, R_, G_: float(np.sum(dy * (C_ @ np.linalg.solve(G_, R_ @ x))))
    for name, M, idx in (("dC", C, (7, 2)), ("dR", R, (1, 11)), ("dG", G, (3, 4))):
        Mp, Mm = M.copy(), M.copy(); Mp[idx] += h; Mm[idx] -= h
        args_p = dict(C_=C, R_=R, G_=G); args_m = dict(C_=C, R_=R, G_=G)
        key = {"dC": "C_", "dR": "R_", "dG": "G_"}[name]
        args_p[key] = Mp; args_m[key] = Mm
        fdv = (f(**args_p) - f(**args_m)) / (2 * h)
        assert abs(fdv - b[name][idx]) <= 1e-6 * max(1.0, abs(fdv)), (name, fdv, b[name][idx])


# ------------------------------------------------------------------ r-projective volume (Alg. alg1tor, algprjvlm)
def _vol_r(M, r):
    """r-projective volume v_{2,r}: the product of the r largest singular values."""
    return float(np.prod(np.linalg.svd(M, compute_uv=False)[:r]))


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("k,n", [(6, 30), (12, 40), (8, 8), (10, 6)])
def test_alg1tor_is_column_pivoted_qr(seed, k, n):
    """Algorithm alg1tor's greedy expansions are Householder QR with column
    pivoting: the same pivots as LAPACK's pivoted QR (scipy.linalg.qr), the same
    |R|, the column Gram matrix kept (the reflections are orthogonal), and the
    pivot columns exactly zero below their step."""
    sl = pytest.importorskip("scipy.linalg")
    A = np.random.default_rng(100 + seed).standard_normal((k, n))
    r, J0, Ah = oracle.alg1tor(A, tol=1e-13)
    q = min(k, n)
    assert r == q
    _, R, P = sl.qr(A, pivoting=True, mode="economic")
    np.testing.assert_array_equal(J0, P[:q])
    scale = np.linalg.norm(A)
    np.testing.assert_allclose(np.abs(np.triu(Ah[:q][:, J0])), np.abs(R[:q, :q]), rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(Ah.T @ Ah, A.T @ A, rtol=0, atol=1e-13 * scale ** 2)
    for g, j in enumerate(J0):
        assert np.all(Ah[g + 1:, j] == 0.0)


def test_alg1tor_numerical_rank():
    """The greedy sequence stops at the numerical rank: exact rank-r products
    give r (tol 1e-10), a generic matrix min(k, n), the zero matrix 0; the
    stop is the first |R_gg| <= tol |R_00| of LAPACK's pivoted QR."""
    sl = pytest.importorskip("scipy.linalg")
    g = np.random.default_rng(7)
    for (k, n, r) in [(10, 50, 4), (16, 30, 9), (8, 8, 1)]:
        A = g.standard_normal((k, r)) @ g.standard_normal((r, n))
        assert oracle.alg1tor(A, tol=1e-10)[0] == r
        d = np.abs(np.diag(sl.qr(A, pivoting=True, mode="economic")[1]))
        assert d[r - 1] > 1e-10 * d[0] >= d[r] if r < min(k, n) else True
        assert oracle.alg1tor(A + 1e-3 * g.standard_normal((k, n)), tol=1e-10)[0] == min(k, n)
    assert oracle.alg1tor(np.zeros((5, 9)))[0] == 0


def _prj_case(seed, r=6, k=10, m=70, n=90):
    p = li.dense_lowrank(m, n, r=r, noise=0.0, seed=seed)
    o = oracle.ca_run(p, k, 3, li.initial_rows(m, k, seed))
    return p, o


@pytest.mark.parametrize("seed", range(4))
def test_prjvol_swaps_then_expansions_maximise_r_projective_volume(seed):
    """Algorithm algprjvlm on a rank-r strip W[I, :] with k > r rows: the r
    columns after the swaps have locally h-maximal r-projective volume in the
    strip (no single exchange raises v_{2,r} by more than h), and each column
    Algorithm algrup appends maximises v_{2,r} of the grown set.  Every volume
    here comes from numpy singular values of the original strip (Lemma
    leprwnmp ties them to R')."""
    h, r = 1.01, 6
    p, o = _prj_case(seed, r=r)
    pv = oracle.prjvol(p, o["I"], o["J"], 2, h=h, rank_tol=1e-10)
    assert pv["srank"] == r and pv["l"] == 12
    A = p.W[o["I"], :]
    J = [int(j) for j in pv["J"]]
    base = _vol_r(A[:, J[:r]], r)
    for i in range(r):
        for q in range(p.n):
            if q in J[:r]:
                continue
            S = J[:r].copy()
            S[i] = q
            assert _vol_r(A[:, S], r) <= h * base * (1 + 1e-9), (i, q)
    for g in range(r, len(J)):
        vols = [(_vol_r(A[:, J[:g] + [q]], r) if q not in J[:g] else -1.0) for q in range(p.n)]
        assert _vol_r(A[:, J[:g + 1]], r) >= max(vols) * (1 - 1e-9), g


def test_prjvol_recovers_exact_low_rank_and_full_rank_strips_are_dominant():
    """On an exact rank-r input the k x l generator (k > r) reproduces W to
    rounding with the nucleus truncated at rank r; on a full-rank strip the
    first k columns are a dominant k x k submatrix of the strip (Lemma
    lelcliden: |B^{-1} A| <= h)."""
    for seed in range(3):
        p, o = _prj_case(seed, r=7)
        pv = oracle.prjvol(p, o["I"], o["J"], 3, rank_tol=1e-10)
        assert pv["srank"] == 7 and pv["rank"] == 7 and pv["status"] == 16
        assert np.linalg.norm(p.W - pv["C"] @ pv["U"] @ pv["R"]) <= 1e-12 * np.linalg.norm(p.W)
        np.testing.assert_array_equal(pv["C"], p.W[:, pv["J"]])
        np.testing.assert_array_equal(pv["R"], p.W[o["I"], :])
    h = 1.01
    p = li.dense_lowrank(60, 80, r=12, noise=1e-3, seed=5)
    o = oracle.ca_run(p, 8, 3, li.initial_rows(60, 8, 5))
    pv = oracle.prjvol(p, o["I"], o["J"], 0, h=h, rank_tol=1e-10)
    assert pv["srank"] == 8 and pv["l"] == 8 and pv["status"] == 0
    A = p.W[o["I"], :]
    assert np.abs(np.linalg.solve(A[:, pv["J"]], A)).max() <= h * (1 + 1e-12)


def test_prjvol_degenerate_cases():
    """A zero strip keeps the square generator (r = 0); with no swaps allowed
    the first r columns are Algorithm alg1tor's pivots; l is clipped at n."""
    p = li.Problem(li.SRC_DENSE, 20, 12, W=np.zeros((20, 12)))
    I = np.arange(4, dtype=np.int32); J = np.array([3, 1, 7, 0], dtype=np.int32)
    pv = oracle.prjvol(p, I, J, 3)
    assert pv["srank"] == 0 and pv["l"] == 4 and pv["status"] == 16
    np.testing.assert_array_equal(pv["J"], J)
    p, o = _prj_case(2, r=5, k=8, m=40, n=11)
    r, J0, _ = oracle.alg1tor(p.W[o["I"], :], tol=1e-10)
    pv = oracle.prjvol(p, o["I"], o["J"], 0, h=1e300, max_swaps=0, rank_tol=1e-10)
    assert pv["srank"] == r == 5 and pv["swaps"] == 0
    np.testing.assert_array_equal(pv["J"][:r], J0)
    pv = oracle.prjvol(p, o["I"], o["J"], 20, rank_tol=1e-10)
    assert pv["l"] == 11 and sorted(pv["J"].tolist()) == list(range(11))
