"""GPU parity of the CUDA C-A path with the FP64 oracle (through the C ABI).

Bar: row and column index sets bit-exact (lowest-index tie-break); gathered
factors C = W'[:,J] and R = W[I,:] identical; the nucleus U within 1e-10
relative (max-norm); swap / loop counters and statuses equal.
"""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import assert_parity, gpu_ca  # noqa: E402


def run_both(p, k, sweeps, I0, **kw):
    o = oracle.ca_run(p, k, sweeps, I0, **kw)
    g = gpu_ca(p, k, sweeps, I0, **kw)
    return o, g


# ---------------------------------------------------------------- the 256 x 256 workload
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("noise", [1e-8, 0.0])
def test_dense_256_rank8(seed, noise):
    """256 x 256 FP64, U diag(2^-i) V^T (+1e-8 noise), k = 8, 3 sweeps."""
    p = li.dense_lowrank(256, 256, r=8, noise=noise, seed=seed)
    I0 = li.initial_rows(256, 8, 1000 + seed)
    o, g = run_both(p, 8, 3, I0)
    assert_parity(o, g)
    err = np.linalg.norm(p.W - g["C"] @ g["U"] @ g["R"]) / np.linalg.norm(p.W)
    assert err < (1e-12 if noise == 0 else 1e-5)


# ---------------------------------------------------------------- multi-CTA, ragged chunks
@pytest.mark.parametrize("m,n,k", [(2000, 1500, 16), (1001, 77, 7), (77, 3001, 12), (4099, 4097, 40)])
def test_dense_multi_cta_ragged(m, n, k):
    p = li.factor_gaussian(max(m, n), k + 2, 1e-3, seed=m + n)
    p.W = np.ascontiguousarray(p.W[:m, :n])
    p.m, p.n = m, n
    I0 = li.initial_rows(m, k, 7)
    o, g = run_both(p, k, 3, I0)
    assert_parity(o, g)


@pytest.mark.parametrize("ctas", [1, 2, 5, 19, 64, 152])
def test_grid_size_does_not_change_results(ctas):
    """The pivots, factors and counters are the oracle's whatever the number of
    CTAs sharing the run (lra_ca_params.ctas): one CTA (the whole strip, in
    global scratch), uneven chunks (5, 19) and the full grid; ARHT multiplier."""
    p = li.factor_gaussian(3000, 22, 1e-4, seed=41)
    p.W = np.ascontiguousarray(p.W[:2500, :])
    p.m = 2500
    li.with_arht(p, 2, seed=42)
    I0 = li.initial_rows(2500, 20, 43)
    o = oracle.ca_run(p, 20, 3, I0)
    g = gpu_ca(p, 20, 3, I0, ctas=ctas)
    assert_parity(o, g)


@pytest.mark.parametrize("mult,arg", [("arht", 2), ("arht", 3), ("sparse", 4), ("bidiag", 3)])
@pytest.mark.parametrize("m,n", [(3000, 700), (1024, 96)])
def test_left_multipliers_tall_inputs(mult, arg, m, n):
    """m > n: the multiplier pre-multiplies (Remark re2orddmn), W' = M^T W with M
    m x m; C = W[:, J], R = W'[I, :].  Multi-CTA grid (3000 x 700) and one CTA
    (1024 x 96), FP32 spiky and FP64 factor-Gaussian inputs."""
    if m == 3000:
        p = li.factor_gaussian(m, 20, 1e-4, seed=m + arg)
        p.W = np.ascontiguousarray(p.W[:, :n])
        p.n = n
    else:
        p = li.dense_spiky(m, r=12, seed=8)
        p.W = np.ascontiguousarray(p.W[:, :n])
        p.n = n
    if mult == "arht":
        li.with_arht(p, arg, 31, side="left")
    elif mult == "bidiag":
        li.with_bidiag(p, arg, 31, side="left")
    else:
        li.with_sparse(p, arg, 31, side="left")
    I0 = li.initial_rows(m, 16, 5)
    o, g = run_both(p, 16, 4, I0)
    assert_parity(o, g)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fourier_multiplier_real_form(d):
    """The real-form ARFT (W' = W [Re M, Im M], 2n columns, real weights of
    cos / sin of the roots of unity times D): J indexes the 2n columns; FP32
    spiky input on one CTA."""
    p = li.dense_spiky(1024, r=16, seed=13)
    li.with_arft(p, d, 23)
    I0 = li.initial_rows(1024, 24, 6)
    o, g = run_both(p, 24, 4, I0)
    assert_parity(o, g)
    assert g["J"].max() < 2048


def test_fourier_multiplier_multi_cta_and_laplace():
    """ARFT on the cooperative grid (3000 x 2600 FP64 factor-Gaussian, depth 3)
    and on Laplace entries evaluated on the fly (depth 2)."""
    p = li.factor_gaussian(3000, 20, 1e-4, seed=77)
    p.W = np.ascontiguousarray(p.W[:, :2600])
    p.n = 2600
    li.with_arft(p, 3, 5)
    I0 = li.initial_rows(3000, 20, 8)
    o, g = run_both(p, 20, 3, I0)
    assert_parity(o, g)
    q = li.laplace_clusters(2000, 1200, seed=5)
    li.with_arft(q, 2, 6)
    I0 = li.initial_rows(2000, 16, 4)
    o, g = run_both(q, 16, 3, I0)
    assert_parity(o, g)


def test_left_multiplier_laplace_entries():
    """A tall Laplace block (targets 4000, sources 600) with a left ARHT: the
    pre-processed rows combine kernel entries evaluated on the fly."""
    p = li.laplace_clusters(4000, 600, seed=3)
    li.with_arht(p, 3, 12, side="left")
    I0 = li.initial_rows(4000, 24, 2)
    o, g = run_both(p, 24, 3, I0)
    assert_parity(o, g)


@pytest.mark.parametrize("mult,arg", [("arht", 1), ("arht", 2), ("arht", 3), ("sparse", 4), ("bidiag", 1), ("bidiag", 3), ("bidiag", 5)])
def test_float32_with_multipliers(mult, arg):
    p = li.dense_spiky(1024, r=16, seed=3)
    if mult == "arht":
        li.with_arht(p, arg, 11)
    elif mult == "bidiag":
        li.with_bidiag(p, arg, 11)
    else:
        li.with_sparse(p, arg, 11)
    I0 = li.initial_rows(1024, 24, 5)
    o, g = run_both(p, 24, 4, I0)
    assert_parity(o, g)


@pytest.mark.parametrize("n,k,q", [(256, 31, 20), (1024, 39, 20), (512, 35, 12)])
def test_hmt11_laplacian_bidiagonal(n, k, q):
    """The single-layer Laplacian input with q bidiagonal factors (every column of
    the product dense at q = 20), five C-A loops as in Tests 2."""
    p = li.hmt11_laplacian(n)
    li.with_bidiag(p, q, 100 + k)
    I0 = li.initial_rows(n, k, k)
    o, g = run_both(p, k, 5, I0)
    assert_parity(o, g)


def test_hmt11_laplacian_arht():
    """The same input under the abridged Hadamard multiplier, k = 15 (the ARHT/ARFT
    table's rank)."""
    p = li.hmt11_laplacian(512)
    li.with_arht(p, 3, 21)
    I0 = li.initial_rows(512, 15, 4)
    o, g = run_both(p, 15, 5, I0)
    assert_parity(o, g)


@pytest.mark.parametrize("k", [8, 32])
def test_laplace_kernel_entries(k):
    p = li.laplace_clusters(3000, 2500, seed=2)
    I0 = li.initial_rows(3000, k, 9)
    o, g = run_both(p, k, 3, I0)
    assert_parity(o, g)


def test_gaussian_kernel_close_to_oracle():
    """exp() is not bit-identical across libraries: compare approximation quality."""
    p = li.gaussian_clusters(900, 800, ell=0.3, seed=4)
    I0 = li.initial_rows(900, 12, 3)
    o, g = run_both(p, 12, 3, I0)
    X, Y = p.X, p.Y
    K = np.exp(-np.sum((X[:, None, :] - Y[None, :, :]) ** 2, axis=2) / (2 * 0.3 ** 2))
    eo = np.linalg.norm(K - o["C"] @ o["U"] @ o["R"]) / np.linalg.norm(K)
    eg = np.linalg.norm(K - g["C"] @ g["U"] @ g["R"]) / np.linalg.norm(K)
    assert g["status"] == o["status"] and eg <= 2 * eo + 1e-14


# ---------------------------------------------------------------- edge cases
def test_k_equals_one():
    p = li.factor_gaussian(300, 3, 1e-2, seed=1)
    o, g = run_both(p, 1, 3, li.initial_rows(300, 1, 0))
    assert_parity(o, g)


def test_k_equals_min_dimension():
    p = li.factor_gaussian(40, 5, 1e-2, seed=1)
    p.W = np.ascontiguousarray(p.W[:, :12]); p.n = 12
    o, g = run_both(p, 12, 2, li.initial_rows(40, 12, 0))
    assert_parity(o, g)


def test_rank_deficient_strip_status():
    p = li.factor_gaussian(200, 5, 0.0, seed=2)
    p.W[:, 3] = 0.0
    W = p.W.copy(); W[:, :] = 0.0; W[:, :3] = p.W[:, :3]      # exact rank <= 3
    p.W = W
    o, g = run_both(p, 6, 2, li.initial_rows(200, 6, 1))
    assert o["status"] == 16 and g["status"] == 16
    np.testing.assert_array_equal(g["I"], o["I"])
    np.testing.assert_array_equal(g["J"], o["J"])


def test_nonfinite_input_status():
    p = li.dense_lowrank(128, 128, r=4, seed=0)
    I0 = li.initial_rows(128, 4, 1)
    p.W[I0[2], 17] = np.nan
    o, g = run_both(p, 4, 2, I0)
    assert o["status"] == 3 and g["status"] == 3


def test_max_swaps_zero_not_converged():
    p = li.factor_gaussian(500, 10, 1e-2, seed=8)
    o, g = run_both(p, 10, 2, li.initial_rows(500, 10, 3), max_swaps=0)
    assert_parity(o, g)
    assert g["status"] == 17


def test_invalid_initial_rows_reported():
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(64, 64, r=4, seed=0)
    g = gpu_ca(p, 4, 2, np.array([1, 2, 2, 3], np.int32))
    assert g["status"] == lra.LRA_ERR_INVALID_ARG


def test_host_side_rejections():
    import paper_1710_07946_gb300 as lra
    from gpu_helpers import to_device
    p = li.dense_lowrank(64, 64, r=4, seed=0)
    prob, _ = to_device(p)
    I0 = torch.arange(8, dtype=torch.int32, device="cuda")
    with pytest.raises(lra.LraError):
        lra.lra_ca_run(prob, I0, 65)          # k > 64
    with pytest.raises(lra.LraError):
        lra.lra_ca_run(prob, I0, 8, h=0.5)     # h < 1
    with pytest.raises(lra.LraError):
        lra.lra_ca_run(prob, I0, 8, workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))
    with pytest.raises(lra.LraError):
        lra.lra_ca_run(prob, I0, 8, ctas=-1)


def test_repeatable_and_stream_ordered():
    p = li.dense_lowrank(512, 384, r=8, noise=1e-6, seed=5)
    I0 = li.initial_rows(512, 8, 2)
    a = gpu_ca(p, 8, 3, I0)
    b = gpu_ca(p, 8, 3, I0)
    for key in ("I", "J", "C", "U", "R"):
        np.testing.assert_array_equal(a[key], b[key])


# ---------------------------------------------------------------- apply / residual
def test_resume_from_output_sets():
    """lra_ca_run_warm resumed from a finished run's (I, J) equals the oracle's warm
    run and never loses volume; an invalid J0 is reported in the status word."""
    import paper_1710_07946_gb300 as lra
    p = li.factor_gaussian(600, 14, 1e-4, seed=6)
    I0 = li.initial_rows(600, 12, 2)
    a = gpu_ca(p, 12, 1, I0)
    o = oracle.ca_run(p, 12, 3, a["I"], J0=a["J"])
    g = gpu_ca(p, 12, 3, a["I"], J0=torch.from_numpy(a["J"]).cuda())
    assert_parity(o, g)
    va = np.linalg.slogdet(p.W[np.ix_(a["I"], a["J"])])[1]
    vg = np.linalg.slogdet(p.W[np.ix_(g["I"], g["J"])])[1]
    assert vg >= va - 1e-9
    bad = a["J"].copy()
    bad[1] = bad[0]
    gb = gpu_ca(p, 12, 3, a["I"], J0=torch.from_numpy(bad).cuda())
    assert gb["status"] == lra.LRA_ERR_INVALID_ARG


def test_cur_apply_matches_oracle():
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(700, 900, r=6, noise=1e-6, seed=1)
    o = oracle.ca_run(p, 6, 2, li.initial_rows(700, 6, 0))
    X = li.rhs(900, 5, 3)
    Yo = oracle.cur_apply(o["C"], o["U"], o["R"], X)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Yg = lra.lra_cur_apply(t(o["C"]), t(o["U"]), t(o["R"]), t(X)).cpu().numpy()
    assert np.abs(Yg - Yo).max() <= 1e-12 * np.abs(Yo).max()


U32 = 2.0 ** -24


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,k,nrhs", [(700, 900, 6, 5), (3001, 2049, 40, 1), (1024, 4100, 64, 64),
                                        (257, 255, 17, 16), (64, 1, 1, 3)])
def test_cur_apply_stored_low_precision(dtype, m, n, k, nrhs):
    """Stored factors in FP32 / BF16 with FP32 products and one refinement step
    (the FP64 vector split into FP32 head and tail), element by element against
    the oracle's FP64 product of the same rounded factors.  Bound: R X sums runs
    of at most 512 terms as 16 products per lane and a 5-level butterfly (at most
    22 roundings on any term's path), C T2 sums k terms: |dY| <= |C| |U| (22 u
    |R| |X|) + (k + 1) u |C| |T2|, u = 2^-24 (the split leaves O(u^2)); asserted
    with a factor 2 of slack.  Shapes: ragged tiles, rows of R not 16-byte
    aligned (n = 255, 2049), k = 1 and 64, 1 to 64 right-hand sides."""
    import paper_1710_07946_gb300 as lra
    g = np.random.default_rng(m + n + k + nrhs)
    C = g.standard_normal((m, k))
    R = g.standard_normal((k, n))
    U = g.standard_normal((k, k)) / np.sqrt(k)
    X = g.standard_normal((n, nrhs))
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    Cl = torch.from_numpy(C).to(tdt).cuda()
    Rl = torch.from_numpy(R).to(tdt).cuda()
    Ct, Rt = Cl.double().cpu().numpy(), Rl.double().cpu().numpy()      # the stored values, exactly
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Yg = lra.lra_cur_apply(Cl, t(U), Rl, t(X)).cpu().numpy()
    Yo = oracle.cur_apply(Ct, U, Rt, X)
    T2 = U @ (Rt @ X)
    bound = np.abs(Ct) @ (np.abs(U) @ (22 * U32 * (np.abs(Rt) @ np.abs(X)))) + (k + 1) * U32 * (np.abs(Ct) @ np.abs(T2))
    err = np.abs(Yg - Yo)
    assert np.all(err <= 2 * bound + 1e-300), (err / np.maximum(bound, 1e-300)).max()
    # against the FP64 factors the storage rounding dominates (u or 2^-9 per entry)
    rel = np.linalg.norm(Yg - oracle.cur_apply(C, U, R, X)) / np.linalg.norm(Yo)
    assert rel < (1e-5 if dtype == "f32" else 3e-2), rel


def test_cur_apply_rejects_mixed_or_unsupported_dtypes():
    import paper_1710_07946_gb300 as lra
    C = torch.zeros(8, 4, dtype=torch.float32, device="cuda")
    R = torch.zeros(4, 8, dtype=torch.float64, device="cuda")
    U = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    X = torch.zeros(8, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        lra.lra_cur_apply(C, U, R, X)
    with pytest.raises(lra.LraError):
        lra.lra_cur_apply(C, U, R.float(), torch.zeros(8, 65, dtype=torch.float64, device="cuda"))   # nrhs > 64


def test_residual_sample_matches_oracle():
    import paper_1710_07946_gb300 as lra
    from gpu_helpers import to_device
    p = li.dense_lowrank(300, 280, r=5, noise=1e-5, seed=2)
    o = oracle.ca_run(p, 5, 2, li.initial_rows(300, 5, 0))
    Q, S = li.sample_positions(300, 280, 40, 30, 6)
    st_o = oracle.residual_sample(p, o["C"], o["U"], o["R"], Q, S)
    prob, _ = to_device(p)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    st_g = lra.lra_residual_sample(prob, t(o["C"]), t(o["U"]), t(o["R"]), t(Q), t(S)).cpu().numpy()
    np.testing.assert_allclose(st_g[1:], st_o[1:], rtol=1e-9)
    assert abs(st_g[0] - st_o[0]) <= 1e-9 * st_o[2]


# ---------------------------------------------------------------- full-size benchmark workload
@pytest.mark.parametrize("mult", ["arht", "sparse", "bidiag"])
def test_dense8192_benchmark_workload(mult):
    """8192 x 8192 FP32 rank-32 + 1% spikes, ARHT d=2, sparse +-1 or a product of 3
    bidiagonal factors, k = 48, 4 loops: the benchmark's configuration, compared in full."""
    p = li.dense_spiky(8192, r=32, seed=0)
    if mult == "arht":
        li.with_arht(p, 2, 7)
    elif mult == "bidiag":
        li.with_bidiag(p, 3, 7)
    else:
        li.with_sparse(p, 4, 7)
    I0 = li.initial_rows(8192, 48, 11)
    o, g = run_both(p, 48, 4, I0)
    assert_parity(o, g)
