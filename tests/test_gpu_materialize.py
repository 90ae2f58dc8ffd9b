"""The pre-processed input written out (lra_multiplier_apply) and the CUR's
rows gathered from the original input (lra_gather_rows), against the FP64
oracle: W' bit-exact for every multiplier kind; C-A on the written-out W'
(single runs and a batched launch over stacked copies, as the HMT11 benchmark
runs it) selects the oracle's pivots of C-A on (W, M), and with R = W[I, :] the
factors match; the grid-wide residual statistics over 10^6 samples."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import assert_parity, to_device  # noqa: E402


def _with(p, kind):
    if kind == "bidiag20":
        li.with_bidiag(p, 20, 5)
    elif kind == "bidiag3":
        li.with_bidiag(p, 3, 6)
    elif kind == "arht":
        li.with_arht(p, 2, 7)
    elif kind == "sparse":
        li.with_sparse(p, 4, 8)
    elif kind == "arft":
        li.with_arft(p, 3, 9)
    elif kind == "arht_left":
        li.with_arht(p, 2, 10, side="left")
    return p


@pytest.mark.parametrize("kind", ["none", "bidiag20", "bidiag3", "arht", "sparse", "arft", "arht_left"])
def test_apply_is_bit_exact(kind):
    import paper_1710_07946_gb300 as lra
    p = _with(li.dense_spiky(512, r=12, seed=2), kind)
    prob, mult = to_device(p)
    Wp = lra.lra_multiplier_apply(prob, mult).cpu().numpy()
    ref = oracle.gather_rows(p, np.arange(p.m, dtype=np.int32))
    np.testing.assert_array_equal(Wp, ref)


@pytest.mark.parametrize("m,n", [(300, 200), (33, 65), (1, 1000)])
def test_dense_product_ragged_tiles(m, n):
    """Products whose columns can all be full (2^q >= n) take the register-tiled
    kernel: ragged row and column tiles, FP64 input."""
    import paper_1710_07946_gb300 as lra
    g = np.random.default_rng(m + n)
    p = li.Problem(li.SRC_DENSE, m, n, W=g.standard_normal((m, n)))
    li.with_bidiag(p, 20, 17)
    prob, mult = to_device(p)
    Wp = lra.lra_multiplier_apply(prob, mult).cpu().numpy()
    np.testing.assert_array_equal(Wp, oracle.gather_rows(p, np.arange(m, dtype=np.int32)))


def test_apply_on_laplace_entries_and_strided_output():
    import paper_1710_07946_gb300 as lra
    p = li.laplace_clusters(300, 256, seed=3)
    li.with_bidiag(p, 6, 9)
    prob, mult = to_device(p)
    big = torch.full((300, 300), 7.0, dtype=torch.float64, device="cuda")
    view = big[:, :256]
    with pytest.raises(ValueError):
        lra.lra_multiplier_apply(prob, mult, out=view)          # non-contiguous rows are refused by the binding
    Wp = lra.lra_multiplier_apply(prob, mult).cpu().numpy()
    np.testing.assert_array_equal(Wp, oracle.gather_rows(p, np.arange(300, dtype=np.int32)))


def _run_on_materialized(p, k, sweeps, I0):
    import paper_1710_07946_gb300 as lra
    prob, mult = to_device(p)
    Wp = lra.lra_multiplier_apply(prob, mult)
    I0d = torch.from_numpy(np.ascontiguousarray(I0, dtype=np.int32)).cuda()
    out = lra.lra_ca_run(lra.Problem.dense(Wp), I0d, k, sweeps)
    R = lra.lra_gather_rows(prob, out["I"])
    torch.cuda.synchronize()
    res = {key: v.cpu().numpy() for key, v in out.items() if not key.startswith("_")}
    info = res.pop("info")
    res.update(rank=int(info[0]), swaps=int(info[1]), loops=int(info[2]), status=int(info[3]))
    res["R"] = R.cpu().numpy()
    return res


@pytest.mark.parametrize("n,k", [(256, 31), (512, 39)])
def test_ca_on_materialized_matches_ca_with_multiplier(n, k):
    p = li.hmt11_laplacian(n)
    li.with_bidiag(p, 20, 40 + k)
    I0 = li.initial_rows(n, k, k)
    o = oracle.ca_run(p, k, 5, I0)
    g = _run_on_materialized(p, k, 5, I0)
    assert_parity(o, g)


def test_batched_runs_on_stacked_materialized_inputs():
    """Four runs with their own multipliers and initial rows as blocks of one
    batched launch over the stacked W'_r (the HMT11 benchmark's step)."""
    import paper_1710_07946_gb300 as lra
    n, k, runs = 256, 31, 4
    base = li.hmt11_laplacian(n)
    W = torch.from_numpy(base.W).cuda()
    prob = lra.Problem.dense(W)
    Wp = torch.empty(runs * n, n, dtype=torch.float64, device="cuda")
    ps, I0s = [], []
    for r in range(runs):
        pr = li.Problem(li.SRC_DENSE, n, n, W=base.W)
        li.with_bidiag(pr, 20, 200 + r)
        _, mult = to_device(pr)
        lra.lra_multiplier_apply(prob, mult, Wp[r * n:(r + 1) * n])
        ps.append(pr)
        I0s.append(li.initial_rows(n, k, 300 + r))
    blocks = np.array([[r * n, n, 0, n] for r in range(runs)], dtype=np.int64)
    bt = lra.Batch(lra.Problem.dense(Wp), blocks, k, 5, np.stack(I0s), rank_tol=1e-13, order=None)
    lra.lra_ca_run_batched(bt)
    torch.cuda.synchronize()
    for r in range(runs):
        g = bt.block(r)
        R = lra.lra_gather_rows(prob, bt.out["I"][r]).cpu().numpy()
        o = oracle.ca_run(ps[r], k, 5, I0s[r], rank_tol=1e-13)
        assert (g["status"], g["rank"], g["swaps"], g["loops"]) == (o["status"], o["rank"], o["swaps"], o["loops"])
        np.testing.assert_array_equal(g["I"], o["I"])
        np.testing.assert_array_equal(g["J"], o["J"])
        np.testing.assert_array_equal(g["C"], o["C"])
        np.testing.assert_array_equal(R, o["R"])
        assert np.abs(g["U"] - o["U"]).max() <= 1e-10 * np.abs(o["U"]).max()


def test_gather_rows_flags_rows_out_of_range():
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(40, 30, r=3, seed=1)
    prob, _ = to_device(p)
    I = torch.tensor([3, -1, 39, 40], dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    R = lra.lra_gather_rows(prob, I, status=st).cpu().numpy()
    assert int(st.item()) == lra.LRA_ERR_INVALID_ARG
    np.testing.assert_array_equal(R[0], p.W[3])
    np.testing.assert_array_equal(R[2], p.W[39])
    assert np.isnan(R[1]).all() and np.isnan(R[3]).all()
    st.zero_()
    lra.lra_gather_rows(prob, torch.tensor([0, 5], dtype=torch.int32, device="cuda"), status=st)
    assert int(st.item()) == 0


def test_residual_statistics_over_a_million_entries():
    """The exact Frobenius ratio of the HMT11 benchmark: every entry of a
    1024 x 1024 input sampled (grid-wide partial sums)."""
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(1024, 1024, r=20, noise=1e-7, seed=4)
    o = oracle.ca_run(p, 16, 3, li.initial_rows(1024, 16, 2))
    QS = np.arange(1024, dtype=np.int32)
    st_o = oracle.residual_sample(p, o["C"], o["U"], o["R"], QS, QS)
    prob, _ = to_device(p)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    st_g = lra.lra_residual_sample(prob, t(o["C"]), t(o["U"]), t(o["R"]), t(QS), t(QS)).cpu().numpy()
    np.testing.assert_allclose(st_g[1:], st_o[1:], rtol=1e-9)
    assert abs(st_g[0] - st_o[0]) <= 1e-9 * st_o[2]
    E = p.W - o["C"] @ o["U"] @ o["R"]
    assert abs(st_g[4] - np.linalg.norm(E) / np.linalg.norm(p.W)) <= 1e-9 * st_g[4]


def test_bidiag20_products_written_out_are_nearly_gaussian():
    """Figure LowRkTest1's experiment on the device path: W' = I M for products
    M of 20 permuted cyclic bidiagonal factors (n = 1024), written out by
    lra_multiplier_apply with M's scale 2^{-10}.  The first product equals the
    oracle's integer product bit for bit.  One fixed entry over 60 independent
    products, times 32 (1 / its standard deviation 2^{-10} sqrt(2^20 / 1024)),
    passes the Kolmogorov-Smirnov test for N(0, 1), and two entries are
    uncorrelated."""
    import paper_1710_07946_gb300 as lra
    st = pytest.importorskip("scipy.stats")
    n, q, reps = 1024, 20, 60
    prob = lra.Problem.dense(torch.eye(n, dtype=torch.float64, device="cuda"))
    a, b = [], []
    for rep in range(reps):
        perms, signs = li.bidiag_descriptor(n, q, 7000 + rep)
        mult = lra.lra_precondition("bidiag", n, q, perms, signs)
        Mp = lra.lra_multiplier_apply(prob, mult)
        if rep == 0:
            rows, vals = oracle.bidiag_columns(n, q, perms, signs)
            M = np.zeros((n, n))
            cols = np.broadcast_to(np.arange(n)[:, None], rows.shape)
            msk = vals != 0
            M[rows[msk], cols[msk]] = vals[msk]
            np.testing.assert_array_equal(Mp.cpu().numpy(), M * 2.0 ** -10)
        a.append(Mp[17, 400].item() * 32.0)
        b.append(Mp[900, 33].item() * 32.0)
    assert st.kstest(np.array(a), "norm").pvalue > 0.01
    assert st.kstest(np.array(b), "norm").pvalue > 0.01
    assert abs(np.corrcoef(a, b)[0, 1]) < 4.0 / np.sqrt(reps)
