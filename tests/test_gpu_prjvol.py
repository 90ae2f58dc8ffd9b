"""Generators of maximal r-projective volume (Algorithm algprjvlm, with
Algorithm alg1tor's pivoted QR to the numerical rank, dominance swaps on R' and
greedy expansion) for every block of a batched C-A run, against the FP64
oracle block by block: the strip rank, swap count, column set and gathered
factors bit-exact, U within 1e-10."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import to_device  # noqa: E402
from test_gpu_oversample import sub_problem  # noqa: E402


def run(p, blocks, k, pextra, rank_tol, stages=None, seed=0, h=1.01, max_swaps=None, check=None, margin=0):
    import paper_1710_07946_gb300 as lra
    prob, _ = to_device(p)
    I0 = li.block_initial_rows(blocks, k, seed)
    bt = lra.Batch(prob, blocks, k, 3, I0, h=h, rank_tol=rank_tol, stages=stages, rank_margin=margin)
    lra.lra_ca_run_batched(bt)
    pv = lra.lra_prjvol_batched(bt, pextra, max_swaps=max_swaps)
    torch.cuda.synchronize()
    out = []
    for b in (range(len(blocks)) if check is None else check):
        g0 = bt.block(b)
        o = oracle.prjvol(sub_problem(p, blocks[b]), g0["I"], g0["J"], pextra, h=h,
                          max_swaps=1000 if max_swaps is None else max_swaps, rank_tol=rank_tol)
        g = pv.block(b)
        assert (g["status"], g["rank"], g["l"], g["k"]) == (o["status"], o["rank"], o["l"], len(g0["I"])), b
        assert (g["srank"], g["swaps"]) == (o["srank"], o["swaps"]), b
        np.testing.assert_array_equal(g["J"], o["J"])
        np.testing.assert_array_equal(g["C"], o["C"])
        np.testing.assert_array_equal(g["R"], o["R"])
        if o["rank"] > 0:
            assert np.abs(g["U"] - o["U"]).max() <= 1e-10 * np.abs(o["U"]).max()
        out.append((g, o))
    return bt, pv, out


def test_fmm_blocks_staged_then_prjvol():
    """Laplace FMM blocks of 64..2048 points (strips in shared memory and in the
    global scratch), staged sizes 28/40/64, rank_tol 1e-6."""
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=64, seed=8)
    _, _, out = run(p, blocks, 64, 8, 1e-6, stages=(28, 40, 64), h=1.05, margin=2)
    assert any(g["srank"] < g["k"] for g, _ in out)


def test_fmm_blocks_fp32_entries():
    p, blocks, lev = li.fmm_blocks(npts=1 << 14, leaf=64, min_size=64, max_size=1024, nblocks=32, seed=3)
    q = li.Problem(p.src, p.m, p.n, X=p.X, Y=p.Y, entries="f32")
    run(q, blocks, 32, 4, 1e-6, stages=(16, 24, 32), h=1.05)


def test_dense_rank_deficient_strips_recover_the_input():
    """Exact rank-10 blocks with k = 16: the strips have rank 10, the generators
    reproduce every block to rounding; narrow blocks clip l."""
    p = li.factor_gaussian(900, 10, 0.0, seed=2)
    blocks = li.dense_blocks(900, sizes=(16, 20, 64, 300), seed=3)
    _, pv, out = run(p, blocks, 16, 6, 1e-10)
    for (g, o), blk in zip(out, blocks):
        assert g["srank"] == min(10, g["k"])
        r0, nr, c0, nc = (int(v) for v in blk)
        W = p.W[r0:r0 + nr, c0:c0 + nc]
        assert np.linalg.norm(W - g["C"] @ g["U"] @ g["R"]) <= 1e-11 * np.linalg.norm(W)


def test_swap_limits_zero_strips_and_full_rank_strips():
    """max_swaps = 0 leaves Algorithm alg1tor's pivots (status says whether a swap
    was wanted); a zero block gives r = 0 and keeps the square generator; a
    full-rank noisy input gives r = k."""
    p = li.dense_lowrank(600, 700, r=30, noise=1e-7, seed=5)
    blocks = np.array([[0, 600, 0, 700], [10, 300, 40, 20], [100, 200, 300, 400], [0, 64, 0, 70]], dtype=np.int64)
    run(p, blocks, 12, 6, 1e-13, max_swaps=0)
    _, _, out = run(p, blocks, 12, 6, 1e-13)
    assert all(g["srank"] == g["k"] for g, _ in out)
    W = np.random.default_rng(1).standard_normal((300, 300))
    W[:, 100:200] = 0.0
    W[100:200, :] = 0.0
    q = li.Problem(li.SRC_DENSE, 300, 300, W=W)
    run(q, np.array([[100, 100, 100, 100], [0, 300, 0, 300]], dtype=np.int64), 8, 3, 1e-13)


def test_fmm_benchmark_workload_sampled_blocks():
    """The 2^20-point, 4096-block FMM batch in the configuration the benchmark
    times (FP32 entries with FP64 pivots, staged 28/40/64, h = 1.05, p = 8):
    the smallest and largest blocks against the oracle."""
    p, blocks, lev = li.fmm_blocks(npts=1 << 20, seed=0)
    q = li.Problem(p.src, p.m, p.n, X=p.X, Y=p.Y, entries="f32")
    sizes = blocks[:, 1] * blocks[:, 3]
    pick = list(np.argsort(sizes)[:3]) + list(np.argsort(sizes)[-3:])
    run(q, blocks, 64, 8, 1e-6, stages=(28, 40, 64), h=1.05, check=pick, margin=2)


def test_dense_fp32_input_single_column_generators_and_no_extra_columns():
    """A dense FP32 input (entries widened exactly) of rank 6 plus noise: k = 12
    with no extra columns (l = k), and k = 1 grown by three columns."""
    g = np.random.default_rng(4)
    W = (g.standard_normal((500, 6)) @ g.standard_normal((6, 400)) + 1e-4 * g.standard_normal((500, 400)))
    p = li.Problem(li.SRC_DENSE, 500, 400, W=np.ascontiguousarray(W.astype(np.float32)))
    blocks = np.array([[0, 500, 0, 400], [10, 200, 30, 300], [100, 64, 100, 65], [7, 33, 5, 29]], dtype=np.int64)
    _, _, out = run(p, blocks, 12, 0, 1e-3)
    assert all(g_["l"] == g_["k"] for g_, _ in out)
    assert any(g_["srank"] < g_["k"] for g_, _ in out)
    run(p, blocks, 1, 3, 1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_random_configurations(seed):
    """Randomised sweep: input rank 2..24 with no, small or large noise; block
    sizes from 1 to 300 in every pairing; k 1..32; 0..8 extra columns; h and
    rank tolerances across their useful range."""
    g = np.random.default_rng(500 + seed)
    r = int(g.integers(2, 25))
    noise = (0.0, 1e-9, 1e-4)[seed % 3]
    p = li.factor_gaussian(700, r, noise, seed=seed)
    blocks = li.dense_blocks(700, sizes=(1, 9, 33, 64, 300), seed=seed)
    k = int(g.integers(1, 33))
    pextra = int(g.integers(0, 9))
    tol = (1e-13, 1e-8, 1e-4)[(seed // 3 + seed) % 3]
    h = (1.01, 1.05, 1.2)[seed % 3]
    run(p, blocks, k, pextra, tol, h=h, seed=seed)
