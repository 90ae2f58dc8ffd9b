"""C-A with DMM08 Algorithm 1 on the sketches (SVD-based leverage scores by
round-robin Jacobi, Exactly/Expected sampling) through the C ABI, against the
FP64 oracle block by block: sampled index lists, gathered C and R bit-exact, U
within 1e-10, ranks and statuses equal."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import to_device  # noqa: E402


def sub_problem(p, blk):
    r0, nr, c0, nc = (int(v) for v in blk)
    if p.src == li.SRC_DENSE:
        return li.Problem(li.SRC_DENSE, nr, nc, W=np.ascontiguousarray(p.W[r0:r0 + nr, c0:c0 + nc]))
    return li.Problem(p.src, nr, nc, X=p.X[r0:r0 + nr], Y=p.Y[c0:c0 + nc], ell=p.ell, entries=p.entries)


def run(p, blocks, k, r, iters, kind, seed=0):
    import paper_1710_07946_gb300 as lra
    blocks = np.asarray(blocks, dtype=np.int64)
    nb = len(blocks)
    max_len = int(max(blocks[:, 1].max(), blocks[:, 3].max()))
    draws = np.random.default_rng(seed).random((nb, 2 * iters, max_len))
    I0 = li.block_initial_rows(blocks, k, seed + 1)
    prob, _ = to_device(p)
    lb = lra.LevBatch(prob, blocks, k, r, iters, kind, I0, draws)
    lra.lra_ca_lev_batched(lb)
    torch.cuda.synchronize()
    for b in range(nb):
        sub = sub_problem(p, blocks[b])
        L = max(sub.m, sub.n)
        o = oracle.ca_lev(sub, k, r, iters, kind, draws[b][:, :L], I0[b], rank_tol=1e-6)
        g = lb.block(b)
        assert (g["status"], g["rank"], g["kI"], g["kJ"]) == (o["status"], o["rank"], o["kI"], o["kJ"]), b
        np.testing.assert_array_equal(g["I"], o["I"])
        np.testing.assert_array_equal(g["J"], o["J"])
        np.testing.assert_array_equal(g["C"], o["C"])
        np.testing.assert_array_equal(g["R"], o["R"])
        if o["rank"] > 0:
            assert np.abs(g["U"] - o["U"]).max() <= 1e-10 * np.abs(o["U"]).max(), b
    return lb


@pytest.mark.parametrize("kind", [0, 1])
def test_dense_blocks(kind):
    p = li.dense_lowrank(900, 800, r=24, noise=1e-8, seed=3)
    blocks = [[0, 900, 0, 800], [100, 300, 50, 700], [17, 64, 3, 65], [500, 400, 400, 400]]
    run(p, blocks, 12, 6, 8, kind, seed=kind)


@pytest.mark.parametrize("k,r", [(4, 4), (24, 6), (64, 16)])
def test_sizes_exactly(k, r):
    p = li.dense_lowrank(700, 650, r=20, noise=1e-9, seed=k)
    run(p, [[0, 700, 0, 650], [50, 300, 100, 500]], k, r, 4, 0, seed=k)


def test_hmt11_laplacian_and_exact_low_rank():
    run(li.hmt11_laplacian(512), [[0, 512, 0, 512], [0, 256, 256, 256]], 40, 10, 8, 0, seed=7)
    run(li.hmt11_laplacian(512), [[0, 512, 0, 512]], 40, 10, 8, 1, seed=8)
    q = li.factor_gaussian(400, 8, 0.0, seed=2)
    lb = run(q, [[0, 400, 0, 400]], 16, 8, 8, 0, seed=9)
    g = lb.block(0)
    assert np.linalg.norm(q.W - g["C"] @ g["U"] @ g["R"]) <= 1e-10 * np.linalg.norm(q.W)


def test_laplace_kernel_blocks():
    p, blocks, lev = li.fmm_blocks(npts=1 << 14, leaf=64, min_size=64, max_size=2048, nblocks=24, seed=4)
    run(p, blocks, 16, 8, 4, 0, seed=11)


def test_benchmark_configuration_sampled_runs():
    """The benchmark's configuration (1000 x 1000 of numerical rank 10, k = 40,
    r = 10, eight iterations, Exactly) on 8 runs, all compared."""
    p = li.dense_lowrank(1000, 1000, r=10, noise=1e-9, seed=0)
    run(p, [[0, 1000, 0, 1000]] * 8, 40, 10, 8, 0, seed=77)


@pytest.mark.parametrize("kind", [2, 3])
def test_uniform_scores(kind):
    """Uniform scores (no SVD stage) on perturbed factor-Gaussian inputs and on
    blocks of a graded low-rank one; the benchmark's uniform configuration."""
    p = li.factor_gaussian(600, 10, 1e-9, seed=kind)
    run(p, [[0, 600, 0, 600], [100, 300, 50, 500], [17, 64, 3, 65]], 40, 10, 4, kind, seed=kind)
    q = li.dense_lowrank(700, 650, r=20, noise=1e-9, seed=3)
    run(q, [[0, 700, 0, 650], [50, 300, 100, 500]], 24, 6, 3, kind, seed=5)
    f = li.factor_gaussian(1000, 10, 1e-9, seed=0)
    lb = run(f, [[0, 1000, 0, 1000]] * 4, 40, 10, 8, kind, seed=77)
    g = lb.block(0)
    assert np.linalg.norm(f.W - g["C"] @ g["U"] @ g["R"]) <= 1e-7 * np.linalg.norm(f.W)
