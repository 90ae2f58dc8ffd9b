"""y = M x for the Laplace matrix of uniform points held FMM-style (far blocks
with batched C-A generators, dense near field) through the C ABI: against the
oracle's matvec built from the oracle's own generators (pivots bit-exact, so
within rounding), and against the direct product."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def build(npts, leaf, seed, k=64, stages=(28, 40, 64)):
    import paper_1710_07946_gb300 as lra
    p, far, near, L = li.fmm_partition(npts, leaf=leaf, seed=seed)
    X = torch.from_numpy(p.X).cuda()
    prob = lra.Problem.kernel("laplace", X, X)
    I0 = li.block_initial_rows(far[:, :4], k, seed + 1)
    hm = lra.HMatrix(prob, far, near, L, I0, k=k, stages=stages)
    hm.build()
    return p, far, near, L, I0, hm


def direct_rows(P, x, rows):
    d = np.sqrt(((P[rows, None, :] - P[None, :, :]) ** 2).sum(axis=2))
    with np.errstate(divide="ignore"):
        K = np.where(d > 0.0, 1.0 / d, 0.0)
    return K @ x


def test_matvec_matches_oracle_and_direct():
    p, far, near, L, I0, hm = build(1 << 13, 128, 0)
    x = li.rhs(p.m, 1, 7)[:, 0]
    y = hm.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    info = hm.batch.out["info"].cpu().numpy()
    assert np.all((info[:, 3] == 0) | (info[:, 3] >= 16))
    gens = []
    for b, (r0, nr, c0, nc, lev, tb) in enumerate(far):
        sub = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=p.X[r0:r0 + nr], Y=p.X[c0:c0 + nc])
        o = oracle.ca_run_adaptive(sub, (28, 40, 64), 2, 3, I0[b], h=1.05, rank_tol=1e-6)
        assert int(info[b, 6]) == o["k"], b
        gens.append((o["C"], o["U"], o["R"]))
    y_o = oracle.hmatvec(p, far, near, gens, x)
    assert np.abs(y - y_o).max() <= 1e-10 * np.abs(y_o).max()
    rows = np.arange(0, p.m, 7)
    y_d = direct_rows(p.X, x, rows)
    assert np.linalg.norm(y[rows] - y_d) <= 2e-6 * np.linalg.norm(y_d)


def test_three_levels_against_direct_rows():
    p, far, near, L, I0, hm = build(1 << 15, 64, 3)
    assert L == 3
    x = li.rhs(p.m, 1, 9)[:, 0]
    y = hm.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    rows = np.random.default_rng(1).choice(p.m, 400, replace=False)
    y_d = direct_rows(p.X, x, rows)
    assert np.linalg.norm(y[rows] - y_d) <= 2e-6 * np.linalg.norm(y_d)
    # linear in x up to rounding (sums of 1/r terms up to ~1e3 in the near field)
    x2 = li.rhs(p.m, 1, 10)[:, 0]
    y2 = hm.matvec(torch.from_numpy(x2).cuda()).cpu().numpy()
    y3 = hm.matvec(torch.from_numpy(x + 2.0 * x2).cuda()).cpu().numpy()
    assert np.abs(y3 - (y + 2.0 * y2)).max() <= 1e-9 * np.abs(y3).max()
    # the same x twice: bit-identical (fixed summation order)
    y4 = hm.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(y4, y)


def test_benchmark_size_sampled_blocks_and_rows():
    """The benchmark's partition (2^16 points, 128-point leaves, 56,448 far
    blocks): 60 randomly chosen far blocks' generators against the oracle (pivots,
    sizes and gathered factors bit-exact), the matvec against direct rows."""
    p, far, near, L, I0, hm = build(1 << 16, 128, 0)
    b = hm.batch
    rng = np.random.default_rng(5)
    for idx in rng.choice(len(far), 60, replace=False):
        r0, nr, c0, nc = (int(v) for v in far[idx, :4])
        sub = li.Problem(li.SRC_LAPLACE, nr, nc, X=p.X[r0:r0 + nr], Y=p.X[c0:c0 + nc])
        o = oracle.ca_run_adaptive(sub, (28, 40, 64), 2, 3, I0[idx], h=1.05, rank_tol=1e-6)
        g = b.block(int(idx))
        assert (g["k"], g["status"], g["rank"]) == (o["k"], o["status"], o["rank"]), idx
        np.testing.assert_array_equal(g["I"], o["I"])
        np.testing.assert_array_equal(g["J"], o["J"])
        np.testing.assert_array_equal(g["C"], o["C"])
        np.testing.assert_array_equal(g["R"], o["R"])
    x = li.rhs(p.m, 1, 2)[:, 0]
    y = hm.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    rows = rng.choice(p.m, 256, replace=False)
    y_d = direct_rows(p.X, x, rows)
    assert np.linalg.norm(y[rows] - y_d) <= 2e-6 * np.linalg.norm(y_d)


@pytest.mark.parametrize("entries", ["f64", "f32"])
def test_matrix_free_matvec_equals_stored_factors(entries):
    """The matrix-free form (the batch keeps only I, J and U; C_b and R_b are
    re-evaluated from the points on every call) gives the stored form's y bit
    for bit, on FP64 and FP32 kernel entries (2^16 points, 128-point leaves)."""
    import paper_1710_07946_gb300 as lra
    p, far, near, L = li.fmm_partition(1 << 16, leaf=128, seed=4)
    X = torch.from_numpy(p.X).cuda()
    prob = lra.Problem.kernel("laplace", X, X, entries=entries)
    I0 = li.block_initial_rows(far[:, :4], 64, 5)
    stored = lra.HMatrix(prob, far, near, L, I0, k=64)
    free = lra.HMatrix(prob, far, near, L, I0, k=64, matrix_free=True)
    assert "C" not in free.batch.out and "R" not in free.batch.out
    stored.build()
    free.build()
    x = torch.from_numpy(li.rhs(p.m, 1, 11)[:, 0]).cuda()
    y1 = stored.matvec(x)
    y2 = free.matvec(x)
    torch.cuda.synchronize()
    for key in ("I", "J", "U", "info"):
        assert torch.equal(stored.batch.out[key], free.batch.out[key]), key
    assert torch.equal(y1, y2)


def test_matrix_free_matvec_at_two_to_the_twenty_points():
    """FMM stage (iii) on 2^20 uniform points (1024-point leaves: far blocks of
    levels 2..4 with 16k-, 2k- and 256-point boxes, the level-2 pairs cut into
    8k pieces, 657k generator runs in one batched launch, FP32 kernel entries):
    the matrix-free matvec against the
    direct product on 256 sampled rows.  The generators hold every block to
    1e-6 (tolerance and staged sizes of the FMM batch), so the matvec's
    relative error is of that order; 2e-6 is asserted."""
    import paper_1710_07946_gb300 as lra
    p, far, near, L = li.fmm_partition(1 << 20, leaf=1024, seed=1, max_block=8192)
    assert L == 4 and len(far) > 600000 and far[:, 1].max() <= 8192
    X = torch.from_numpy(p.X).cuda()
    prob = lra.Problem.kernel("laplace", X, X, entries="f32")
    hm = lra.HMatrix(prob, far, near, L, li.block_initial_rows(far[:, :4], 64, 2), k=64, matrix_free=True)
    hm.build()
    x = li.rhs(p.m, 1, 3)[:, 0]
    y = hm.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    info = hm.batch.out["info"].cpu().numpy()
    assert np.all((info[:, 3] == 0) | (info[:, 3] >= 16))
    rows = np.random.default_rng(4).choice(p.m, 256, replace=False)
    y_d = np.concatenate([direct_rows(p.X, x, rows[i:i + 4]) for i in range(0, 256, 4)])
    assert np.linalg.norm(y[rows] - y_d) <= 2e-6 * np.linalg.norm(y_d)
