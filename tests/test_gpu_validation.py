"""Host-side argument checks of the newer entry points: bad sizes, kinds and
problems are refused with LRA_ERR_INVALID_ARG before anything is launched."""
import ctypes as ct

import numpy as np
import pytest

import lra_inputs as li

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import to_device  # noqa: E402


def _err(fn, *a, **kw):
    import paper_1710_07946_gb300 as lra
    with pytest.raises(lra.LraError) as e:
        fn(*a, **kw)
    return e.value


def test_rhtcur_rejects_bad_sizes():
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(50, 40, r=4, seed=1)
    prob, _ = to_device(p)
    e = _err(lra.lra_rhtcur_run, prob, torch.zeros(40, 41, dtype=torch.float64, device="cuda"))   # k > min(m, n)
    assert "INVALID_ARG" in str(e)
    e = _err(lra.lra_rhtcur_run, prob, torch.zeros(40, 65, dtype=torch.float64, device="cuda"))
    assert "INVALID_ARG" in str(e)
    with pytest.raises(ValueError):
        lra.lra_rhtcur_run(prob, torch.zeros(39, 4, dtype=torch.float64, device="cuda"))         # n rows needed


def test_leverage_batch_rejects_bad_parameters():
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(100, 100, r=4, seed=2)
    prob, _ = to_device(p)
    blocks = np.array([[0, 100, 0, 100]], dtype=np.int64)
    I0 = li.block_initial_rows(blocks, 8, 1)
    draws = np.zeros((1, 2, 100))
    assert "INVALID_ARG" in str(_err(lra.LevBatch, prob, blocks, 8, 9, 1, 0, I0, draws))          # r > k
    assert "INVALID_ARG" in str(_err(lra.LevBatch, prob, blocks, 8, 4, 1, 4, I0, draws))          # kind 4
    assert "INVALID_ARG" in str(_err(lra.LevBatch, prob, blocks, 8, 4, 1, -1, I0, draws))         # kind -1
    with pytest.raises(ValueError):
        lra.LevBatch(prob, blocks, 8, 4, 2, 0, I0, draws)                                          # draws too short


def test_leverage_batch_flags_blocks_smaller_than_k():
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(100, 100, r=4, seed=3)
    prob, _ = to_device(p)
    blocks = np.array([[0, 100, 0, 100], [0, 6, 0, 100], [0, 100, 95, 10]], dtype=np.int64)       # small, outside
    I0 = np.zeros((3, 8), dtype=np.int32)
    lb = lra.LevBatch(prob, blocks, 8, 4, 1, 0, I0, np.random.default_rng(0).random((3, 2, 100)))
    lra.lra_ca_lev_batched(lb)
    info = lb.out["info"].cpu().numpy()
    assert info[0, 3] in (0, 16) and info[1, 3] == lra.LRA_ERR_INVALID_ARG and info[2, 3] == lra.LRA_ERR_INVALID_ARG


def test_hmatvec_rejects_non_laplace_problems():
    import paper_1710_07946_gb300 as lra
    p, far, near, L = li.fmm_partition(1 << 10, leaf=16, seed=1)
    X = torch.from_numpy(p.X).cuda()
    hm = lra.HMatrix(lra.Problem.kernel("laplace", X, X), far, near, L, li.block_initial_rows(far[:, :4], 8, 1), k=8,
                     stages=None)
    hm.build()
    x = torch.zeros(p.m, dtype=torch.float64, device="cuda")
    hm.matvec(x)
    hm.problem = lra.Problem.kernel("gaussian", X, X, 0.5)
    assert "INVALID_ARG" in str(_err(hm.matvec, x))


def test_oversample_cycles_reject_bad_pmax():
    import paper_1710_07946_gb300 as lra
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=8, seed=8)
    prob, _ = to_device(p)
    bt = lra.Batch(prob, blocks, 8, 2, li.block_initial_rows(blocks, 8, 1))
    lra.lra_ca_run_batched(bt)
    assert "INVALID_ARG" in str(_err(lra.Oversampled, bt, 4, 17))
    ov = lra.Oversampled(bt, 4, 2)
    assert "INVALID_ARG" in str(_err(lra.lra_oversample_cycle_batched, bt, 4, 2, -1, ov))       # max cycles < 0
    with pytest.raises(ValueError):
        lra.lra_oversample_cycle_batched(bt, 4, 3, 4, ov)                                         # workspace for pmax 2


def test_multiplier_apply_and_gather_reject_bad_arguments():
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(30, 20, r=3, seed=4)
    prob, _ = to_device(p)
    q = li.Problem(li.SRC_DENSE, 30, 21, W=np.zeros((30, 21)))
    li.with_bidiag(q, 2, 1)
    _, mult21 = to_device(q)
    assert "INVALID_ARG" in str(_err(lra.lra_multiplier_apply, prob, mult21))                     # n mismatch
    assert "INVALID_ARG" in str(_err(lra.lra_gather_rows, prob, torch.zeros(0, dtype=torch.int32, device="cuda")))
    with pytest.raises(ValueError):
        lra.lra_multiplier_apply(prob, None, out=torch.zeros(30, 19, dtype=torch.float64, device="cuda"))


def test_residual_sample_catches_out_of_range_indices():
    """A sample index outside [0, m) or [0, n) is caught on the device before it
    is read through: every statistic is NaN, and the next valid call is fine."""
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(64, 48, r=4, seed=5)
    prob, _ = to_device(p)
    I0 = torch.arange(4, dtype=torch.int32, device="cuda")
    out = lra.lra_ca_run(prob, I0, 4, 2)
    good_q = torch.arange(0, 64, 3, dtype=torch.int32, device="cuda")
    good_s = torch.arange(0, 48, 5, dtype=torch.int32, device="cuda")
    for q, s in ((torch.tensor([0, -1, 5], dtype=torch.int32, device="cuda"), good_s),
                 (torch.tensor([0, 64], dtype=torch.int32, device="cuda"), good_s),
                 (good_q, torch.tensor([48, 1], dtype=torch.int32, device="cuda")),
                 (good_q, torch.tensor([2, -7], dtype=torch.int32, device="cuda"))):
        st = lra.lra_residual_sample(prob, out["C"], out["U"], out["R"], q, s).cpu().numpy()
        assert np.isnan(st).all(), st
    st = lra.lra_residual_sample(prob, out["C"], out["U"], out["R"], good_q, good_s).cpu().numpy()
    assert np.isfinite(st).all() and st[4] < 1e-4


def test_batched_residual_flags_only_the_block_with_a_bad_index():
    import paper_1710_07946_gb300 as lra
    p, blocks, lev = li.fmm_blocks(npts=1 << 13, leaf=64, min_size=64, max_size=2048, nblocks=4, seed=9)
    prob, _ = to_device(p)
    bt = lra.Batch(prob, blocks, 8, 2, li.block_initial_rows(blocks, 8, 1))
    lra.lra_ca_run_batched(bt)
    nb = len(blocks)
    Q = np.zeros((nb, 6), dtype=np.int32)
    S = np.zeros((nb, 5), dtype=np.int32)
    for b in range(nb):
        Q[b] = np.arange(6) % blocks[b, 1]
        S[b] = np.arange(5) % blocks[b, 3]
    Q[1, 2] = -3                       # negative row in block 1
    S[2, 4] = blocks[2, 3]             # one past the last column in block 2
    st = lra.lra_residual_sample_batched(bt, torch.from_numpy(Q).cuda(), torch.from_numpy(S).cuda()).cpu().numpy()
    assert np.isnan(st[1]).all() and np.isnan(st[2]).all()
    assert np.isfinite(st[0]).all() and np.isfinite(st[3]).all()


def test_gauss_apply_flags_out_of_range_pivots():
    import paper_1710_07946_gb300 as lra
    rng = np.random.default_rng(11)
    nb, m, n, k, nrhs = 3, 96, 80, 8, 4
    X = torch.from_numpy(rng.random((nb, m, 3))).cuda()
    Y = torch.from_numpy(rng.random((nb, n, 3)) + np.array([2.0, 0, 0])).cuda()
    I = np.stack([rng.choice(m, k, replace=False) for _ in range(nb)]).astype(np.int32)
    J = np.stack([rng.choice(n, k, replace=False) for _ in range(nb)]).astype(np.int32)
    I[1, 3] = m                        # block 1: row pivot out of range
    J[2, 0] = -1                       # block 2: column pivot out of range
    x = torch.from_numpy(rng.standard_normal((nb, n, nrhs)).astype(np.float32)).cuda()
    y, ctx = lra.lra_gauss_cur_forward(X, Y, torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda(), 0.3, x)
    y = y.cpu().numpy()
    assert np.isnan(y[1]).all() and np.isnan(y[2]).all() and np.isfinite(y[0]).all()
    assert np.isnan(ctx[1].cpu().numpy()).all()
    dy = torch.ones(nb, m, nrhs, dtype=torch.float32, device="cuda")
    g = lra.lra_gauss_cur_backward(X, Y, torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda(), 0.3, x, dy, ctx,
                                   entry_grads=True)
    for key in ("dx", "dC", "dR", "dG"):
        v = g[key].cpu().numpy()
        assert np.isnan(v[1]).all() and np.isnan(v[2]).all() and np.isfinite(v[0]).all(), key
    dl = g["dell"].cpu().numpy()
    assert np.isnan(dl[1]) and np.isnan(dl[2]) and np.isfinite(dl[0])


def test_left_multiplier_order_must_match_rows():
    """A left multiplier is m x m: a handle of order n (or a right one of order m)
    is refused before anything is launched."""
    import paper_1710_07946_gb300 as lra
    p = li.dense_lowrank(64, 32, r=3, seed=6)
    prob, _ = to_device(p)
    q = li.Problem(li.SRC_DENSE, 64, 32, W=np.zeros((64, 32)))
    li.with_arht(q, 2, 1, side="right")                       # order 32
    wrong = lra.lra_precondition("arht", 32, 2, q.perm, q.dsign, side="left")
    I0 = torch.arange(3, dtype=torch.int32, device="cuda")
    assert "INVALID_ARG" in str(_err(lra.lra_ca_run, prob, I0, 3, 2, multiplier=wrong))
    li.with_arht(q, 2, 1, side="left")                        # order 64
    right64 = lra.lra_precondition("arht", 64, 2, q.perm, q.dsign, side="right")
    assert "INVALID_ARG" in str(_err(lra.lra_ca_run, prob, I0, 3, 2, multiplier=right64))
    with pytest.raises(KeyError):
        lra.lra_precondition("arht", 64, 2, q.perm, q.dsign, side="up")
