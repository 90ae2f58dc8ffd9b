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
