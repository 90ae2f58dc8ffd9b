"""Mixed precision (LRA_MODE_MIXED): maxvol steps run in FP32 with certified
decisions and fall back to FP64 when the bounds cannot certify one.  The index
sets, swap counts, C, R and U must equal the FP64 oracle's exactly; the volume
trace is computed from FP32 pivots (relative accuracy ~1e-6)."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import gpu_ca, to_device  # noqa: E402

MIXED = 1


def check_exact(o, g):
    assert g["status"] == o["status"], (g["status"], o["status"])
    assert g["loops"] == o["loops"] and g["swaps"] == o["swaps"], (g["loops"], o["loops"], g["swaps"], o["swaps"])
    np.testing.assert_array_equal(g["I"], o["I"])
    np.testing.assert_array_equal(g["J"], o["J"])
    np.testing.assert_array_equal(g["C"], o["C"])
    np.testing.assert_array_equal(g["R"], o["R"])
    assert g["rank"] == o["rank"]
    if o["rank"]:
        assert np.abs(g["U"] - o["U"]).max() <= 1e-10 * np.abs(o["U"]).max()
    lo, lg = o["logvol"], g["logvol"]
    fin = np.isfinite(lo)
    assert np.array_equal(np.isnan(lo), np.isnan(lg))
    np.testing.assert_allclose(lg[fin], lo[fin], rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("noise", [1e-8, 0.0])
def test_mixed_dense_256(seed, noise):
    p = li.dense_lowrank(256, 256, r=8, noise=noise, seed=seed)
    I0 = li.initial_rows(256, 8, 1000 + seed)
    o = oracle.ca_run(p, 8, 3, I0)
    g = gpu_ca(p, 8, 3, I0, mode=MIXED)
    check_exact(o, g)
    assert g["fp32_steps"] + g["fp64_steps"] == 2 * g["loops"]


@pytest.mark.parametrize("mult,arg", [("none", 0), ("arht", 1), ("arht", 2), ("arht", 3), ("sparse", 4)])
def test_mixed_float32_multipliers(mult, arg):
    p = li.dense_spiky(1024, r=16, seed=3)
    if mult == "arht":
        li.with_arht(p, arg, 11)
    elif mult == "sparse":
        li.with_sparse(p, arg, 11)
    I0 = li.initial_rows(1024, 24, 5)
    o = oracle.ca_run(p, 24, 4, I0)
    g = gpu_ca(p, 24, 4, I0, mode=MIXED)
    check_exact(o, g)
    if mult == "arht" and arg == 2:
        assert g["fp32_steps"] > 0       # this input certifies most steps in FP32


@pytest.mark.parametrize("k", [8, 32, 64])
def test_mixed_laplace(k):
    p = li.laplace_clusters(1500, 1300, seed=2)
    I0 = li.initial_rows(1500, k, 9)
    o = oracle.ca_run(p, k, 3, I0, rank_tol=1e-6)
    g = gpu_ca(p, k, 3, I0, mode=MIXED, rank_tol=1e-6)
    check_exact(o, g)


def test_mixed_exact_ties_fall_back_and_stay_exact():
    """Duplicated columns give exact ties that no bound can separate: the steps
    fall back to FP64 and the result is still the oracle's."""
    g0 = np.random.default_rng(1)
    base = g0.standard_normal((300, 40))
    W = np.ascontiguousarray(np.concatenate([base, base[:, :20]], axis=1))
    p = li.Problem(li.SRC_DENSE, 300, 60, W=W)
    I0 = li.initial_rows(300, 10, 4)
    o = oracle.ca_run(p, 10, 3, I0)
    g = gpu_ca(p, 10, 3, I0, mode=MIXED)
    check_exact(o, g)


def test_mixed_rank_deficient_and_nonfinite():
    p = li.factor_gaussian(200, 5, 0.0, seed=2)
    W = p.W.copy(); W[:, :] = 0.0; W[:, :3] = p.W[:, :3]
    p.W = W
    I0 = li.initial_rows(200, 6, 1)
    o = oracle.ca_run(p, 6, 2, I0)
    g = gpu_ca(p, 6, 2, I0, mode=MIXED)
    assert o["status"] == g["status"] == 16
    np.testing.assert_array_equal(g["I"], o["I"])
    np.testing.assert_array_equal(g["J"], o["J"])
    p2 = li.dense_lowrank(128, 128, r=4, seed=0)
    I0 = li.initial_rows(128, 4, 1)
    p2.W[I0[2], 17] = np.nan
    assert gpu_ca(p2, 4, 2, I0, mode=MIXED)["status"] == 3


def test_mixed_batched_fmm_blocks_equal_fp64():
    """The FMM batch in mixed mode: every block's results equal the FP64 run's
    (and the oracle's on sampled blocks), whichever path each step took."""
    import paper_1710_07946_gb300 as lra
    p, blocks, lev = li.fmm_blocks(npts=1 << 17, nblocks=256, seed=3)
    prob, _ = to_device(p)
    I0 = li.block_initial_rows(blocks, 64, 7)
    b64 = lra.Batch(prob, blocks, 64, 3, I0, rank_tol=1e-6)
    lra.lra_ca_run_batched(b64)
    b32 = lra.Batch(prob, blocks, 64, 3, I0, rank_tol=1e-6, mode=MIXED)
    lra.lra_ca_run_batched(b32)
    torch.cuda.synchronize()
    for key in ("I", "J", "C", "R", "U"):
        np.testing.assert_array_equal(b32.out[key].cpu().numpy(), b64.out[key].cpu().numpy())
    i64, i32 = b64.out["info"].cpu().numpy(), b32.out["info"].cpu().numpy()
    np.testing.assert_array_equal(i32[:, :4], i64[:, :4])
    assert (i32[:, 4] + i32[:, 5] == 2 * i32[:, 2]).all()
    for b in (0, len(blocks) - 1):
        r0, nr, c0, nc = blocks[b]
        sub = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=p.X[r0:r0 + nr], Y=p.Y[c0:c0 + nc])
        o = oracle.ca_run(sub, 64, 3, I0[b], rank_tol=1e-6)
        g = b32.block(b)
        np.testing.assert_array_equal(g["I"], o["I"])
        np.testing.assert_array_equal(g["J"], o["J"])
