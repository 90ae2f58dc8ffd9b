"""Batched C-A (one persistent launch over many blocks) against the FP64 oracle
run block by block: pivots bit-exact, C and R identical, U within 1e-10."""
import numpy as np
import pytest

import lra_inputs as li
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_helpers import to_device  # noqa: E402


def check_block(o, g):
    assert g["status"] == o["status"], (g["status"], o["status"])
    assert g["swaps"] == o["swaps"] and g["loops"] == o["loops"]
    np.testing.assert_array_equal(g["I"], o["I"])
    np.testing.assert_array_equal(g["J"], o["J"])
    np.testing.assert_array_equal(g["C"], o["C"])
    np.testing.assert_array_equal(g["R"], o["R"])
    assert g["rank"] == o["rank"]
    if o["rank"] > 0:
        assert np.abs(g["U"] - o["U"]).max() <= 1e-10 * np.abs(o["U"]).max()


def run_batch(p, blocks, k, sweeps, rank_tol, seed=0, check=None, h=1.01):
    import paper_1710_07946_gb300 as lra
    prob, _ = to_device(p)
    I0 = li.block_initial_rows(blocks, k, seed)
    bt = lra.Batch(prob, blocks, k, sweeps, I0, h=h, rank_tol=rank_tol)
    lra.lra_ca_run_batched(bt)
    torch.cuda.synchronize()
    idx = range(len(blocks)) if check is None else check
    for b in idx:
        r0, nr, c0, nc = blocks[b]
        kb = int(min(k, nr, nc))
        if p.src == li.SRC_DENSE:
            sub = li.Problem(li.SRC_DENSE, int(nr), int(nc), W=np.ascontiguousarray(p.W[r0:r0 + nr, c0:c0 + nc]))
        else:
            sub = li.Problem(p.src, int(nr), int(nc), X=p.X[r0:r0 + nr], Y=p.Y[c0:c0 + nc], ell=p.ell,
                             entries=p.entries)
        o = oracle.ca_run(sub, kb, sweeps, I0[b, :kb], h=h, rank_tol=rank_tol)
        check_block(o, bt.block(b))
    return bt, I0


def run_batch_staged(p, blocks, stages, margin, sweeps, rank_tol, seed=0, check=None, h=1.01):
    """Batched run with staged generator sizes; blocks checked against the oracle's
    staged run (final size, stage count, pivots, factors, counters)."""
    import paper_1710_07946_gb300 as lra
    prob, _ = to_device(p)
    kmax = stages[-1]
    I0 = li.block_initial_rows(blocks, kmax, seed)
    bt = lra.Batch(prob, blocks, kmax, sweeps, I0, h=h, rank_tol=rank_tol, stages=stages, rank_margin=margin)
    lra.lra_ca_run_batched(bt)
    torch.cuda.synchronize()
    idx = range(len(blocks)) if check is None else check
    for b in idx:
        r0, nr, c0, nc = blocks[b]
        if p.src == li.SRC_DENSE:
            sub = li.Problem(li.SRC_DENSE, int(nr), int(nc), W=np.ascontiguousarray(p.W[r0:r0 + nr, c0:c0 + nc]))
        else:
            sub = li.Problem(p.src, int(nr), int(nc), X=p.X[r0:r0 + nr], Y=p.Y[c0:c0 + nc], ell=p.ell,
                             entries=p.entries)
        o = oracle.ca_run_adaptive(sub, stages, margin, sweeps, I0[b], h=h, rank_tol=rank_tol)
        g = bt.block(b)
        assert g["k"] == o["k"], (b, g["k"], o["k"])
        check_block(o, g)
    return bt, I0


def test_staged_sizes_fmm_blocks():
    """Generator sizes 28, 40, 64 (margin 2) fitted per block to the nucleus rank:
    every block equals the oracle's staged run, bit for bit in the pivots."""
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=96, seed=2)
    bt, _ = run_batch_staged(p, blocks, (28, 40, 64), 2, 3, 1e-6)
    info = bt.out["info"].cpu().numpy()
    assert set(info[:, 6]) <= {28, 40, 64} and info[:, 6].max() >= 40     # some blocks grew
    np.testing.assert_array_equal(info[:, 7], info[:, 6])                 # square generators


def test_staged_sizes_dense_low_rank_and_small_blocks():
    """Dense blocks of exact rank 12 (some smaller than the stages): stages 8, 16, 32
    with margin 2 stop at 16; blocks below a stage size are clipped."""
    p = li.factor_gaussian(1200, 12, 0.0, seed=4)
    blocks = li.dense_blocks(1200, sizes=(5, 12, 15, 40, 300), seed=2)
    run_batch_staged(p, blocks, (8, 16, 32), 2, 3, 1e-9)


def test_staged_sizes_fmm_benchmark_workload_sampled_blocks():
    p, blocks, lev = li.fmm_blocks(npts=1 << 20, seed=0)
    sizes = blocks[:, 1] * blocks[:, 3]
    pick = list(np.argsort(sizes)[:3]) + list(np.argsort(sizes)[-2:])
    run_batch_staged(p, blocks, (28, 40, 64), 2, 3, 1e-6, check=pick, h=1.05)


def test_cta_shapes_give_identical_results_and_tuner_picks_one():
    """Every CTA shape of the batched kernel (threads per CTA x CTAs per SM) computes
    the same bits; the autotuner times them all and stores a known shape."""
    import paper_1710_07946_gb300 as lra
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=96, seed=5)
    prob, _ = to_device(p)
    I0 = li.block_initial_rows(blocks, 64, 1)
    shapes = lra.lra_ca_batched_shapes()
    assert len(shapes) >= 2 and all(t * c == 512 for t, c in shapes)
    outs = []
    ran = []
    for t, c in shapes:
        bt = lra.Batch(prob, blocks, 64, 3, I0, rank_tol=1e-6, stages=(28, 40, 64))
        bt.cb.cta_threads, bt.cb.ctas_per_sm = t, c
        try:
            lra.lra_ca_run_batched(bt)
        except RuntimeError:          # a shape whose shared memory cannot hold k = 64
            continue
        ran.append((t, c))
        torch.cuda.synchronize()
        outs.append({key: v.cpu().numpy() for key, v in bt.out.items()})
    for o in outs[1:]:
        for key in outs[0]:
            np.testing.assert_array_equal(o[key], outs[0][key], err_msg=key)
    bt = lra.Batch(prob, blocks, 64, 3, I0, rank_tol=1e-6, stages=(28, 40, 64))
    ms = lra.lra_ca_batched_tune(bt, reps=1)
    assert len(ran) >= 2 and set(ms) == set(ran) and all(v > 0 for v in ms.values())
    assert (bt.cb.cta_threads, bt.cb.ctas_per_sm) == min(ms, key=ms.get)
    for key, v in bt.out.items():
        np.testing.assert_array_equal(v.cpu().numpy(), outs[0][key], err_msg=key)
    bt.cb.cta_threads, bt.cb.ctas_per_sm = 300, 1          # not a built shape
    with pytest.raises(RuntimeError):
        lra.lra_ca_run_batched(bt)


@pytest.mark.parametrize("shape", [(512, 1), (256, 2)])
def test_cta_pairs_for_large_blocks(shape):
    """Blocks larger than pair_min_len run on pairs of CTAs that split their strips
    (lra_batch.pair_blocks): every block equals the oracle's staged run on the same
    FP32 entries, bit for bit in the pivots, and the outputs equal a run without
    pairs."""
    import paper_1710_07946_gb300 as lra
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=96, seed=8)
    prob64, _ = to_device(p)
    prob = lra.Problem.kernel("laplace", prob64.X, prob64.Y, entries="f32")
    stages = (28, 40, 50, 64)
    I0 = li.block_initial_rows(blocks, 64, 5)
    mx = np.maximum(blocks[:, 1], blocks[:, 3])
    lim = int(np.sort(mx)[len(mx) * 2 // 3])          # the largest third run on pairs
    bp = lra.Batch(prob, blocks, 64, 2, I0, h=1.05, rank_tol=1e-6, stages=stages, rank_margin=2, pair_min_len=lim)
    assert 0 < bp.cb.pair_blocks < len(blocks)
    bp.cb.cta_threads, bp.cb.ctas_per_sm = shape
    lra.lra_ca_run_batched(bp)
    bs = lra.Batch(prob, blocks, 64, 2, I0, h=1.05, rank_tol=1e-6, stages=stages, rank_margin=2)
    lra.lra_ca_run_batched(bs)
    torch.cuda.synchronize()
    op = {key: v.cpu().numpy() for key, v in bp.out.items()}
    os_ = {key: v.cpu().numpy() for key, v in bs.out.items()}
    np.testing.assert_array_equal(op["info"], os_["info"])
    for b in range(len(blocks)):
        gp, gs = bp.block(b, op), bs.block(b, os_)
        for key in ("I", "J", "C", "U", "R"):
            np.testing.assert_array_equal(gp[key], gs[key], err_msg=f"{key} of block {b}")
        r0, nr, c0, nc = (int(x) for x in blocks[b])
        if mx[b] > lim or b % 5 == 0:
            pb = li.Problem(li.SRC_LAPLACE, nr, nc, X=p.X[r0:r0 + nr], Y=p.Y[c0:c0 + nc], entries="f32")
            o = oracle.ca_run_adaptive(pb, stages, 2, 2, I0[b], h=1.05, rank_tol=1e-6)
            assert gp["k"] == o["k"], (b, gp["k"], o["k"])
            check_block(o, gp)


def test_stage_schedule_tuner_keeps_the_error_bound():
    """lra_ca_batched_tune_stages times every candidate schedule of generator sizes,
    keeps those under which every block's sampled error against the FP64 entries is
    <= tol, and leaves the fastest one's results in the batch: they equal a direct
    run of that schedule bit for bit, and every block equals the oracle run under it
    on the same FP32 entries.  No qualifying schedule and a malformed one are errors."""
    import paper_1710_07946_gb300 as lra
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=96, seed=9)
    prob64, _ = to_device(p)
    prob = lra.Problem.kernel("laplace", prob64.X, prob64.Y, entries="f32")
    I0 = li.block_initial_rows(blocks, 64, 3)
    Q, S = li.block_sample_positions(blocks, 16, 16, 4)
    Qd, Sd = torch.from_numpy(Q).cuda(), torch.from_numpy(S).cuda()
    cands = [(28, 40, 64), ((28, 40, 52, 64), 2), (24, 64), ((32, 48, 64), 1)]
    bt = lra.Batch(prob, blocks, 64, 2, I0, h=1.05, rank_tol=1e-6, stages=(28, 40, 64))
    table = lra.lra_ca_batched_tune_stages(bt, cands, Qd, Sd, exact=prob64, tol=1e-6, reps=1)
    assert len(table) == len(cands)
    chosen = (tuple(bt.stages), bt.rank_margin)
    ok = {key: v for key, v in table.items() if v[1] <= 1e-6}
    assert chosen in ok and table[chosen][0] == min(v[0] for v in ok.values())
    tuned = {key: v.cpu().numpy() for key, v in bt.out.items()}
    direct = lra.Batch(prob, blocks, 64, 2, I0, h=1.05, rank_tol=1e-6, stages=chosen[0], rank_margin=chosen[1])
    lra.lra_ca_run_batched(direct)
    torch.cuda.synchronize()
    dout = {key: v.cpu().numpy() for key, v in direct.out.items()}
    np.testing.assert_array_equal(dout["info"], tuned["info"])
    np.testing.assert_array_equal(dout["logvol"], tuned["logvol"])
    for b in range(len(blocks)):        # the slots a block uses (earlier candidates may have left the rest)
        gd, gt = direct.block(b, dout), bt.block(b, tuned)
        for key in ("I", "J", "C", "U", "R"):
            np.testing.assert_array_equal(gd[key], gt[key], err_msg=f"{key} of block {b}")
    for b in range(0, len(blocks), 7):
        r0, nr, c0, nc = (int(x) for x in blocks[b])
        pb = li.Problem(li.SRC_LAPLACE, nr, nc, X=p.X[r0:r0 + nr], Y=p.Y[c0:c0 + nc], entries="f32")
        o = oracle.ca_run_adaptive(pb, chosen[0], chosen[1], 2, I0[b], h=1.05, rank_tol=1e-6)
        g = direct.block(b, dout)
        assert g["k"] == o["k"], (b, g["k"], o["k"])
        check_block(o, g)
    with pytest.raises(lra.LraError):
        lra.lra_ca_batched_tune_stages(bt, [(28, 40, 64)], Qd, Sd, exact=prob64, tol=1e-30, reps=1)
    with pytest.raises(lra.LraError):
        lra.lra_ca_batched_tune_stages(bt, [(28, 40, 60)], Qd, Sd, exact=prob64, tol=1e-6, reps=1)


def test_dense_blocks_of_mixed_sizes():
    p = li.factor_gaussian(1500, 12, 1e-4, seed=3)
    blocks = li.dense_blocks(1500, sizes=(1, 7, 40, 64, 65, 300, 900), seed=1)
    run_batch(p, blocks, 16, 3, 1e-13)


def test_laplace_fmm_blocks_small_tree():
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=96, seed=2)
    assert len(blocks) > 20
    run_batch(p, blocks, 32, 3, 1e-6)


def test_laplace_fmm_blocks_f32_entries():
    """FP32 kernel entries, FP64 pivots and nucleus: every block equals the oracle run
    on the same FP32 entries, and the largest residual sampled against the FP64
    entries stays within twice the FP64 run's plus the FP32 perturbation."""
    import paper_1710_07946_gb300 as lra
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=96, seed=2)
    p32 = li.Problem(p.src, p.m, p.n, X=p.X, Y=p.Y, entries="f32")
    bt32, I0 = run_batch(p32, blocks, 32, 3, 1e-6)
    prob64, _ = to_device(p)
    bt64 = lra.Batch(prob64, blocks, 32, 3, I0, rank_tol=1e-6)
    lra.lra_ca_run_batched(bt64)
    Q, S = li.block_sample_positions(blocks, 32, 32, 5)
    Qd, Sd = torch.from_numpy(Q).cuda(), torch.from_numpy(S).cuda()
    e32 = lra.lra_residual_sample_batched(bt32, Qd, Sd, problem=prob64).cpu().numpy()[:, 4]
    e64 = lra.lra_residual_sample_batched(bt64, Qd, Sd).cpu().numpy()[:, 4]
    assert e32.max() <= 2 * e64.max() + 2.0 ** -22, (e32.max(), e64.max())


def test_invalid_block_is_isolated():
    import paper_1710_07946_gb300 as lra
    p = li.factor_gaussian(300, 5, 1e-3, seed=1)
    blocks = np.array([[0, 100, 0, 120], [250, 100, 0, 50], [10, 60, 200, 90]], dtype=np.int64)
    prob, _ = to_device(p)
    I0 = li.block_initial_rows(np.array([[0, 100, 0, 120], [250, 50, 0, 50], [10, 60, 200, 90]]), 8, 0)
    bt = lra.Batch(prob, blocks, 8, 2, I0)
    lra.lra_ca_run_batched(bt)
    torch.cuda.synchronize()
    st = bt.out["info"][:, 3].cpu().numpy()
    assert st[1] == lra.LRA_ERR_INVALID_ARG and st[0] in (0, 16) and st[2] in (0, 16)


def test_batched_residual_matches_oracle():
    import paper_1710_07946_gb300 as lra
    p = li.factor_gaussian(800, 10, 1e-4, seed=5)
    blocks = li.dense_blocks(800, sizes=(30, 200), seed=4)
    bt, I0 = run_batch(p, blocks, 12, 2, 1e-13, check=[0])
    Q, S = li.block_sample_positions(blocks, 16, 12, 9)
    st = lra.lra_residual_sample_batched(bt, torch.from_numpy(Q).cuda(), torch.from_numpy(S).cuda()).cpu().numpy()
    for b in range(len(blocks)):
        r0, nr, c0, nc = blocks[b]
        sub = li.Problem(li.SRC_DENSE, int(nr), int(nc), W=np.ascontiguousarray(p.W[r0:r0 + nr, c0:c0 + nc]))
        g = bt.block(b)
        so = oracle.residual_sample(sub, g["C"], g["U"], g["R"], Q[b], S[b])
        np.testing.assert_allclose(st[b, 1:], so[1:], rtol=1e-9, atol=1e-300)
        assert abs(st[b, 0] - so[0]) <= 1e-9 * so[2] + 1e-300


def test_fmm_benchmark_workload_sampled_blocks():
    """The 1M-point octree workload (about 4096 well-separated block pairs, 64..2048
    points per box, Laplace kernel, k <= 64, rank tolerance 1e-6), as the
    benchmark runs it; the oracle checks a sample of small and large blocks."""
    p, blocks, lev = li.fmm_blocks(npts=1 << 20, seed=0)
    sizes = blocks[:, 1] * blocks[:, 3]
    pick = list(np.argsort(sizes)[:3]) + list(np.argsort(sizes)[-2:])
    run_batch(p, blocks, 64, 3, 1e-6, check=pick, h=1.05)


def test_headline_fmm_configuration_every_block():
    """The benchmark's default step exactly as bench.py builds it (2^20 points,
    4096 block pairs, FP32 Laplace entries, staged sizes 28/40/50/64 with margin 2,
    h = 1.05, tol 1e-6, the autotuned CTA shape, then the residual sample against
    the FP64 entries): every block equals the oracle's staged run on the same
    FP32 entries -- final size, counters, status, pivots, C and R bit for bit, U
    within 1e-10 -- and every block's sampled Frobenius ratio agrees with the
    oracle's to 1e-6 relative (an allowed 1e-10 difference in U can move the
    ~1e-7 residual in its later digits), with the same verdict at the 1e-6
    bound that the metric counts."""
    import bench
    wl = bench.FmmWorkload(entries="f32")
    h = wl.host(0)
    d = wl.device(h, torch.device("cuda:0"))
    wl.step(d)
    torch.cuda.synchronize()
    bt = d["bt"]
    gstats = d["stats"].cpu().numpy()
    p, blocks = h["p"], h["blocks"]
    assert len(blocks) == 4096
    out = {key: v.cpu().numpy() for key, v in bt.out.items()}          # one read-back of the whole batch
    o_err = np.empty(len(blocks))
    for b in range(len(blocks)):
        r0, nr, c0, nc = (int(v) for v in blocks[b])
        sub = li.Problem(li.SRC_LAPLACE, nr, nc, X=p.X[r0:r0 + nr], Y=p.Y[c0:c0 + nc])
        sube = li.Problem(li.SRC_LAPLACE, nr, nc, X=sub.X, Y=sub.Y, entries="f32")
        o = oracle.ca_run_adaptive(sube, wl.stages, wl.margin, wl.sweeps, h["I0"][b], h=wl.h, rank_tol=wl.tol)
        g = bt.block(b, out)
        assert g["k"] == o["k"], (b, g["k"], o["k"])
        check_block(o, g)
        o_err[b] = oracle.residual_sample(sub, o["C"], o["U"], o["R"], h["Q"][b], h["S"][b])[4]
    np.testing.assert_allclose(gstats[:, 4], o_err, rtol=1e-6, atol=0)
    np.testing.assert_array_equal(gstats[:, 4] <= bench.ERR_BOUND, o_err <= bench.ERR_BOUND)


def test_bf16_laplace_entries_fmm_blocks():
    """BF16 Laplace entries (the FP32 entry rounded to bfloat16) with FP64 pivots,
    LU, swaps and nucleus: every block of a staged batch equals the oracle's run
    on the same BF16 entries, bit for bit in the pivots."""
    p, blocks, lev = li.fmm_blocks(npts=1 << 15, leaf=64, min_size=64, max_size=2048, nblocks=48, seed=6)
    p.entries = "bf16"
    run_batch_staged(p, blocks, (28, 40, 64), 2, 3, 1e-6, h=1.05)


def test_kernel_counts_the_algorithmic_flops_of_each_block():
    """lra_cur_batch.work: per block, every maxvol step's LU, back substitution,
    reciprocals, swaps and entries plus 5 k^3 per nucleus.  On square blocks
    without stages both phases of a loop see the same strip length, so the total
    follows from the loop and swap counts alone: the first (cold) step, then warm
    steps, each swap 2 (k - 1) n + n."""
    import paper_1710_07946_gb300 as lra
    p = li.factor_gaussian(1200, 12, 1e-3, seed=9)
    blocks = np.array([[0, 300, 300, 300], [300, 500, 700, 500], [100, 64, 900, 64]], dtype=np.int64)
    prob, _ = to_device(p)
    k = 16
    I0 = li.block_initial_rows(blocks, k, 3)
    bt = lra.Batch(prob, blocks, k, 3, I0, rank_tol=1e-9)
    lra.lra_ca_run_batched(bt)
    work = bt.work.cpu().numpy()
    info = bt.out["info"].cpu().numpy()

    def step(k, n):
        lu = (n - k) * k * (k - 1) / 2 + (k - 1) * k * (2 * k - 1) / 6
        bs = (n - k) * k * (k - 1) / 2
        return 2 * (lu + bs) + (n - k) * k + 2 * k

    for b, (r0, nr, c0, nc) in enumerate(blocks):
        loops, swaps = int(info[b, 2]), int(info[b, 1])
        kb = min(k, nr)
        expect = 2 * loops * step(kb, nr) + swaps * (2 * (kb - 1) * nr + nr) + 5.0 * kb ** 3
        np.testing.assert_allclose(work[b], expect, rtol=1e-12)
