"""The multi-GPU path of the benchmark on CPU: world-size-2 gloo ranks.

The batched FMM workload on N GPUs is one block list of N batches of the
recipe, partitioned across the ranks by LPT on rows x columns x k (paper:
Section "Application: HSS / FMM" -- the generators are independent), with no
collective on the data path; the only exchange is the whole-job total after the
timed region: the slowest rank's time and the sum of the ranks' units.  A
replica mode (an independent problem per rank) remains as an option.  The
reference arm runs on rank 0 alone."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r: 10 (r + 1) ms and 100 + r units
        t, u = bench.job_totals(10.0 * (rank + 1), 100 + rank, world, torch.device("cpu"))
        # per-rank problem of the benchmark recipe (small size): same shape, different draw
        wl = bench.FmmWorkload(npts=1 << 12, nblocks=24, k=16)
        h = wl.host(rank)
        sig = (len(h["blocks"]), int(h["I0"].shape[1]), float(h["p"].X[:4].sum()))
        q.put((rank, t, u, sig))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_total_and_independent_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t, u, _ in res:
        assert t == 20.0 and u == 201.0              # max of times, sum of units, on every rank
    (_, _, _, s0), (_, _, _, s1) = res
    assert s0[:2] == s1[:2] and s0[2] != s1[2]        # same problem size, independent draws


def _lpt_rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        wl = bench.FmmWorkload(npts=1 << 12, nblocks=12, k=16, stages=(8, 16), margin=2)
        wl.world = world
        h = wl.host(rank)
        # this rank's units: the oracle's C-A + nucleus + residual on every block of its share
        good, n, _ = bench.fmm_oracle_blocks(wl.oracle_ctx(h), range(len(h["blocks"])), float("inf"))
        _, total = bench.job_totals(1.0, good, world, torch.device("cpu"))
        q.put((rank, [int(v) for v in h["share"]], n, good, total))
    finally:
        dist.destroy_process_group()


def test_lpt_shards_of_one_block_list_on_two_gloo_ranks():
    """The two ranks' shares partition the job's one list (complete, disjoint),
    their loads are LPT-balanced (differ by at most the largest block), and the
    ranks' unit counts add up, through the host reduction, to the count of the
    whole list processed on one rank."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1710_07946_gb300 import shard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lpt_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = bench.FmmWorkload(npts=1 << 12, nblocks=12, k=16, stages=(8, 16), margin=2)
    full = wl.job_list(2)
    nb = len(full["blocks"])
    assert nb == 2 * len(wl.problem(0)["blocks"])
    s0, s1 = set(res[0][1]), set(res[1][1])
    assert s0.isdisjoint(s1) and s0 | s1 == set(range(nb))
    cost = shard.block_costs(full["blocks"], wl.k)
    l0, l1 = cost[sorted(s0)].sum(), cost[sorted(s1)].sum()
    assert abs(l0 - l1) <= cost.max()
    good_one, n_one, _ = bench.fmm_oracle_blocks(wl.oracle_ctx(full), range(nb), float("inf"))
    assert n_one == nb and res[0][2] + res[1][2] == nb
    assert res[0][4] == res[1][4] == float(good_one) == float(res[0][3] + res[1][3])


def test_lpt_partition_rule():
    """LPT list scheduling by hand on a small case, ties to the lower index / part."""
    from paper_1710_07946_gb300 import shard
    parts = shard.lpt_partition([5, 3, 3, 2, 2, 1], 2)
    # order 5(0) 3(1) 3(2) 2(3) 2(4) 1(5): 0->A(5); 1->B(3); 2->B(6); 3->A(7); 4->B(8); 5->A(8)
    assert [list(p) for p in parts] == [[0, 3, 5], [1, 2, 4]]
    assert [list(p) for p in shard.lpt_partition([1, 1, 1], 5)] == [[0], [1], [2], [], []]
    one = shard.lpt_partition(np.arange(10.0), 1)
    assert list(one[0]) == list(range(10))
    with pytest.raises(ValueError):
        shard.lpt_partition([1, -1], 2)
    b = np.array([[0, 100, 0, 50], [0, 10, 5, 70]])
    np.testing.assert_array_equal(shard.block_costs(b, 16), [100 * 50 * 16, 10 * 70 * 10])


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class NoWork:
        def host(self, rank):
            raise AssertionError("rank 1 must not build the workload")

    class Args:
        steps, warmup, ref_budget, gpus = 1, 0, 1.0, 2

    assert bench.run_reference(Args(), NoWork()) is None
    assert capsys.readouterr().out == ""


def test_single_rank_totals_are_the_local_figures():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(12.5, 7, 1, torch.device("cpu")) == (12.5, 7.0)
    assert np.isfinite(bench.job_totals(0.5, 0, 1, "cpu")[0])
