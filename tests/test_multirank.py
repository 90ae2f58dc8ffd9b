"""The multi-GPU path of the benchmark on CPU: world-size-2 gloo ranks.

Each rank runs its own independent problem of the same size (weak scaling; no
collective on the data path); the only exchange is the whole-job total after the
timed region: the slowest rank's time and the sum of the ranks' units.  The
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
