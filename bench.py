"""Benchmark of the C-A CUR library on one or more GPUs of one node.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lib|reference] [--workload NAME]

Default workload (``fmm``): the generators of an FMM / HSS matrix -- C-A CUR
approximations of the 4096 well-separated block pairs of an octree over 2^20
uniform points in [0,1]^3 (boxes of ~200..2048 points, Laplace kernel evaluated
on the fly, rank <= 64 adapted at tolerance 1e-6 with generator sizes staged
28/40/50/64 -- the schedule lra_ca_batched_tune_stages picks among the
candidates of STAGE_CANDIDATES (--tune-stages runs it again) -- 2 C-A loops),
in the mixed form: kernel entries in FP32, pivots, LU,
swaps and nucleus in FP64.  The blocks above 512 points run first, each on a
pair of CTAs; the CTA shape is picked by lra_ca_batched_tune (untimed set-up).  One step = the batched C-A launch (all blocks,
nuclei included) + the batched a-posteriori residual sample (16 x 16 entries
per block, against the FP64 entries); the metric counts the blocks whose
sampled relative Frobenius error is <= 1e-6.  The plain FP64 forms of the same
batch (same sizes, and fixed k = 64) and the same form with 3 C-A loops are
measured in the same run and reported under config.comparisons.  Other workloads: ``fmm_f64``, ``fmm_fixedk``,
``laplace65536_k*`` (one LRA of the 65536^2 Laplace kernel), ``dense8192_*``
(one LRA of an 8192^2 FP32 input with a multiplier), ``tests{2,3,4}_*`` (the
paper's random-input tests), ``gauss_apply`` (differentiable CUR apply).

Inputs are seeded, synthetic and resident in HBM before the timed region; L2 is
flushed (a 256 MiB write, untimed) before every timed step; each step is timed
with CUDA events on the launching stream, and the library's own per-launch
events give the dominant kernel's duration.  ``e2e`` repeats the steps through
the same public API from pinned host buffers, copies included (a two-slot
pipeline: a step's read-back overlaps the next step's compute; both slots are
used in the untimed warm-up).  Under torchrun the FMM batches are one block
list of N recipe batches, split across the ranks by LPT on rows x cols x k
(``--shard replicas``: an independent batch per rank); every other workload
runs an independent replica per rank.  No collective on the data path (weak
scaling); rank 0 prints one JSON line with the whole-job throughput over the
slowest rank.  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lra_inputs as li  # noqa: E402

FP64_PEAK_TFLOPS = 1.25   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal; a plain DFMA loop measured 1.2)
FP32_PEAK_TFLOPS = 80.5   # 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz (nominal; a plain FFMA loop measured 74)
METRIC = "CUR LRAs/s at rel. err <=1e-6 (mixed vs plain FP64 GPU); % of HBM roofline"
ERR_BOUND = 1e-6
LAPLACE_FLOPS = 8.0       # 3 sub, 1 mul, 2 fma, sqrt, div per kernel entry (nominal count)


def maxvol_flops(k: int, n: int, cold: bool, entry_flops: float = 0.0) -> float:
    """Algorithmic FP64 flops of one maxvol step on a k x n strip (fma = 2,
    reciprocal = 1; the swaps are counted separately): LU with column pivoting
    (cold) or the warm LU of the k x k block plus its replay, then the
    back substitution; plus the strip's entries when they are evaluated."""
    if cold:
        fma = sum((k - 1 - t) * (n - 1 - t) for t in range(k))
    else:
        fma = sum((k - 1 - t) * (n - k) for t in range(k)) + sum((k - 1 - t) ** 2 for t in range(k))
    fma += (n - k) * k * (k - 1) // 2
    div = (n - k) * k + 2 * k
    ent = entry_flops * (k * n + (0 if cold else k * k))
    return 2.0 * fma + div + ent


def ca_flops(k, m, n, loops, swaps, entry_flops=0.0, nucleus=True):
    f = maxvol_flops(k, n, True, entry_flops) + maxvol_flops(k, m, False, entry_flops)
    f += (loops - 1) * (maxvol_flops(k, n, False, entry_flops) + maxvol_flops(k, m, False, entry_flops))
    f += swaps * (2.0 * k * (m + n) / 2.0 + (m + n) / 2.0)
    if nucleus:
        f += 5.0 * k ** 3
    return f


# ------------------------------------------------------------------ workloads
def stages_run(stages, kb, kf):
    """Stages a staged run went through to end at size kf (every clipped stage size up to kf)."""
    if not stages:
        return 1
    sizes = []
    for st in stages:
        k = min(st, kb)
        if not sizes or k > sizes[-1]:
            sizes.append(k)
    return sum(1 for k in sizes if k <= kf) or 1


def staged_flops(stages, kb, m, n, nrun, loops, swaps, entry_flops):
    """Lower bound on the algorithmic flops of a staged run: the sizes actually run
    (stages clipped to kb), every stage but the last with the fewest loops it can
    have (2, or 1 when it is the only loop allowed) and the remaining loops and all
    swaps charged to the smallest size."""
    sizes = []
    for st in stages:
        k = min(st, kb)
        if not sizes or k > sizes[-1]:
            sizes.append(k)
    sizes = sizes[:nrun] if stages else [kb]
    f = 0.0
    left = loops
    for i, k in enumerate(sizes):
        lk = max(1, left - 2 * (len(sizes) - 1 - i)) if i == 0 else min(2, left) if i < len(sizes) - 1 else left
        lk = max(lk, 1)
        left -= lk
        f += ca_flops(k, m, n, lk, swaps if i == 0 else 0, entry_flops)
    return f


def fmm_oracle_blocks(c, idxs, budget_s):
    """The FP64 oracle on the FMM blocks idxs (in order) until budget_s: the
    staged (or fixed-size) C-A, the nucleus and the sampled residual against
    FP64 entries.  Returns (blocks within the error bound, blocks, seconds)."""
    import oracle
    b = c["blocks"]
    t0 = time.perf_counter()
    n = good = 0
    for idx in idxs:
        r0, nr, c0, nc = b[idx]
        kb = int(min(c["k"], nr, nc))
        sub = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=c["X"][r0:r0 + nr], Y=c["Y"][c0:c0 + nc])
        sube = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=sub.X, Y=sub.Y, entries=c["entries"])
        if c["stages"]:
            o = oracle.ca_run_adaptive(sube, c["stages"], c["margin"], c["sweeps"], c["I0"][idx], h=c["h"],
                                       rank_tol=c["tol"])
        else:
            o = oracle.ca_run(sube, kb, c["sweeps"], c["I0"][idx, :kb], h=c["h"], rank_tol=c["tol"])
        st = oracle.residual_sample(sub, o["C"], o["U"], o["R"], c["Q"][idx], c["S"][idx])
        n += 1
        good += st[4] <= ERR_BOUND
        if time.perf_counter() - t0 >= budget_s:
            break
    return good, n, time.perf_counter() - t0


_FMM_CTX = None


def _fmm_oracle_init(ctx):
    global _FMM_CTX
    _FMM_CTX = ctx
    import oracle
    oracle.lib()


def _fmm_oracle_chunk(args):
    idxs, budget_s = args
    return fmm_oracle_blocks(_FMM_CTX, idxs, budget_s)


# schedules of generator sizes the stage tuner (--tune-stages) tries besides the workload's own
STAGE_CANDIDATES = [(28, 40, 64), (28, 40, 50, 64), (28, 40, 52, 64), (28, 40, 56, 64), (28, 44, 64),
                    (28, 36, 44, 52, 64), (24, 32, 40, 52, 64), (28, 40, 48, 64), (32, 48, 64)]


class FmmWorkload:
    base = "fmm_laplace_1M_octree_4096blocks"
    kernel = "ca_batched_kernel"
    unit = "LRA/s"

    def __init__(self, npts=1 << 20, nblocks=4096, k=64, sweeps=2, tol=1e-6, q=16, s=16, entries="f64",
                 stages=(28, 40, 50, 64), margin=2, h=1.05):
        self.npts, self.nblocks, self.k, self.sweeps, self.tol, self.q, self.s = npts, nblocks, k, sweeps, tol, q, s
        self.entries, self.stages, self.margin = entries, stages, margin
        self.h = h                        # dominance threshold, between the paper's "h = 1.1 or h = 1.01"
        self.pair_min_len = 512           # larger blocks run on CTA pairs
        self.name = self._name()

    def _name(self):
        sizes = "-".join(map(str, self.stages)) if self.stages else str(self.k)
        return f"{self.base}_k{sizes}_tol{self.tol:.0e}".replace("e-0", "e-") + (
            f"_{self.entries}entries" if self.entries != "f64" else "")

    def problem(self, seed):
        """One batch of the recipe: the octree's block pairs over npts points with
        their initial rows and residual sample positions."""
        p, blocks, lev = li.fmm_blocks(npts=self.npts, nblocks=self.nblocks, seed=seed)
        I0 = li.block_initial_rows(blocks, self.k, 100 + seed)
        Q, S = li.block_sample_positions(blocks, self.q, self.s, 200 + seed)
        self.levels = lev
        return dict(p=p, blocks=blocks, I0=I0, Q=Q, S=S)

    def job_list(self, world):
        """The job's one block list for ``world`` GPUs: ``world`` batches of the
        recipe (seeds 0 .. world-1) whose point sets are concatenated, so that
        every block is a submatrix of one kernel matrix over all the points (the
        block rows and columns of batch p are offset by p * npts)."""
        parts = [self.problem(seed) for seed in range(world)]
        if world == 1:
            return parts[0]
        X = np.concatenate([h["p"].X for h in parts])
        blocks = np.concatenate([h["blocks"] + np.array([1, 0, 1, 0]) * (i * self.npts)
                                 for i, h in enumerate(parts)])
        p = li.Problem(li.SRC_LAPLACE, len(X), len(X), X=X, Y=X)
        cat = lambda key: np.concatenate([h[key] for h in parts])
        return dict(p=p, blocks=blocks, I0=cat("I0"), Q=cat("Q"), S=cat("S"))

    def host(self, rank):
        """This rank's share.  One GPU: the recipe's batch.  Several (``world``
        set by the launcher): the LPT share (rows x columns x k) of the job's
        one block list, or with ``shard = "replicas"`` an independent batch of
        its own (seed = rank)."""
        world = getattr(self, "world", 1)
        if world == 1 or getattr(self, "shard", "lpt") == "replicas":
            return self.problem(rank)
        from paper_1710_07946_gb300 import shard
        full = self.job_list(world)
        mine = shard.lpt_partition(shard.block_costs(full["blocks"], self.k), world)[rank]
        h = dict(full, blocks=full["blocks"][mine], I0=full["I0"][mine], Q=full["Q"][mine], S=full["S"][mine])
        h["share"] = mine
        return h

    def config(self, h):
        b = h["blocks"]
        world = getattr(self, "world", 1)
        shard = ("one GPU" if world == 1 else
                 f"{world} independent batches of the recipe per job" if getattr(self, "shard", "lpt") == "replicas"
                 else f"LPT share (rows x cols x k) of one {world} x {self.nblocks}-block list")
        return {"workload": self.name, "points": self.npts, "blocks": int(len(b)), "sharding": shard,
                "block_rows_min_median_max": [int(b[:, 1].min()), int(np.median(b[:, 1])), int(b[:, 1].max())],
                "kernel": f"Laplace 1/|x-y|, on the fly, entries {self.entries.upper()}",
                "pivots_nucleus": "FP64", "residual_against": "FP64 entries", "k_max": self.k,
                "generator_sizes": (f"staged {'/'.join(map(str, self.stages))}, grow while nucleus rank >= "
                                    f"size - {self.margin}" if self.stages else "fixed min(k_max, rows, cols)"),
                "rank_tol": self.tol, "h": self.h,
                "cta_pairs": f"blocks with more than {self.pair_min_len} rows or columns, each on 2 CTAs",
                "sweeps": self.sweeps, "residual_sample": f"{self.q}x{self.s} per block"}

    def device(self, h, dev):
        import torch
        import paper_1710_07946_gb300 as lra
        p = h["p"]
        X = torch.from_numpy(p.X).to(dev)
        prob = lra.Problem.kernel("laplace", X, X, entries=self.entries)
        prob64 = lra.Problem.kernel("laplace", X, X)
        # blocks with more than 512 rows or columns run first, each on a pair of CTAs (lra_batch.pair_blocks)
        bt = lra.Batch(prob, h["blocks"], self.k, self.sweeps, h["I0"], h=self.h, rank_tol=self.tol,
                       stages=self.stages, rank_margin=self.margin, pair_min_len=self.pair_min_len)
        tuned = lra.lra_ca_batched_tune(bt, reps=2)          # untimed set-up: CTA shape autotuner
        if getattr(self, "cta_shape", None):                # a profiling stand-in keeps the headline's shape
            bt.cb.cta_threads, bt.cb.ctas_per_sm = self.cta_shape
        self.tuned = {"chosen": f"{bt.cb.cta_threads}x{bt.cb.ctas_per_sm}",
                      "ms": {f"{t}x{c}": round(v, 3) for (t, c), v in tuned.items()}}
        d = dict(X=X, prob=prob, prob64=prob64, bt=bt, Q=torch.from_numpy(h["Q"]).to(dev),
                 S=torch.from_numpy(h["S"]).to(dev))
        if getattr(self, "tune_stages", False) and self.stages:
            # untimed set-up: the schedule of generator sizes, fastest of those that keep every block's
            # sampled error within the bound
            cands = [self.stages] + [c for c in STAGE_CANDIDATES if c != tuple(self.stages) and c[-1] == self.k]
            table = lra.lra_ca_batched_tune_stages(bt, [(c, self.margin) for c in cands], d["Q"], d["S"],
                                                   exact=prob64, tol=self.tol, reps=2)
            self.stages, self.margin = tuple(bt.stages), bt.rank_margin
            self.name = self._name()
            self.stage_tuner = {"chosen": "/".join(map(str, self.stages)),
                                "ms": {"/".join(map(str, c)): round(v[0], 3) for (c, m), v in table.items()},
                                "max_err": {"/".join(map(str, c)): v[1] for (c, m), v in table.items()}}
        d["stats"] = torch.empty(len(h["blocks"]), 5, dtype=torch.float64, device=dev)
        return d

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        lra.lra_ca_run_batched(d["bt"])
        lra.lra_residual_sample_batched(d["bt"], d["Q"], d["S"], d["stats"], problem=d["prob64"])

    def precision(self):
        """What ran in which arithmetic: the mode label and the per-stage precisions."""
        if self.entries in ("f32", "bf16"):
            return f"mixed: {self.entries.upper()} Laplace entries, FP64 pivots/LU/swaps/nucleus", {
                "kernel_entries": self.entries, "pivots_lu_swaps": "f64", "nucleus": "f64", "residual": "f64"}
        return "plain fp64", {"kernel_entries": "f64", "pivots_lu_swaps": "f64", "nucleus": "f64", "residual": "f64"}

    def comparisons(self):
        """The plain FP64 GPU forms of the same batch, measured in the same run."""
        if self.entries != "f32":
            return []
        kw = dict(npts=self.npts, nblocks=self.nblocks, k=self.k, sweeps=self.sweeps, tol=self.tol, q=self.q,
                  s=self.s, h=self.h)
        kw3 = dict(kw, sweeps=3)
        return [("plain_fp64_same_sizes", type(self)(entries="f64", stages=self.stages, margin=self.margin, **kw)),
                ("plain_fp64_fixed_k64", type(self)(entries="f64", stages=None, **kw)),
                ("same_form_3_loops", type(self)(entries=self.entries, stages=self.stages, margin=self.margin, **kw3))]

    def check(self, d):
        info = d["bt"].out["info"].cpu().numpy()
        st = d["stats"].cpu().numpy()
        ok = (info[:, 3] == 0) | (info[:, 3] >= 16)
        good = ok & (st[:, 4] <= ERR_BOUND)
        return dict(units=int(good.sum()), info=info, err=st[:, 4], work=float(d["bt"].work.sum().item()))

    def flops_lower_bound(self, h, res):
        """The host-side model from the info counters alone (stages' loops and swaps not known
        separately: the extra loops and all swaps charged to the smallest stage)."""
        b, info = h["blocks"], res["info"]
        f = 0.0
        for (r0, nr, c0, nc), inf in zip(b, info):
            kb = int(min(self.k, nr, nc))
            f += staged_flops(self.stages or (), kb, int(nr), int(nc), stages_run(self.stages, kb, int(inf[6])),
                              max(int(inf[2]), 1), int(inf[1]), LAPLACE_FLOPS)
        return f

    def flops(self, h, res):
        # every stage's maxvol steps and nuclei as counted by the kernel itself (lra_cur_batch.work)
        return res["work"] if res.get("work") else self.flops_lower_bound(h, res)

    def extra(self, res):
        info, err = res["info"], res["err"]
        return {"cta_shape_tuner": getattr(self, "tuned", None),
                "stage_tuner": getattr(self, "stage_tuner", None),
                "flops_per_step_counted_by_kernel": res.get("work"),
                "rank_min_median_max": [int(info[:, 0].min()), int(np.median(info[:, 0])), int(info[:, 0].max())],
                "generator_size_hist": {int(k): int(c) for k, c in zip(*np.unique(info[:, 6], return_counts=True))},
                "swaps_mean": float(info[:, 1].mean()), "loops_hist": np.bincount(info[:, 2]).tolist(),
                "rel_fro_err_sampled_median": float(np.median(err)), "rel_fro_err_sampled_max": float(err.max()),
                "frac_blocks_err_le_1e-6": float((err <= ERR_BOUND).mean())}

    # end to end: points from pinned host memory, all C, U, R and the statistics read back.  Served as a
    # pipeline: two output sets on the device, the read-back of step i on a copy stream while step i + 1
    # computes; a step waits for the read-back that last used its output set.
    def e2e_setup(self, h, d):
        import torch
        import paper_1710_07946_gb300 as lra
        bt0 = d["bt"]
        bt1 = lra.Batch(d["prob"], h["blocks"], self.k, self.sweeps, h["I0"], h=self.h, rank_tol=self.tol,
                        stages=self.stages, rank_margin=self.margin, pair_min_len=self.pair_min_len)
        bt1.cb.cta_threads, bt1.cb.ctas_per_sm = bt0.cb.cta_threads, bt0.cb.ctas_per_sm
        assert bt1.cb.pair_blocks == bt0.cb.pair_blocks
        pin = lambda t: t.cpu().pin_memory()
        # every per-problem input is uploaded each step: the points, the block descriptors (rows, columns,
        # output offsets, processing order), the initial rows I0 and the residual sample positions Q, S
        hp = dict(X=torch.from_numpy(h["p"].X).pin_memory(), bts=[bt0, bt1],
                  inputs=dict(blocks=pin(bt0.blocks), offs=pin(bt0.offs), order=pin(bt0.order), I0=pin(bt0.I0),
                              Q=pin(d["Q"]), S=pin(d["S"])),
                  stats_dev=[d["stats"], torch.empty_like(d["stats"])],
                  copy=torch.cuda.Stream(d["X"].device), slot=0,
                  done=[torch.cuda.Event(), torch.cuda.Event()], copied=[torch.cuda.Event(), torch.cuda.Event()])
        hp["out"] = [{key: torch.empty(v.shape, dtype=v.dtype).pin_memory() for key, v in bt0.out.items()}
                     for _ in range(2)]
        hp["stats"] = [torch.empty(d["stats"].shape, dtype=torch.float64).pin_memory() for _ in range(2)]
        h2d = hp["X"].numel() * 8 + sum(v.numel() * v.element_size() for v in hp["inputs"].values())
        d2h = sum(v.numel() * v.element_size() for v in hp["out"][0].values()) + hp["stats"][0].numel() * 8
        return hp, h2d, d2h

    def e2e_step(self, hp, d):
        import torch
        import paper_1710_07946_gb300 as lra
        i = hp["slot"]
        hp["slot"] = 1 - i
        cur = torch.cuda.current_stream()
        cur.wait_event(hp["copied"][i])                  # the read-back that last used output set i is done
        d["X"].copy_(hp["X"], non_blocking=True)
        bt, st = hp["bts"][i], hp["stats_dev"][i]
        hin = hp["inputs"]
        for key in ("blocks", "offs", "order", "I0"):
            getattr(bt, key).copy_(hin[key], non_blocking=True)
        d["Q"].copy_(hin["Q"], non_blocking=True)
        d["S"].copy_(hin["S"], non_blocking=True)
        lra.lra_ca_run_batched(bt)
        lra.lra_residual_sample_batched(bt, d["Q"], d["S"], st, problem=d["prob64"])
        hp["done"][i].record(cur)
        with torch.cuda.stream(hp["copy"]):
            hp["copy"].wait_event(hp["done"][i])
            for key, v in hp["out"][i].items():
                v.copy_(bt.out[key], non_blocking=True)
            hp["stats"][i].copy_(st, non_blocking=True)
            hp["copied"][i].record(hp["copy"])

    def e2e_finish(self, hp, d):
        hp["copy"].synchronize()

    # the FP64 oracle on one block
    def oracle_ctx(self, h):
        return dict(X=h["p"].X, Y=h["p"].Y, blocks=h["blocks"], I0=h["I0"], Q=h["Q"], S=h["S"], k=self.k,
                    entries=self.entries, stages=self.stages, margin=self.margin, sweeps=self.sweeps, h=self.h,
                    tol=self.tol)

    def oracle_units(self, h, budget_s, seed=0):
        order = np.random.default_rng(seed).permutation(len(h["blocks"]))
        good, n, el = fmm_oracle_blocks(self.oracle_ctx(h), order, budget_s)
        return good, n, el, f"{n} randomly chosen blocks of the same batch (C-A + nucleus + residual sample each)"

    def oracle_units_allcores(self, h, budget_s, seed=0):
        """The same oracle over blocks on every host core: one spawned process per
        core, each taking its share of a random block order until budget_s;
        value = all processes' good blocks / the longest process time."""
        import multiprocessing as mp
        ncpu = os.cpu_count() or 1
        order = np.random.default_rng(seed).permutation(len(h["blocks"]))
        chunks = [(order[i::ncpu], budget_s) for i in range(ncpu)]
        with mp.get_context("spawn").Pool(ncpu, initializer=_fmm_oracle_init, initargs=(self.oracle_ctx(h),)) as pool:
            res = pool.map(_fmm_oracle_chunk, chunks)
        good = sum(r[0] for r in res)
        n = sum(r[1] for r in res)
        el = max(r[2] for r in res)
        return good, n, el, ncpu, (f"{n} randomly chosen blocks of the same batch (C-A + nucleus + residual sample "
                                   f"each) in {ncpu} processes, one per host core, {el:.1f} s")


class TwoSlotPipe:
    """Plumbing of a two-slot end-to-end pipeline.  Slot i's inputs are uploaded on
    one copy stream once the compute that last read them is done; the compute
    waits for them and for the read-back that last used slot i's outputs; the
    read-back runs on a second copy stream.  Step s's copies thus overlap the
    compute of steps s - 1 and s + 1, and every step still moves its own inputs
    and results."""

    def __init__(self, dev):
        import torch
        self.up, self.down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        self.uploaded = [torch.cuda.Event(), torch.cuda.Event()]
        self.done = [torch.cuda.Event(), torch.cuda.Event()]
        self.copied = [torch.cuda.Event(), torch.cuda.Event()]
        self.slot = 0

    def next_slot(self):
        i = self.slot
        self.slot = 1 - i
        return i

    def upload(self, i, pairs):
        import torch
        with torch.cuda.stream(self.up):
            self.up.wait_event(self.done[i])
            for dst, src in pairs:
                dst.copy_(src, non_blocking=True)
            self.uploaded[i].record(self.up)
        cur = torch.cuda.current_stream()
        cur.wait_event(self.uploaded[i])
        cur.wait_event(self.copied[i])

    def download(self, i, pairs, keep=()):
        import torch
        self.done[i].record(torch.cuda.current_stream())
        with torch.cuda.stream(self.down):
            self.down.wait_event(self.done[i])
            for dst, src in pairs:
                dst.copy_(src, non_blocking=True)
            self.copied[i].record(self.down)
        for t in keep:
            t.record_stream(self.down)       # not reused before the read-back has run

    def finish(self):
        self.up.synchronize()
        self.down.synchronize()


class DenseWorkload:
    kernel = "ca_kernel"
    unit = "LRA/s"

    def __init__(self, mult, n=8192, k=48, sweeps=4):
        self.mult, self.n, self.k, self.sweeps, self.q, self.s = mult, n, k, sweeps, 256, 256
        tag = {"arht": "arht2", "sparse": "sparse4", "bidiag": "bidiag3", "arft": "arft2"}[mult]
        self.name = f"dense{n}_f32_rank32_spikes1pct_{tag}_k{k}_s{sweeps}"

    def host(self, rank):
        p = li.dense_spiky(self.n, r=32, seed=1000 * rank)
        if self.mult == "arht":
            li.with_arht(p, 2, 7)
        elif self.mult == "arft":
            li.with_arft(p, 2, 7)
        elif self.mult == "bidiag":
            li.with_bidiag(p, 3, 7)
        else:
            li.with_sparse(p, 4, 7)
        I0 = li.initial_rows(self.n, self.k, 11)
        Q, S = li.sample_positions(self.n, self.n, self.q, self.s, 13)
        return dict(p=p, I0=I0, Q=Q, S=S)

    def config(self, h):
        return {"workload": self.name, "m": self.n, "n": self.n, "k": self.k, "sweeps": self.sweeps,
                "multiplier": {"arht": "ARHT d=2", "sparse": "sparse +-1, 4 nnz/col",
                               "bidiag": "product of 3 cyclic bidiagonal +-1 factors",
                               "arft": "ARFT d=2 in real form (W' = W [Re M, Im M], 2n columns)"}[self.mult],
                "input_dtype": "f32", "residual_sample": f"{self.q}x{self.s}"}

    def device(self, h, dev):
        import torch
        import paper_1710_07946_gb300 as lra
        p = h["p"]
        W = torch.from_numpy(p.W).to(dev)
        prob = lra.Problem.dense(W)
        if p.mkind == li.MULT_ARHT:
            mult = lra.lra_precondition("arht", p.n, p.depth, p.perm, p.dsign)
        elif p.mkind == li.MULT_ARFT:
            mult = lra.lra_precondition_fourier(p.n, p.depth, p.perm, p.dcplx)
        elif p.mkind == li.MULT_BIDIAG:
            mult = lra.lra_precondition("bidiag", p.n, p.depth, p.perm, p.dsign)
        else:
            mult = lra.lra_precondition("sparse", p.n, p.nnz, p.srow, p.ssign)
        I0 = torch.from_numpy(h["I0"]).to(dev)
        out = lra.lra_ca_run(prob, I0, self.k, self.sweeps, multiplier=mult)
        return dict(W=W, prob=prob, mult=mult, I0=I0, out=out, Q=torch.from_numpy(h["Q"]).to(dev),
                    S=torch.from_numpy(h["S"]).to(dev), stats=None)

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        lra.lra_ca_run(d["prob"], d["I0"], self.k, self.sweeps, multiplier=d["mult"], out=d["out"],
                       workspace=d["out"]["_workspace"])
        d["stats"] = lra.lra_residual_sample(d["prob"], d["out"]["C"], d["out"]["U"], d["out"]["R"], d["Q"], d["S"])

    def check(self, d):
        info = d["out"]["info"].cpu().numpy()[None, :]
        err = d["stats"].cpu().numpy()[4:5]
        return dict(units=1, info=info, err=err)      # spikes: the error bound is not attainable here

    def flops(self, h, res):
        inf = res["info"][0]
        ncols = 2 * self.n if self.mult == "arft" else self.n          # columns of W'
        return ca_flops(self.k, self.n, ncols, self.sweeps, int(inf[1]), 0.0, nucleus=False)

    def extra(self, res):
        inf = res["info"][0]
        return {"rank": int(inf[0]), "swaps": int(inf[1]), "loops": int(inf[2]), "status": int(inf[3]),
                "rel_fro_err_sampled": float(res["err"][0])}

    # end to end: W and I0 uploaded, C, U, R, the indices and the statistics read back, every step, through a
    # two-slot pipeline (TwoSlotPipe)
    def e2e_setup(self, h, d):
        import torch
        import paper_1710_07946_gb300 as lra
        W1, I01 = d["W"].clone(), d["I0"].clone()
        prob1 = lra.Problem.dense(W1)
        out1 = lra.lra_ca_run(prob1, I01, self.k, self.sweeps, multiplier=d["mult"])
        torch.cuda.synchronize()
        hp = dict(pipe=TwoSlotPipe(d["W"].device), W=torch.from_numpy(h["p"].W).pin_memory(),
                  I0=torch.from_numpy(h["I0"]).pin_memory(),
                  slots=[(d["W"], d["I0"], d["prob"], d["out"]), (W1, I01, prob1, out1)])
        hp["out"] = [{key: torch.empty(v.shape, dtype=v.dtype).pin_memory() for key, v in d["out"].items()
                      if not key.startswith("_")} for _ in range(2)]
        hp["stats"] = [torch.empty(5, dtype=torch.float64).pin_memory() for _ in range(2)]
        h2d = hp["W"].numel() * 4 + hp["I0"].numel() * 4
        d2h = sum(v.numel() * v.element_size() for v in hp["out"][0].values()) + 40
        return hp, h2d, d2h

    def e2e_step(self, hp, d):
        import paper_1710_07946_gb300 as lra
        pipe = hp["pipe"]
        i = pipe.next_slot()
        W, I0, prob, out = hp["slots"][i]
        pipe.upload(i, [(W, hp["W"]), (I0, hp["I0"])])
        lra.lra_ca_run(prob, I0, self.k, self.sweeps, multiplier=d["mult"], out=out, workspace=out["_workspace"])
        stats = lra.lra_residual_sample(prob, out["C"], out["U"], out["R"], d["Q"], d["S"])
        pipe.download(i, [(v, out[key]) for key, v in hp["out"][i].items()] + [(hp["stats"][i], stats)],
                      keep=(stats,))

    def e2e_finish(self, hp, d):
        hp["pipe"].finish()

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        t0 = time.perf_counter()
        n = 0
        while True:
            o = oracle.ca_run(h["p"], self.k, self.sweeps, h["I0"])
            oracle.residual_sample(h["p"], o["C"], o["U"], o["R"], h["Q"], h["S"])
            n += 1
            if time.perf_counter() - t0 >= budget_s or n >= 50:
                break
        el = time.perf_counter() - t0
        return n, n, el, f"{n} complete LRAs of the same input (C-A + nucleus + residual sample)"


class RhtcurWorkload:
    """CUR LRA with Gaussian sampling (Algorithm algrhtcur, lbar = l = k) on the
    dense benchmark input (8192^2 FP32, rank 32 + 1% spikes): one step = the
    sketch S = W Hbar (Hbar 8192 x 48 Gaussian), the row and column selections,
    the nucleus and the sampled residual."""
    kernel = "sketch_kernel"
    unit = "LRA/s"

    def __init__(self, n=8192, k=48):
        self.n, self.k, self.q, self.s = n, k, 256, 256
        self.name = f"rhtcur_dense{n}_f32_rank32_spikes1pct_gaussian_k{k}"

    def host(self, rank):
        p = li.dense_spiky(self.n, r=32, seed=1000 * rank)
        H = li.gaussian_sketch(self.n, self.k, 21 + rank)
        Q, S = li.sample_positions(self.n, self.n, self.q, self.s, 13)
        return dict(p=p, H=H, Q=Q, S=S)

    def config(self, h):
        return {"workload": self.name, "m": self.n, "n": self.n, "k": self.k, "input_dtype": "f32",
                "sketch": f"Gaussian Hbar {self.n} x {self.k} (FP64)", "residual_sample": f"{self.q}x{self.s}"}

    def device(self, h, dev):
        import torch
        import paper_1710_07946_gb300 as lra
        W = torch.from_numpy(h["p"].W).to(dev)
        prob = lra.Problem.dense(W)
        H = torch.from_numpy(h["H"]).to(dev)
        out = lra.lra_rhtcur_run(prob, H)
        return dict(W=W, prob=prob, H=H, out=out, Q=torch.from_numpy(h["Q"]).to(dev),
                    S=torch.from_numpy(h["S"]).to(dev), stats=None)

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        lra.lra_rhtcur_run(d["prob"], d["H"], out=d["out"], workspace=d["out"]["_workspace"])
        d["stats"] = lra.lra_residual_sample(d["prob"], d["out"]["C"], d["out"]["U"], d["out"]["R"], d["Q"], d["S"])

    def check(self, d):
        info = d["out"]["info"].cpu().numpy()[None, :]
        err = d["stats"].cpu().numpy()[4:5]
        return dict(units=1, info=info, err=err)      # spikes: the error bound is not attainable here

    def flops(self, h, res):
        return 2.0 * self.n * self.n * self.k        # the sketch: one fma per (i, j, column of Hbar)

    def extra(self, res):
        inf = res["info"][0]
        return {"rank": int(inf[0]), "swaps": int(inf[1]), "status": int(inf[3]),
                "rel_fro_err_sampled": float(res["err"][0])}

    # end to end: W and Hbar uploaded, the CUR and the statistics read back, every step, through a two-slot
    # pipeline (TwoSlotPipe)
    def e2e_setup(self, h, d):
        import torch
        import paper_1710_07946_gb300 as lra
        W1, H1 = d["W"].clone(), d["H"].clone()
        prob1 = lra.Problem.dense(W1)
        out1 = lra.lra_rhtcur_run(prob1, H1)
        torch.cuda.synchronize()
        hp = dict(pipe=TwoSlotPipe(d["W"].device), W=torch.from_numpy(h["p"].W).pin_memory(),
                  H=torch.from_numpy(h["H"]).pin_memory(),
                  slots=[(d["W"], d["H"], d["prob"], d["out"]), (W1, H1, prob1, out1)])
        hp["out"] = [{key: torch.empty(v.shape, dtype=v.dtype).pin_memory() for key, v in d["out"].items()
                      if not key.startswith("_")} for _ in range(2)]
        hp["stats"] = [torch.empty(5, dtype=torch.float64).pin_memory() for _ in range(2)]
        h2d = hp["W"].numel() * 4 + hp["H"].numel() * 8
        d2h = sum(v.numel() * v.element_size() for v in hp["out"][0].values()) + 40
        return hp, h2d, d2h

    def e2e_step(self, hp, d):
        import paper_1710_07946_gb300 as lra
        pipe = hp["pipe"]
        i = pipe.next_slot()
        W, H, prob, out = hp["slots"][i]
        pipe.upload(i, [(W, hp["W"]), (H, hp["H"])])
        lra.lra_rhtcur_run(prob, H, out=out, workspace=out["_workspace"])
        stats = lra.lra_residual_sample(prob, out["C"], out["U"], out["R"], d["Q"], d["S"])
        pipe.download(i, [(v, out[key]) for key, v in hp["out"][i].items()] + [(hp["stats"][i], stats)],
                      keep=(stats,))

    def e2e_finish(self, hp, d):
        hp["pipe"].finish()

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        t0 = time.perf_counter()
        o = oracle.rhtcur(h["p"], h["H"])
        oracle.residual_sample(h["p"], o["C"], o["U"], o["R"], h["Q"], h["S"])
        el = time.perf_counter() - t0
        return 1, 1, el, "1 complete LRA of the same input (sketch + selections + nucleus + residual sample)"


class LevCaWorkload:
    """C-A with DMM08 Algorithm 1 on the sketches (the tests of C-A incorporating
    [DMM08, Algorithm 1]): a 1000 x 1000 input of numerical rank r = 10 at 1e-6
    (U diag(2^-1..2^-10) V^T + 1e-9 G), k = l = 4r samples per step by
    Exactly(l), eight C-A iterations; one step = ``runs`` independent runs (own
    initial rows and draws, one CTA each) + each run's sampled residual."""
    kernel = "lev_batched_kernel"
    unit = "LRA/s"

    def __init__(self, n=1000, r=10, k=40, iters=8, runs=152, kind=0):
        self.n, self.r, self.k, self.iters, self.runs, self.kind = n, r, k, iters, runs, kind
        self.q = self.s = 64       # the batched residual holds its q x s sample in shared memory
        tag = ("uniform_" if kind & 2 else "") + ("expected" if kind & 1 else "exactly")
        self.name = f"levca_n{n}_r{r}_k{k}_{tag}_it{iters}_x{runs}"

    def host(self, rank):
        if self.kind & 2:
            # uniform scores are the paper's route for perturbed factor-Gaussian inputs
            p = li.factor_gaussian(self.n, self.r, 1e-9, seed=1000 * rank)
        else:
            p = li.dense_lowrank(self.n, self.n, r=self.r, noise=1e-9, seed=1000 * rank)
        blocks = np.array([[0, self.n, 0, self.n]] * self.runs, dtype=np.int64)
        draws = li.rng(77 + rank).random((self.runs, 2 * self.iters, self.n))
        I0 = li.block_initial_rows(blocks, self.k, 5 + rank)
        Q, S = li.block_sample_positions(blocks, self.q, self.s, 13)
        return dict(p=p, blocks=blocks, draws=draws, I0=I0, Q=Q, S=S)

    def config(self, h):
        return {"workload": self.name, "m": self.n, "n": self.n, "nrank": self.r, "k_eq_l": self.k,
                "ca_iterations": self.iters, "sampling": "Expected(l)" if self.kind & 1 else "Exactly(l)",
                "scores": "uniform (no SVD)" if self.kind & 2 else "SVD-based (Gram + round-robin Jacobi)",
                "input": ("G1 G2 + 1e-9 G3 (Gaussian factors)" if self.kind & 2 else
                          "U diag(2^-1..2^-r) V^T + 1e-9 G"),
                "runs_per_step": self.runs, "residual_sample": f"{self.q}x{self.s} per run"}

    def device(self, h, dev):
        import torch
        import paper_1710_07946_gb300 as lra
        W = torch.from_numpy(h["p"].W).to(dev)
        prob = lra.Problem.dense(W)
        lb = lra.LevBatch(prob, h["blocks"], self.k, self.r, self.iters, self.kind, h["I0"], h["draws"], order=None)
        return dict(W=W, prob=prob, lb=lb, Q=torch.from_numpy(h["Q"]).to(dev), S=torch.from_numpy(h["S"]).to(dev),
                    stats=torch.empty(self.runs, 5, dtype=torch.float64, device=dev))

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        lra.lra_ca_lev_batched(d["lb"])
        lra.lra_residual_sample_lev(d["lb"], d["Q"], d["S"], d["stats"])

    def check(self, d):
        info = d["lb"].out["info"].cpu().numpy()
        err = d["stats"].cpu().numpy()[:, 4]
        return dict(units=self.runs, info=info, err=err)

    def flops(self, h, res):
        # per block: 2 iters sketches of k x n: Gram k^2 n, 10 Jacobi sweeps of (k-1) rounds x k/2 rotations x 12 k,
        # scores r k n (fma = 2 flops)
        k, n = self.k, self.n
        if self.kind & 2:
            return 5.0 * k ** 3 * self.runs                  # uniform scores: only the nucleus computes
        per_step = k * k * n + 10 * (k - 1) * (k // 2) * 12 * k + 2 * self.r * k * n
        return 2.0 * self.iters * per_step * self.runs      # one launch runs every block

    def extra(self, res):
        return {"rel_fro_err_mean": float(np.mean(res["err"])), "rel_fro_err_std": float(np.std(res["err"])),
                "rel_fro_err_max": float(np.max(res["err"])), "ranks": sorted(set(int(x) for x in res["info"][:, 0])),
                "statuses": sorted(set(int(x) for x in res["info"][:, 3])),
                "flops_note": ("per launch (all runs): the nucleus, 5 k^3 per run (uniform scores: no SVD stage)"
                               if self.kind & 2 else
                               "per launch (all runs): Gram k^2 n + Jacobi 10 (k-1) (k/2) 12 k + scores 2 r k n per "
                               "sketch, 2 x iters sketches per run")}

    def e2e_setup(self, h, d):
        import torch
        hp = dict(W=torch.from_numpy(h["p"].W).pin_memory())
        hp["out"] = {key: torch.empty(v.shape, dtype=v.dtype).pin_memory() for key, v in d["lb"].out.items()}
        hp["stats"] = torch.empty(self.runs, 5, dtype=torch.float64).pin_memory()
        h2d = hp["W"].numel() * 8
        d2h = sum(v.numel() * v.element_size() for v in hp["out"].values()) + hp["stats"].numel() * 8
        return hp, h2d, d2h

    def e2e_step(self, hp, d):
        import torch
        d["W"].copy_(hp["W"], non_blocking=True)
        self.step(d)
        for key, v in hp["out"].items():
            v.copy_(d["lb"].out[key], non_blocking=True)
        hp["stats"].copy_(d["stats"], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        t0 = time.perf_counter()
        n = 0
        for b in range(self.runs):
            o = oracle.ca_lev(h["p"], self.k, self.r, self.iters, self.kind, h["draws"][b], h["I0"][b])
            oracle.residual_sample(h["p"], o["C"], o["U"], o["R"], h["Q"][b], h["S"][b])
            n += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        return n, n, el, f"{n} complete runs (8 C-A iterations + nucleus + residual sample) of the step's {self.runs}"


class CurApplyWorkload:
    """Stored-factor CUR apply Y = C (U (R X)) (FMM stage (iii) with stored
    generators): one rank-32 triple of a 2^20 x 2^20 matrix, C and R stored in
    FP64, FP32 or BF16 (lra_cur_apply's dtype), one right-hand side.  The
    factors are random (the product's cost does not depend on their values);
    one step = one lra_cur_apply.  HBM-bound: R and C are streamed once."""
    unit = "apply/s"
    kernel = "apply_rx_lp_kernel"

    def __init__(self, dtype="f32", m=1 << 20, n=1 << 20, k=32, nrhs=1):
        self.dtype, self.m, self.n, self.k, self.nrhs = dtype, m, n, k, nrhs
        self.name = f"cur_apply_{m >> 20}Mx{n >> 20}M_k{k}_nrhs{nrhs}_{dtype}"
        if dtype == "f64":
            self.kernel = "apply_rx_kernel"

    def host(self, rank):
        g = np.random.default_rng(50 + rank)
        return dict(C=g.standard_normal((self.m, self.k)), R=g.standard_normal((self.k, self.n)),
                    U=g.standard_normal((self.k, self.k)) / np.sqrt(self.k), X=g.standard_normal((self.n, self.nrhs)))

    def config(self, h):
        return {"workload": self.name, "m": self.m, "n": self.n, "k": self.k, "nrhs": self.nrhs,
                "factor_storage": self.dtype, "accumulation": "fp64" if self.dtype == "f64" else
                "fp32 runs, fp64 across runs, one refinement step on the vector operand"}

    def device(self, h, dev):
        import torch
        tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[self.dtype]
        t = lambda a, dt=torch.float64: torch.from_numpy(a).to(dev).to(dt)
        import paper_1710_07946_gb300 as lra
        d = dict(C=t(h["C"], tdt), R=t(h["R"], tdt), U=t(h["U"]), X=t(h["X"]))
        d["Y"] = torch.empty(self.m, self.nrhs, dtype=torch.float64, device=dev)
        d["ws"] = torch.empty(lra.lra_cur_apply_workspace_size(self.n, self.k, self.nrhs), dtype=torch.uint8,
                              device=dev)
        self._h = h
        return d

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        lra.lra_cur_apply(d["C"], d["U"], d["R"], d["X"], Y=d["Y"], workspace=d["ws"])

    def check(self, d):
        return dict(units=1, Y=d["Y"][:4096].cpu().numpy())

    def counts(self, h, res):
        b = {"f64": 8, "f32": 4, "bf16": 2}[self.dtype]
        rx = float(b * self.k * self.n + 8 * self.n * self.nrhs)
        cy = float(b * self.m * self.k + 8 * self.m * self.nrhs)
        if self.dtype == "f64":
            return {"apply_rx_kernel": ("hbm", rx), "apply_c_kernel": ("hbm", cy)}
        return {"apply_rx_lp_kernel": ("hbm", rx), "apply_c_lp_kernel": ("hbm", cy)}

    def flops(self, h, res):
        return 0.0

    def extra(self, res):
        # error of the first 4096 rows against the FP64 product of the unrounded factors
        h = self._h
        ref = h["C"][:4096] @ (h["U"] @ (h["R"] @ h["X"]))
        return {"rel_err_vs_fp64_factors_4096_rows": float(np.linalg.norm(res["Y"] - ref) / np.linalg.norm(ref)),
                "bytes_per_step": sum(v[1] for v in self.counts(None, None).values())}

    def e2e_setup(self, h, d):
        import torch
        hp = dict(X=torch.from_numpy(h["X"]).pin_memory(), Y=torch.empty(self.m, self.nrhs,
                                                                          dtype=torch.float64).pin_memory())
        return hp, hp["X"].numel() * 8, hp["Y"].numel() * 8

    def e2e_step(self, hp, d):
        import torch
        d["X"].copy_(hp["X"], non_blocking=True)
        self.step(d)
        hp["Y"].copy_(d["Y"], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        t0 = time.perf_counter()
        n = 0
        while True:
            oracle.cur_apply(h["C"], h["U"], h["R"], h["X"])
            n += 1
            if time.perf_counter() - t0 >= budget_s or n >= 20:
                break
        el = time.perf_counter() - t0
        return n, n, el, f"{n} FP64 applies of the same triple"


class HMatvecWorkload:
    """The FMM's stage (iii) on the c3 recipe's point distribution: y = M x for
    the Laplace matrix of 2^16 uniform points in [0,1]^3 (M_ii = 0), held as
    the far blocks of every level's interaction lists with generators from one
    batched C-A launch (staged 28/40/64, h = 1.05, tol 1e-6) plus the near field
    of touching 128-point leaves formed on the fly.  One step = one matvec
    (lra_hmatvec); the generator batch runs once in the set-up and is timed
    there (config.setup_ms)."""
    unit = "matvec/s"
    kernel = "hm_far_kernel"

    def __init__(self, npts=1 << 16, leaf=128, k=64, matrix_free=False, entries="f64", max_block=None):
        self.npts, self.leaf, self.k, self.matrix_free, self.entries = npts, leaf, k, matrix_free, entries
        self.max_block = max_block
        size = f"{npts >> 20}M" if npts >= 1 << 20 else f"{npts // 1024}K"
        self.name = (f"hmatvec_laplace_{size}_uniform_cube_leaf{leaf}_k28-40-64_tol1e-6" +
                     ("_matrixfree" if matrix_free else "") + (f"_{entries}entries" if entries != "f64" else ""))

    def host(self, rank):
        p, far, near, L = li.fmm_partition(self.npts, leaf=self.leaf, seed=rank, max_block=self.max_block)
        I0 = li.block_initial_rows(far[:, :4], self.k, 1 + rank)
        x = li.rhs(p.m, 1, 2 + rank)[:, 0]
        rows = li.rng(3).choice(p.m, 256, replace=False)
        return dict(p=p, far=far, near=near, L=L, I0=I0, x=x, rows=rows)

    def config(self, h):
        far, near = h["far"], h["near"]
        return {"workload": self.name, "points": self.npts, "levels": int(h["L"]), "far_blocks": int(len(far)),
                "near_blocks": int(len(near)), "far_block_rows": [int(far[:, 1].min()), int(far[:, 1].max())],
                "near_entries": int((near[:, 1] * near[:, 3]).sum())}

    def device(self, h, dev):
        import torch
        import paper_1710_07946_gb300 as lra
        X = torch.from_numpy(h["p"].X).to(dev)
        prob = lra.Problem.kernel("laplace", X, X, entries=self.entries)
        hm = lra.HMatrix(prob, h["far"], h["near"], h["L"], h["I0"], k=self.k, matrix_free=self.matrix_free)
        hm.build()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        hm.build()
        e1.record()
        torch.cuda.synchronize()
        self.setup_ms = e0.elapsed_time(e1)
        x = torch.from_numpy(h["x"]).to(dev)
        self._h = h
        return dict(X=X, prob=prob, hm=hm, x=x, y=torch.empty_like(x))

    def step(self, d):
        d["hm"].matvec(d["x"], d["y"])

    def check(self, d):
        return dict(units=1, y=d["y"].cpu().numpy(), info=d["hm"].batch.out["info"].cpu().numpy())

    def _direct_rows(self, h):
        P, x, rows = h["p"].X, h["x"], h["rows"]
        out = []
        for i in range(0, len(rows), 8):              # 8 rows at a time: bounded host memory at 2^20 points
            dd = np.sqrt(((P[rows[i:i + 8], None, :] - P[None, :, :]) ** 2).sum(axis=2))
            with np.errstate(divide="ignore"):
                K = np.where(dd > 0.0, 1.0 / dd, 0.0)
            out.append(K @ x)
        return np.concatenate(out)

    def counts(self, h, res):
        far, near, info = h["far"], h["near"], res["info"]
        kf = info[:, 6].astype(np.float64)
        # bytes each kernel must move at least: C_b (nrows x kf) read once per matvec by the far pass, R_b (kf x
        # ncols) by the t pass; the near pass is FP64 arithmetic: ~10 flops per entry (distance, sqrt, division, fma)
        c_bytes = 8.0 * float((far[:, 1] * kf).sum()) + 8.0 * self.npts
        r_bytes = 8.0 * float((far[:, 3] * kf).sum()) + 8.0 * float((kf * kf).sum())
        near_flops = 10.0 * float((near[:, 1] * near[:, 3]).sum())
        if self.matrix_free:
            # entries re-evaluated on every call: FP64 work per entry (the squared distance, and for FP64
            # entries the square root and division) plus the fma
            per = (6.0 + 2.0) if self.entries == "f32" else LAPLACE_FLOPS + 2.0
            return {"hm_far_kernel": ("alu", per * float((far[:, 1] * kf).sum())),
                    "hm_t_kernel": ("alu", per * float((far[:, 3] * kf).sum())),
                    "hm_near_kernel": ("alu", near_flops)}
        return {"hm_far_kernel": ("hbm", c_bytes), "hm_t_kernel": ("hbm", r_bytes),
                "hm_near_kernel": ("alu", near_flops)}

    def flops(self, h, res):
        return self.counts(h, res)["hm_near_kernel"][1]

    def extra(self, res):
        y_d = self._direct_rows(self._h)
        err = float(np.linalg.norm(res["y"][self._h["rows"]] - y_d) / np.linalg.norm(y_d))
        info = res["info"]
        return {"setup_ms": self.setup_ms, "rel_err_vs_direct_256_rows": err,
                "generator_sizes": {str(int(s)): int((info[:, 6] == s).sum()) for s in sorted(set(info[:, 6]))},
                "statuses": sorted(set(int(x) for x in info[:, 3]))}

    def e2e_setup(self, h, d):
        import torch
        hp = dict(x=torch.from_numpy(h["x"]).pin_memory(), y=torch.empty(self.npts, dtype=torch.float64).pin_memory())
        return hp, hp["x"].numel() * 8, hp["y"].numel() * 8

    def e2e_step(self, hp, d):
        import torch
        d["x"].copy_(hp["x"], non_blocking=True)
        self.step(d)
        hp["y"].copy_(d["y"], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    def oracle_units(self, h, budget_s, seed=0):
        """The oracle's matvec needs the oracle's generators: one block's C-A per
        far block, so the bounded sample is the generators of as many blocks as
        fit in the budget, scaled to one matvec's share (matvec/s of the full
        pipeline on the host: generators + products)."""
        import oracle
        far, p = h["far"], h["p"]
        order = np.random.default_rng(seed).permutation(len(far))
        t0 = time.perf_counter()
        n = 0
        for idx in order:
            r0, nr, c0, nc = (int(v) for v in far[idx, :4])
            sub = li.Problem(li.SRC_LAPLACE, nr, nc, X=p.X[r0:r0 + nr], Y=p.X[c0:c0 + nc])
            o = oracle.ca_run_adaptive(sub, (28, 40, 64), 2, 3, h["I0"][idx], h=1.05, rank_tol=1e-6)
            _ = o["C"] @ (o["U"] @ (o["R"] @ h["x"][c0:c0 + nc]))
            n += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        frac = n / len(far)
        return frac, n, el, (f"generators and products of {n} of the {len(far)} far blocks (near field not "
                             f"included): {frac:.4f} of one matvec")


class Hmt11Workload:
    """The single-layer Laplacian inputs of the bidiagonal pre-processing tests
    (inputs (i), [HMT11, Section 7.1]): n x n dense FP64, pre-processed by the
    product of q = 20 random bidiagonal factors, C-A with five loops (Tests 2).
    One step = ``runs`` independent LRAs (each its own multiplier draw and
    initial rows, as the paper's mean/std over trials) plus the exact Frobenius
    error of each (the residual over all n^2 entries).

    ``materialize`` (default): the paper's order of work -- every W'_r = W M_r
    is written out (lra_multiplier_apply, bit-identical entries), the runs go
    as blocks of one batched C-A launch over the stacked W'_r, and R_r = W[I_r, :]
    is gathered from W (lra_gather_rows).  Otherwise each run is one lra_ca_run
    on (W, M_r) forming the entries of W' inside the strips."""
    unit = "LRA/s"

    def __init__(self, n=1024, k=39, q=20, runs=10, sweeps=5, materialize=True):
        self.n, self.k, self.q, self.runs, self.sweeps, self.mat = n, k, q, runs, sweeps, materialize
        self.name = f"hmt11_laplacian{n}_bidiag{q}_k{k}_s{sweeps}_x{runs}" + ("" if materialize else "_onthefly")
        self.kernel = "apply_dense_kernel" if materialize else "ca_kernel"

    def host(self, rank):
        p = li.hmt11_laplacian(self.n)
        mults = []
        for r in range(self.runs):
            pr = li.Problem(li.SRC_DENSE, self.n, self.n, W=p.W)
            li.with_bidiag(pr, self.q, 100 + 1000 * rank + r)
            mults.append((pr.perm, pr.dsign))
        I0 = [li.initial_rows(self.n, self.k, 7 + 1000 * rank + r) for r in range(self.runs)]
        # nonzeros of each multiplier column (integer arithmetic on the factors) for the flop count
        nnz = []
        for perm, sg in mults:
            M = np.eye(self.n, dtype=np.int64)
            for f in range(self.q):
                b = perm[f].astype(np.int64)
                b1 = (b + 1) % self.n
                M = M[:, b] + M[:, b1] * sg[f][b1].astype(np.int64)[None, :]
            nnz.append(float((M != 0).sum(axis=0).mean()))
        return dict(p=p, mults=mults, I0=I0, nnz=float(np.mean(nnz)))

    def config(self, h):
        return {"workload": self.name, "m": self.n, "n": self.n, "k": self.k, "sweeps": self.sweeps,
                "multiplier": f"product of {self.q} cyclic bidiagonal +-1 factors (every column dense)",
                "runs_per_step": self.runs, "input_dtype": "f64",
                "form": ("W' = W M written out, runs batched (one CTA each), R from W" if self.mat
                         else "entries of W' formed inside the C-A strips, one run at a time"),
                "residual_sample": f"all {self.n}x{self.n} entries (exact Frobenius ratio)"}

    def device(self, h, dev):
        import torch
        import paper_1710_07946_gb300 as lra
        n, k = self.n, self.k
        W = torch.from_numpy(h["p"].W).to(dev)
        prob = lra.Problem.dense(W)
        mults = [lra.lra_precondition("bidiag", n, self.q, perm, sg) for perm, sg in h["mults"]]
        QS = torch.arange(n, dtype=torch.int32, device=dev)
        d = dict(W=W, prob=prob, mults=mults, Q=QS, S=QS, stats=[None] * self.runs)
        if self.mat:
            Wp = torch.empty(self.runs * n, n, dtype=torch.float64, device=dev)
            blocks = np.array([[r * n, n, 0, n] for r in range(self.runs)], dtype=np.int64)
            bt = lra.Batch(lra.Problem.dense(Wp), blocks, k, self.sweeps, np.stack(h["I0"]), rank_tol=1e-13,
                           order=None)
            views = []
            for r in range(self.runs):
                oc, orr = (int(x) for x in bt.offs_np[r])
                views.append(dict(C=bt.out["C"][oc:oc + n * k].view(n, k), U=bt.out["U"][r],
                                  R=bt.out["R"][orr:orr + k * n].view(k, n), I=bt.out["I"][r]))
            d.update(Wp=Wp, bt=bt, views=views)
        else:
            I0 = [torch.from_numpy(x).to(dev) for x in h["I0"]]
            outs = [lra.lra_ca_run(prob, I0[r], k, self.sweeps, multiplier=mults[r]) for r in range(self.runs)]
            d.update(I0=I0, outs=outs)
        return d

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        n = self.n
        if self.mat:
            for r in range(self.runs):
                lra.lra_multiplier_apply(d["prob"], d["mults"][r], d["Wp"][r * n:(r + 1) * n])
            lra.lra_ca_run_batched(d["bt"])
            for r, v in enumerate(d["views"]):
                lra.lra_gather_rows(d["prob"], v["I"], out=v["R"])
                d["stats"][r] = lra.lra_residual_sample(d["prob"], v["C"], v["U"], v["R"], d["Q"], d["S"])
            return
        for r in range(self.runs):
            o = d["outs"][r]
            lra.lra_ca_run(d["prob"], d["I0"][r], self.k, self.sweeps, multiplier=d["mults"][r], out=o,
                           workspace=o["_workspace"])
            d["stats"][r] = lra.lra_residual_sample(d["prob"], o["C"], o["U"], o["R"], d["Q"], d["S"])

    def _infos(self, d):
        if self.mat:
            return d["bt"].out["info"].cpu().numpy()
        return np.stack([o["info"].cpu().numpy() for o in d["outs"]])

    def check(self, d):
        info = self._infos(d)
        err = np.array([float(st[4].item()) for st in d["stats"]])
        return dict(units=int((err <= ERR_BOUND).sum()), info=info, err=err)

    def flops(self, h, res):
        if self.mat:      # one W' = W M per launch: n^2 entries of nnz fused multiply-adds each
            return 2.0 * self.n * self.n * h["nnz"]
        f = [ca_flops(self.k, self.n, self.n, int(inf[2]), int(inf[1]), 2.0 * h["nnz"], nucleus=False)
             for inf in res["info"]]
        return float(np.mean(f))

    def extra(self, res):
        return {"rel_fro_err_mean": float(np.mean(res["err"])), "rel_fro_err_std": float(np.std(res["err"])),
                "rel_fro_err_max": float(np.max(res["err"])), "swaps_mean": float(np.mean(res["info"][:, 1])),
                "statuses": sorted(set(int(x) for x in res["info"][:, 3])),
                "flops_note": ("per launch of the dominant kernel: 2 x n^2 x mean nonzeros of a multiplier column"
                               if self.mat else "entry cost = 2 x mean nonzeros per multiplier column")}

    def e2e_setup(self, h, d):
        import torch
        hp = dict(W=torch.from_numpy(h["p"].W).pin_memory())
        if self.mat:
            hp["out"] = {key: torch.empty(v.shape, dtype=v.dtype).pin_memory() for key, v in d["bt"].out.items()}
        else:
            hp["out"] = {f"{r}_{key}": torch.empty(v.shape, dtype=v.dtype).pin_memory()
                         for r, o in enumerate(d["outs"]) for key, v in o.items() if not key.startswith("_")}
        hp["stats"] = torch.empty(self.runs, 5, dtype=torch.float64).pin_memory()
        h2d = hp["W"].numel() * 8
        d2h = sum(v.numel() * v.element_size() for v in hp["out"].values()) + 40 * self.runs
        return hp, h2d, d2h

    def e2e_step(self, hp, d):
        import torch
        d["W"].copy_(hp["W"], non_blocking=True)
        self.step(d)
        for key, v in hp["out"].items():
            if self.mat:
                v.copy_(d["bt"].out[key], non_blocking=True)
            else:
                r, name = key.split("_", 1)
                v.copy_(d["outs"][int(r)][name], non_blocking=True)
        for r in range(self.runs):
            hp["stats"][r].copy_(d["stats"][r], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        t0 = time.perf_counter()
        n = good = 0
        QS = np.arange(self.n, dtype=np.int32)
        for r in range(self.runs):
            pr = li.Problem(li.SRC_DENSE, self.n, self.n, W=h["p"].W)
            perm, sg = h["mults"][r]
            pr.mkind, pr.depth, pr.perm, pr.dsign = li.MULT_BIDIAG, self.q, perm, sg
            o = oracle.ca_run(pr, self.k, self.sweeps, h["I0"][r])
            st = oracle.residual_sample(h["p"], o["C"], o["U"], o["R"], QS, QS)
            n += 1
            good += st[4] <= ERR_BOUND
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        return good, n, el, f"{n} complete LRAs (C-A + nucleus + exact residual) of the step's {self.runs}"


class LaplaceSingleWorkload:
    """One C-A CUR of the 65536 x 65536 Laplace kernel between two unit cubes whose
    centres are 3 apart, entries evaluated on the fly (FP64 or FP32), rank k,
    3 loops, FP64 pivots and nucleus, on the whole GPU (cooperative grid)."""
    kernel = "ca_kernel"
    unit = "LRA/s"

    def __init__(self, k, entries="f64", n=65536, sweeps=3, rank_tol=1e-8):
        self.k, self.entries, self.n, self.sweeps, self.q, self.s = k, entries, n, sweeps, 256, 256
        self.rank_tol = rank_tol          # truncation above the core's rounding level
        self.name = f"laplace{n}_cubes3apart_k{k}_s{sweeps}_{entries}entries"

    def host(self, rank):
        p = li.laplace_clusters(self.n, self.n, seed=1 + 1000 * rank)
        I0 = li.initial_rows(self.n, self.k, 0)
        Q, S = li.sample_positions(self.n, self.n, self.q, self.s, 13)
        return dict(p=p, I0=I0, Q=Q, S=S)

    def config(self, h):
        return {"workload": self.name, "m": self.n, "n": self.n, "k": self.k, "sweeps": self.sweeps,
                "kernel": f"Laplace 1/|x-y|, on the fly, entries {self.entries.upper()}",
                "pivots_nucleus": "FP64", "rank_tol": self.rank_tol,
                "residual_sample": f"{self.q}x{self.s} against FP64 entries"}

    def device(self, h, dev):
        import torch
        import paper_1710_07946_gb300 as lra
        p = h["p"]
        X, Y = torch.from_numpy(p.X).to(dev), torch.from_numpy(p.Y).to(dev)
        prob = lra.Problem.kernel("laplace", X, Y, entries=self.entries)
        prob64 = lra.Problem.kernel("laplace", X, Y)
        I0 = torch.from_numpy(h["I0"]).to(dev)
        out = lra.lra_ca_run(prob, I0, self.k, self.sweeps, rank_tol=self.rank_tol)
        return dict(X=X, Y=Y, prob=prob, prob64=prob64, I0=I0, out=out, Q=torch.from_numpy(h["Q"]).to(dev),
                    S=torch.from_numpy(h["S"]).to(dev), stats=None)

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        lra.lra_ca_run(d["prob"], d["I0"], self.k, self.sweeps, rank_tol=self.rank_tol, out=d["out"],
                       workspace=d["out"]["_workspace"])
        d["stats"] = lra.lra_residual_sample(d["prob64"], d["out"]["C"], d["out"]["U"], d["out"]["R"], d["Q"],
                                             d["S"])

    def check(self, d):
        info = d["out"]["info"].cpu().numpy()[None, :]
        err = d["stats"].cpu().numpy()[4:5]
        ok = (info[0, 3] == 0 or info[0, 3] >= 16) and err[0] <= ERR_BOUND
        return dict(units=int(ok), info=info, err=err)

    def flops(self, h, res):
        inf = res["info"][0]
        return ca_flops(self.k, self.n, self.n, max(int(inf[2]), 1), int(inf[1]), LAPLACE_FLOPS, nucleus=False)

    def extra(self, res):
        inf = res["info"][0]
        return {"rank": int(inf[0]), "swaps": int(inf[1]), "loops": int(inf[2]), "status": int(inf[3]),
                "rel_fro_err_sampled": float(res["err"][0])}

    def e2e_setup(self, h, d):
        import torch
        hp = dict(X=torch.from_numpy(h["p"].X).pin_memory(), Y=torch.from_numpy(h["p"].Y).pin_memory(),
                  I0=torch.from_numpy(h["I0"]).pin_memory())
        hp["out"] = {key: torch.empty(v.shape, dtype=v.dtype).pin_memory() for key, v in d["out"].items()
                     if not key.startswith("_")}
        hp["stats"] = torch.empty(5, dtype=torch.float64).pin_memory()
        h2d = (hp["X"].numel() + hp["Y"].numel()) * 8 + hp["I0"].numel() * 4
        d2h = sum(v.numel() * v.element_size() for v in hp["out"].values()) + 40
        return hp, h2d, d2h

    def e2e_step(self, hp, d):
        import torch
        d["X"].copy_(hp["X"], non_blocking=True)
        d["Y"].copy_(hp["Y"], non_blocking=True)
        d["I0"].copy_(hp["I0"], non_blocking=True)
        self.step(d)
        for key, v in hp["out"].items():
            v.copy_(d["out"][key], non_blocking=True)
        hp["stats"].copy_(d["stats"], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        p = h["p"]
        pe = li.Problem(li.SRC_LAPLACE, p.m, p.n, X=p.X, Y=p.Y, entries=self.entries)
        t0 = time.perf_counter()
        n = good = 0
        while True:
            o = oracle.ca_run(pe, self.k, self.sweeps, h["I0"], rank_tol=self.rank_tol)
            st = oracle.residual_sample(p, o["C"], o["U"], o["R"], h["Q"], h["S"])
            n += 1
            good += st[4] <= ERR_BOUND
            if time.perf_counter() - t0 >= budget_s or n >= 50:
                break
        el = time.perf_counter() - t0
        return good, n, el, f"{n} complete LRAs of the same input (C-A + nucleus + residual sample)"


class RandomTestsWorkload:
    """The paper's random-input tests (Table tb_ranrc recipe): nb independent n x n
    inputs W = G1 G2 + 1e-10 G3 of expected rank r, stacked as blocks of one
    matrix, each approximated by Tests 2 (C-A, r x r generators, 5 loops from r
    random rows), Tests 3 (an r x r generator inside a random 4r x 4r sketch) or
    Tests 4 (one C-A loop with 4r x 4r generators from 4r random columns, then
    Tests 3 inside it).  One step = the batched run + a 16 x 16 residual sample
    per block; units = blocks whose sampled error is <= 1e-6."""
    unit = "LRA/s"

    def __init__(self, test, n=256, r=8, nb=4096, sweeps=5):
        self.test, self.n, self.r, self.nb, self.sweeps, self.q = test, n, r, nb, sweeps, 4 * r
        self.kernel = "ca_batched_kernel" if test == 2 else "cynical_batched_kernel"
        self.name = f"tests{test}_factor_gaussian_{nb}x{n}x{n}_r{r}"

    def host(self, rank):
        g = np.random.default_rng(4000 + rank)
        n, r, nb = self.n, self.r, self.nb
        W = np.empty((nb * n, n))
        for b in range(nb):
            W[b * n:(b + 1) * n] = g.standard_normal((n, r)) @ g.standard_normal((r, n))
        W += 1e-10 * g.standard_normal(W.shape)
        blocks = np.array([[b * n, n, 0, n] for b in range(nb)], dtype=np.int64)
        K = np.stack([g.choice(n, self.q, replace=False) for _ in range(nb)]).astype(np.int32)
        L = np.stack([g.choice(n, self.q, replace=False) for _ in range(nb)]).astype(np.int32)
        I0s = np.stack([g.choice(self.q, r, replace=False) for _ in range(nb)]).astype(np.int32)
        I0 = np.stack([g.choice(n, r, replace=False) for _ in range(nb)]).astype(np.int32)
        Q, S = li.block_sample_positions(blocks, 16, 16, 300 + rank)
        return dict(W=W, blocks=blocks, K=K, L=L, I0s=I0s, I0=I0, Q=Q, S=S)

    def config(self, h):
        alg = {2: "C-A (Tests 2): r x r generators, 5 loops from r random rows",
               3: "cynical (Tests 3): r x r generator in a random 4r x 4r sketch, sketch C-A 5 loops",
               4: "Tests 4: one C-A loop with 4r x 4r generators from 4r random columns, then Tests 3"}[self.test]
        return {"workload": self.name, "inputs": f"{self.nb} x (G1 G2 + 1e-10 G3), n = {self.n}, r = {self.r}",
                "algorithm": alg, "sketch": self.q if self.test > 2 else None, "residual_sample": "16x16 per block"}

    def device(self, h, dev):
        import torch
        import paper_1710_07946_gb300 as lra
        W = torch.from_numpy(h["W"]).to(dev)
        prob = lra.Problem.dense(W)
        I0 = h["I0"] if self.test == 2 else h["I0s"]
        bt = lra.Batch(prob, h["blocks"], self.r, self.sweeps, I0, rank_tol=1e-13)
        t = lambda a: torch.from_numpy(a).to(dev)
        d = dict(W=W, prob=prob, bt=bt, K=t(h["K"]), L=t(h["L"]), L0=t(h["L"]), I0s=t(h["I0s"]), Q=t(h["Q"]),
                 S=t(h["S"]))
        d["stats"] = torch.empty(self.nb, 5, dtype=torch.float64, device=dev)
        # untimed set-up: CTA shape autotuner (Tests 4 rewrites its inputs: library default shape)
        if self.test == 2:
            tuned = lra.lra_ca_batched_tune(bt, reps=2)
        elif self.test == 3:
            tuned = lra.lra_cynical_batched_tune(bt, self.q, d["K"], d["L"], d["I0s"], reps=2)
        else:
            tuned = None
        self.tuned = None if tuned is None else {
            "chosen": f"{bt.cb.cta_threads}x{bt.cb.ctas_per_sm}",
            "ms": {f"{a}x{b}": round(v, 3) for (a, b), v in tuned.items()}}
        return d

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        if self.test == 2:
            lra.lra_ca_run_batched(d["bt"])
        else:
            if self.test == 4:
                d["L"].copy_(d["L0"])          # Tests 4 overwrites the sketch sets
            lra.lra_cynical_run_batched(d["bt"], self.test - 3, self.q, d["K"], d["L"], d["I0s"])
        lra.lra_residual_sample_batched(d["bt"], d["Q"], d["S"], d["stats"])

    def check(self, d):
        info = d["bt"].out["info"].cpu().numpy()
        st = d["stats"].cpu().numpy()
        ok = ((info[:, 3] == 0) | (info[:, 3] >= 16)) & (st[:, 4] <= ERR_BOUND)
        return dict(units=int(ok.sum()), info=info, err=st[:, 4])

    def flops(self, h, res):
        n, r, q = self.n, self.r, self.q
        f = 0.0
        for inf in res["info"]:
            loops, swaps = max(int(inf[2]), 1), int(inf[1])
            if self.test == 2:
                f += ca_flops(r, n, n, loops, swaps)
            else:
                f += ca_flops(r, q, q, loops, swaps)
                if self.test == 4:
                    f += maxvol_flops(q, n, True) * 2
        return f

    def extra(self, res):
        err = res["err"]
        return {"cta_shape_tuner": getattr(self, "tuned", None),
                "swaps_mean": float(res["info"][:, 1].mean()), "loops_mean": float(res["info"][:, 2].mean()),
                "rel_fro_err_sampled_median": float(np.median(err)), "rel_fro_err_sampled_max": float(err.max()),
                "frac_blocks_err_le_1e-6": float((err <= ERR_BOUND).mean())}

    # end to end: the stacked inputs uploaded, every block's factors and statistics read back, every step,
    # through a two-slot pipeline (TwoSlotPipe); slot 1 has its own input copy, batch and statistics
    def e2e_setup(self, h, d):
        import torch
        import paper_1710_07946_gb300 as lra
        W1 = d["W"].clone()
        prob1 = lra.Problem.dense(W1)
        bt1 = lra.Batch(prob1, h["blocks"], self.r, self.sweeps, h["I0"] if self.test == 2 else h["I0s"],
                        rank_tol=1e-13)
        bt1.cb.cta_threads, bt1.cb.ctas_per_sm = d["bt"].cb.cta_threads, d["bt"].cb.ctas_per_sm
        d1 = dict(d, W=W1, prob=prob1, bt=bt1, stats=torch.empty_like(d["stats"]))
        self.step(d1)                         # sizes slot 1's workspaces (untimed)
        torch.cuda.synchronize()
        hp = dict(pipe=TwoSlotPipe(d["W"].device), W=torch.from_numpy(h["W"]).pin_memory(), slots=[d, d1])
        hp["out"] = [{key: torch.empty(v.shape, dtype=v.dtype).pin_memory() for key, v in d["bt"].out.items()}
                     for _ in range(2)]
        hp["stats"] = [torch.empty(d["stats"].shape, dtype=torch.float64).pin_memory() for _ in range(2)]
        h2d = hp["W"].numel() * 8
        d2h = sum(v.numel() * v.element_size() for v in hp["out"][0].values()) + hp["stats"][0].numel() * 8
        return hp, h2d, d2h

    def e2e_step(self, hp, d):
        pipe = hp["pipe"]
        i = pipe.next_slot()
        ds = hp["slots"][i]
        pipe.upload(i, [(ds["W"], hp["W"])])
        self.step(ds)
        pipe.download(i, [(v, ds["bt"].out[key]) for key, v in hp["out"][i].items()] +
                      [(hp["stats"][i], ds["stats"])])

    def e2e_finish(self, hp, d):
        hp["pipe"].finish()

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        n, r = self.n, self.r
        t0 = time.perf_counter()
        cnt = good = 0
        for b in np.random.default_rng(seed).permutation(self.nb):
            sub = li.Problem(li.SRC_DENSE, n, n, W=np.ascontiguousarray(h["W"][b * n:(b + 1) * n]))
            if self.test == 2:
                o = oracle.ca_run(sub, r, self.sweeps, h["I0"][b])
            else:
                o = oracle.cynical(sub, self.test - 3, r, self.q, h["K"][b] if self.test == 3 else None, h["L"][b],
                                   h["I0s"][b], sweeps=self.sweeps)
            st = oracle.residual_sample(sub, o["C"], o["U"], o["R"], h["Q"][b], h["S"][b])
            cnt += 1
            good += st[4] <= ERR_BOUND
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        return good, cnt, el, f"{cnt} randomly chosen inputs of the same batch (LRA + residual sample each)"


class GaussApplyWorkload:
    """Differentiable CUR apply: 256 Gaussian-kernel blocks exp(-|x-y|^2/(2 l^2)), l = 0.3, 1024 x 1024 each
    (targets in [0,1]^3, sources in [2,3]x[0,1]^2), pivots of rank 32 from a batched C-A run (untimed set-up);
    one step = forward y = C U R x and the hand-written backward (dx, dl) for nrhs FP32 right-hand sides."""
    kernel = "gauss_bwd_kernel"
    unit = "blocks/s"
    peak_name = "fp32"

    def __init__(self, nblk=256, size=1024, k=32, nrhs=64):
        self.nblk, self.size, self.k, self.nrhs = nblk, size, k, nrhs
        self.name = f"gauss_apply_{nblk}blocks_{size}_k{k}_nrhs{nrhs}_fwd_bwd"

    def host(self, rank):
        X, Y, ell = li.gaussian_blocks(nblk=self.nblk, size=self.size, ell=0.3, seed=rank)
        g = np.random.default_rng(50 + rank)
        x = g.standard_normal((self.nblk, self.size, self.nrhs)).astype(np.float32)
        dy = g.standard_normal((self.nblk, self.size, self.nrhs)).astype(np.float32)
        return dict(X=X, Y=Y, ell=ell, x=x, dy=dy)

    def config(self, h):
        return {"workload": self.name, "blocks": self.nblk, "block": f"{self.size}x{self.size}", "k": self.k,
                "nrhs": self.nrhs, "kernel": "Gaussian l=0.3, entries on the fly in FP32, core inverse FP64",
                "pivots": "batched C-A (FP64), untimed set-up"}

    def device(self, h, dev):
        import torch
        import paper_1710_07946_gb300 as lra
        nb, sz, k = self.nblk, self.size, self.k
        Xall = torch.from_numpy(np.ascontiguousarray(h["X"].reshape(-1, 3))).to(dev)
        Yall = torch.from_numpy(np.ascontiguousarray(h["Y"].reshape(-1, 3))).to(dev)
        prob = lra.Problem.kernel("gaussian", Xall, Yall, h["ell"])
        blocks = np.array([[b * sz, sz, b * sz, sz] for b in range(nb)], dtype=np.int64)
        bt = lra.Batch(prob, blocks, k, 3, li.block_initial_rows(blocks, k, 3), rank_tol=1e-13)
        lra.lra_ca_run_batched(bt)
        torch.cuda.synchronize()
        d = dict(X=Xall.view(nb, sz, 3), Y=Yall.view(nb, sz, 3), I=bt.out["I"].contiguous(),
                 J=bt.out["J"].contiguous(), ell=h["ell"], x=torch.from_numpy(h["x"]).to(dev),
                 dy=torch.from_numpy(h["dy"]).to(dev))
        d["pivots"] = (d["I"].cpu().numpy(), d["J"].cpu().numpy())
        return d

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        y, ctx = lra.lra_gauss_cur_forward(d["X"], d["Y"], d["I"], d["J"], d["ell"], d["x"])
        g = lra.lra_gauss_cur_backward(d["X"], d["Y"], d["I"], d["J"], d["ell"], d["x"], d["dy"], ctx)
        d["y"], d["dx"], d["dell"] = y, g["dx"], g["dell"]

    def check(self, d):
        ok = bool(np.isfinite(d["dell"].cpu().numpy()).all())
        return dict(units=self.nblk if ok else 0, dell=float(d["dell"].sum().item()))

    def flops(self, h, res):
        """FP32 flops per backward launch: entries (exp, distance: ~12 flops) and the fused products."""
        m = n = self.size
        k, r = self.k, self.nrhs
        per_block = (m * k + k * n) * (12 + 2 * r) + 2 * (m * k * r + k * n * r)
        return float(self.nblk * per_block)

    def extra(self, res):
        return {"dl_sum": res["dell"]}

    # end to end: x and dy uploaded from pinned host memory, y, dx and dl read back, every step.  Served as a
    # two-slot pipeline: step i's inputs are uploaded on one copy stream while step i - 1 computes, and its
    # results are read back on another while step i + 1 computes; a slot's inputs are overwritten only after
    # the compute that read them, and the clock stops after the last read-back.
    def e2e_setup(self, h, d):
        import torch
        dev = d["x"].device
        hp = dict(x=torch.from_numpy(h["x"]).pin_memory(), dy=torch.from_numpy(h["dy"]).pin_memory(), slot=0,
                  up=torch.cuda.Stream(dev), down=torch.cuda.Stream(dev),
                  xs=[d["x"], torch.empty_like(d["x"])], dys=[d["dy"], torch.empty_like(d["dy"])],
                  uploaded=[torch.cuda.Event(), torch.cuda.Event()], done=[torch.cuda.Event(), torch.cuda.Event()])
        hp["dx"] = [torch.empty(d["x"].shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        hp["y"] = [torch.empty((self.nblk, self.size, self.nrhs), dtype=torch.float32).pin_memory()
                   for _ in range(2)]
        hp["dell"] = [torch.empty(self.nblk, dtype=torch.float64).pin_memory() for _ in range(2)]
        h2d = 2 * hp["x"].numel() * 4
        d2h = 2 * hp["dx"][0].numel() * 4 + self.nblk * 8
        return hp, h2d, d2h

    def e2e_step(self, hp, d):
        import torch
        import paper_1710_07946_gb300 as lra
        i = hp["slot"]
        hp["slot"] = 1 - i
        cur = torch.cuda.current_stream()
        with torch.cuda.stream(hp["up"]):
            hp["up"].wait_event(hp["done"][i])            # the compute that last read slot i has finished
            hp["xs"][i].copy_(hp["x"], non_blocking=True)
            hp["dys"][i].copy_(hp["dy"], non_blocking=True)
            hp["uploaded"][i].record(hp["up"])
        cur.wait_event(hp["uploaded"][i])
        x, dy = hp["xs"][i], hp["dys"][i]
        y, ctx = lra.lra_gauss_cur_forward(d["X"], d["Y"], d["I"], d["J"], d["ell"], x)
        g = lra.lra_gauss_cur_backward(d["X"], d["Y"], d["I"], d["J"], d["ell"], x, dy, ctx)
        hp["done"][i].record(cur)
        with torch.cuda.stream(hp["down"]):
            hp["down"].wait_event(hp["done"][i])
            hp["y"][i].copy_(y, non_blocking=True)
            hp["dx"][i].copy_(g["dx"], non_blocking=True)
            hp["dell"][i].copy_(g["dell"], non_blocking=True)
        for t in (y, g["dx"], g["dell"]):
            t.record_stream(hp["down"])                   # not reused before the read-back has run

    def e2e_finish(self, hp, d):
        hp["up"].synchronize()
        hp["down"].synchronize()

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        I, J = self._host_pivots
        t0 = time.perf_counter()
        n = 0
        for b in np.random.default_rng(seed).permutation(self.nblk):
            oracle.gauss_cur_backward(h["X"][b], h["Y"][b], I[b], J[b], h["ell"], h["x"][b].astype(np.float64),
                                      h["dy"][b].astype(np.float64))
            n += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        return n, n, el, f"{n} blocks of the same batch (FP64 forward + backward each)"


class FmmOversampleWorkload(FmmWorkload):
    """The FMM batch (mixed form) with every block's square generator grown to a
    rectangular k x (k + p) one by greedy volume expansions (Algorithm algrup);
    one step = the batched C-A launch + the batched expansion + the rectangular
    residual sample against the FP64 entries."""

    def __init__(self, pextra=8, pmax=0, max_cycles=32, **kw):
        super().__init__(entries="f32", **kw)
        self.pextra, self.pmax, self.max_cycles = pextra, pmax, max_cycles
        self.name = self.name + f"_oversample{pextra}" + (f"_cycles{pmax}" if pmax else "")

    def config(self, h):
        c = super().config(h)
        c["generator"] = f"rectangular k x (k + {self.pextra}) by greedy volume expansions"
        if self.pmax:
            c["generator"] += (f", then expansion/contraction cycles (p <= {self.pmax}, "
                               f"<= {self.max_cycles} kept)")
        return c

    def device(self, h, dev):
        import paper_1710_07946_gb300 as lra
        d = super().device(h, dev)
        d["ov"] = lra.Oversampled(d["bt"], self.pextra, self.pmax)
        return d

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        lra.lra_ca_run_batched(d["bt"])
        if self.pmax:
            lra.lra_oversample_cycle_batched(d["bt"], self.pextra, self.pmax, self.max_cycles, d["ov"])
        else:
            lra.lra_oversample_batched(d["bt"], self.pextra, d["ov"])
        lra.lra_residual_sample_oversampled(d["ov"], d["Q"], d["S"], d["stats"], problem=d["prob64"])

    def check(self, d):
        info = d["ov"].out["info"].cpu().numpy()
        st = d["stats"].cpu().numpy()
        ok = (info[:, 3] == 0) | (info[:, 3] >= 16)
        good = ok & (st[:, 4] <= ERR_BOUND)
        return dict(units=int(good.sum()), info=d["bt"].out["info"].cpu().numpy(), err=st[:, 4])

    def comparisons(self):
        return []

    def e2e_setup(self, h, d):
        import torch
        out = d["bt"].out
        hp = dict(X=torch.from_numpy(h["p"].X).pin_memory())
        hp["out"] = {key: torch.empty(v.shape, dtype=v.dtype).pin_memory() for key, v in out.items()}
        hp["stats"] = torch.empty(d["stats"].shape, dtype=torch.float64).pin_memory()
        h2d = hp["X"].numel() * 8
        d2h = sum(v.numel() * v.element_size() for v in hp["out"].values()) + hp["stats"].numel() * 8
        return hp, h2d, d2h

    def e2e_finish(self, hp, d):
        pass

    def e2e_step(self, hp, d):
        import torch
        d["X"].copy_(hp["X"], non_blocking=True)
        self.step(d)
        for key, v in hp["out"].items():
            v.copy_(d["bt"].out[key], non_blocking=True)
        hp["stats"].copy_(d["stats"], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        b = h["blocks"]
        order = np.random.default_rng(seed).permutation(len(b))
        t0 = time.perf_counter()
        n = good = 0
        for idx in order:
            r0, nr, c0, nc = b[idx]
            sub = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=h["p"].X[r0:r0 + nr], Y=h["p"].Y[c0:c0 + nc])
            sube = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=sub.X, Y=sub.Y, entries=self.entries)
            o = oracle.ca_run_adaptive(sube, self.stages, self.margin, self.sweeps, h["I0"][idx], h=self.h,
                                       rank_tol=self.tol)
            ov = oracle.oversample(sube, o["I"], o["J"], self.pextra, h=self.h, rank_tol=self.tol, pmax=self.pmax,
                                   max_cycles=self.max_cycles)
            st = oracle.residual_sample(sub, ov["C"], ov["U"], ov["R"], h["Q"][idx], h["S"][idx])
            n += 1
            good += st[4] <= ERR_BOUND
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        return good, n, el, f"{n} randomly chosen blocks of the same batch (C-A + expansion + residual sample each)"


class FmmPrjvolWorkload(FmmOversampleWorkload):
    """The FMM batch (mixed form) with every block's generator rebuilt as a
    k x (k + p) one of maximal r-projective volume in the row strip W'[I, :]
    (Algorithm algprjvlm: pivoted Householder QR to the numerical rank r,
    Algorithm alg1tor; dominance swaps on R'; greedy expansion, Algorithm
    algrup); one step = the batched C-A launch + the batched selection + the
    rectangular residual sample against the FP64 entries."""

    def __init__(self, pextra=8, **kw):
        super().__init__(pextra, **kw)
        self.name = self.name.replace(f"_oversample{pextra}", f"_prjvol{pextra}")

    def config(self, h):
        c = super().config(h)
        c["generator"] = (f"k x (k + {self.pextra}) of maximal r-projective volume: pivoted QR of W'[I, :] to the "
                          f"numerical rank r at rank_tol, dominance swaps on R' at h, greedy expansion")
        return c

    def device(self, h, dev):
        import paper_1710_07946_gb300 as lra
        d = FmmWorkload.device(self, h, dev)
        d["ov"] = lra.Oversampled(d["bt"], self.pextra, prjvol=True)
        return d

    def step(self, d):
        import paper_1710_07946_gb300 as lra
        lra.lra_ca_run_batched(d["bt"])
        lra.lra_prjvol_batched(d["bt"], self.pextra, d["ov"])
        lra.lra_residual_sample_oversampled(d["ov"], d["Q"], d["S"], d["stats"], problem=d["prob64"])

    def oracle_units(self, h, budget_s, seed=0):
        import oracle
        b = h["blocks"]
        order = np.random.default_rng(seed).permutation(len(b))
        t0 = time.perf_counter()
        n = good = 0
        for idx in order:
            r0, nr, c0, nc = b[idx]
            sub = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=h["p"].X[r0:r0 + nr], Y=h["p"].Y[c0:c0 + nc])
            sube = li.Problem(li.SRC_LAPLACE, int(nr), int(nc), X=sub.X, Y=sub.Y, entries=self.entries)
            o = oracle.ca_run_adaptive(sube, self.stages, self.margin, self.sweeps, h["I0"][idx], h=self.h,
                                       rank_tol=self.tol)
            pv = oracle.prjvol(sube, o["I"], o["J"], self.pextra, h=self.h, rank_tol=self.tol)
            st = oracle.residual_sample(sub, pv["C"], pv["U"], pv["R"], h["Q"][idx], h["S"][idx])
            n += 1
            good += st[4] <= ERR_BOUND
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        return good, n, el, f"{n} randomly chosen blocks of the same batch (C-A + selection + residual sample each)"


class FmmSmallPrjvolWorkload(FmmPrjvolWorkload):
    """fmm_prjvol8's recipe on 2^17 points and 512 block pairs (profiling size)."""
    base = "fmm_laplace_128K_octree_512blocks"

    def __init__(self):
        super().__init__(8, npts=1 << 17, nblocks=512)


class FmmSmallWorkload(FmmWorkload):
    """The headline recipe (mixed form) on 2^17 points and 512 block pairs (profiling size), in the CTA shape the
    headline batch's tuner picks (256 x 2, its large blocks on CTA pairs): the small batch's own tuner prefers
    512 x 1, its few large blocks setting its end."""
    base = "fmm_laplace_128K_octree_512blocks"
    cta_shape = (256, 2)

    def __init__(self):
        super().__init__(npts=1 << 17, nblocks=512, entries="f32")

    def comparisons(self):
        return []


WORKLOADS = {
    "fmm": lambda: FmmWorkload(entries="f32"),
    "fmm_f64": FmmWorkload,
    "fmm_fixedk": lambda: FmmWorkload(stages=None),
    "fmm_bf16entries": lambda: FmmWorkload(entries="bf16"),
    "fmm_oversample8": lambda: FmmOversampleWorkload(8),
    "fmm_oversample8_cycles4": lambda: FmmOversampleWorkload(8, pmax=4),
    "fmm_prjvol8": lambda: FmmPrjvolWorkload(8),
    "fmm_small_prjvol8": FmmSmallPrjvolWorkload,
    "fmm_small": FmmSmallWorkload,
    "hmt11_n1024_k39_bidiag20": Hmt11Workload,
    "rhtcur_dense8192_k48": RhtcurWorkload,
    "levca_n1000_r10_k40": LevCaWorkload,
    "hmatvec_laplace_64K": HMatvecWorkload,
    "hmatvec_laplace_8K": lambda: HMatvecWorkload(npts=1 << 13),
    "hmatvec_laplace_1M_matrixfree": lambda: HMatvecWorkload(npts=1 << 20, leaf=1024, matrix_free=True,
                                                             entries="f32", max_block=8192),
    "levca_n1000_r10_k40_expected": lambda: LevCaWorkload(kind=1),
    "levca_n1000_r10_k40_uniform": lambda: LevCaWorkload(kind=2),
    "hmt11_n1024_k39_bidiag20_onthefly": lambda: Hmt11Workload(materialize=False),
    "hmt11_n256_k31_bidiag20": lambda: Hmt11Workload(n=256, k=31),
    **{f"laplace65536_k{k}{sfx}": (lambda k=k, e=e: LaplaceSingleWorkload(k, e))
       for k in (16, 32, 64) for sfx, e in (("", "f64"), ("_f32", "f32"))},
    "gauss_apply": GaussApplyWorkload,
    "tests2_n256_r8": lambda: RandomTestsWorkload(2),
    "tests3_n256_r8": lambda: RandomTestsWorkload(3),
    "tests4_n256_r8": lambda: RandomTestsWorkload(4),
    "tests3_n256_r16": lambda: RandomTestsWorkload(3, r=16),
    "tests4_n256_r16": lambda: RandomTestsWorkload(4, r=16),
    "tests2_n256_r16": lambda: RandomTestsWorkload(2, r=16),
    "dense8192_arht": lambda: DenseWorkload("arht"),
    "dense8192_sparse": lambda: DenseWorkload("sparse"),
    "dense8192_bidiag": lambda: DenseWorkload("bidiag"),
    "dense8192_arft": lambda: DenseWorkload("arft"),
    **{f"cur_apply_{dt}": (lambda dt=dt: CurApplyWorkload(dt)) for dt in ("f64", "f32", "bf16")},
}


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def csrc_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1710_07946_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` from a committed ncu summary taken on the
    current sources (profiles/<kernel>__<workload>.txt lines 'csrc_hash: ...' and
    'dram_bytes_per_launch: ...'); None otherwise."""
    path = os.path.join(ROOT, "profiles", f"{kernel}__{workload}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line:
            a, b = line.split(":", 1)
            kv[a.strip()] = b.strip()
    if kv.get("csrc_hash") != csrc_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_cores_used() -> int:
    return 1


# ------------------------------------------------------------------ arms
def job_totals(elapsed, units, world, device):
    """Whole-job figures of a weak-scaling run: the slowest rank's elapsed time
    and the units of all ranks (each rank runs its own independent problem; this
    is the only exchange, outside the timed region)."""
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    h = wl.host(0)
    per_step = max(args.ref_budget / max(args.steps + args.warmup, 1), 0.5)
    for w in range(args.warmup):
        wl.oracle_units(h, per_step, seed=w)
    good = n = 0
    el = 0.0
    for s in range(args.steps):
        g, c, e, desc = wl.oracle_units(h, per_step, seed=100 + s)
        good += g
        n += c
        el += e
    v = good / el
    line = {"metric": METRIC, "value": v, "unit": wl.unit, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": wl.config(h),
            "cpu_baseline": {"value": v, "unit": wl.unit, "cores": cpu_cores_used(), "kind": "oracle",
                             "sample": f"{args.steps} steps of ~{per_step:.1f} s, each: " + desc},
            "e2e": {"value": v, "unit": wl.unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_lib(args, wl):
    import torch
    import torch.distributed as dist
    import paper_1710_07946_gb300 as lra

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    wl.world, wl.shard = world, args.shard
    wl.tune_stages = args.tune_stages
    h = wl.host(rank)
    d = wl.device(h, dev)
    if "pivots" in d:
        wl._host_pivots = d["pivots"]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    warm = max(args.warmup, 3)
    for _ in range(warm):
        wl.step(d)
    torch.cuda.synchronize()
    l0 = lra.lra_launch_count()
    wl.step(d)
    torch.cuda.synchronize()
    launches_per_step = lra.lra_launch_count() - l0

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = lra.lra_launch_count()
    lra.lra_profile_enable(True)
    units = 0
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        wl.step(d)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    lra.lra_profile_enable(False)
    launches = lra.lra_launch_count() - launches0
    prof = lra.lra_profile_collect()
    res = wl.check(d)
    units = res["units"] * args.steps
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    total_ms, job_units = job_totals(step_ms, units, world, dev)
    value = job_units / (total_ms / 1e3)

    # the same step replayed from a CUDA graph (cross-check of launch overhead)
    graph_ms = None
    try:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(dev)
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            wl.step(d)
        stream.wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            wl.step(d)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gsum = 0.0
        for i in range(args.steps):
            flush.fill_(float(i))
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            gsum += e0.elapsed_time(e1)
        graph_ms = gsum / args.steps
        del g
    except Exception as exc:  # graph capture is a cross-check only
        graph_ms = f"capture failed: {type(exc).__name__}"

    # end to end through the public API from pinned host buffers
    hp, h2d, d2h = wl.e2e_setup(h, d)
    for _ in range(max(warm, 2)):      # untimed: every slot of the two-slot pipelines used once
        wl.e2e_step(hp, d)
    if hasattr(wl, "e2e_finish"):
        wl.e2e_finish(hp, d)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        wl.e2e_step(hp, d)
    if hasattr(wl, "e2e_finish"):
        wl.e2e_finish(hp, d)          # the last steps' results are on the host before the clock stops
    e2e_s, _ = job_totals(time.perf_counter() - t0, 0, world, dev)
    e2e_value = job_units / e2e_s

    # comparison forms of the same problem (each rank its own; rank 0 reports)
    comparisons = {}
    for label, other in (wl.comparisons() if hasattr(wl, "comparisons") else []):
        d2 = other.device(h, dev)
        for _ in range(warm):
            other.step(d2)
        torch.cuda.synchronize()
        nst = args.steps                 # the same number of timed steps as this line
        ms2 = 0.0
        for i in range(nst):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            other.step(d2)
            e1.record(stream)
            e1.synchronize()
            ms2 += e0.elapsed_time(e1)
        r2 = other.check(d2)
        v2 = r2["units"] * nst / (ms2 / 1e3)
        comparisons[label] = {"workload": other.name, "value": v2, "ms_per_step": ms2 / nst, "steps": nst,
                              "rel_fro_err_sampled_max": float(np.max(r2["err"])),
                              "frac_blocks_err_le_1e-6": float(np.mean(r2["err"] <= ERR_BOUND)),
                              "speedup_of_this_line": None}
        del d2
    if rank == 0:
        peaks = load_peaks()
        bound, runit = "alu", "TFLOP/s"
        if hasattr(wl, "counts"):
            # per-kernel (bound, algorithmic amount per launch); the dominant kernel is the one with the most time
            counts = wl.counts(h, res)
            wl.kernel = max(counts, key=lambda kname: prof.get(kname, (0.0, 0))[0])
            bound, amount = counts[wl.kernel]
        kms, kn = prof.get(wl.kernel, (float("nan"), 0))
        kavg = kms / max(kn, 1) / 1e3
        flops = amount if bound == "hbm" else (amount if hasattr(wl, "counts") else wl.flops(h, res))
        fp32 = getattr(wl, "peak_name", "fp64") == "fp32"
        if bound == "hbm":
            achieved, peak, runit = flops / kavg / 1e9, float(peaks.get("hbm_gbs") or 6800.0), "GB/s"
            peak_src = ("measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peaks.get("hbm_gbs") else
                        "fallback 6.8 TB/s (MEASURED_PEAKS.json absent on this machine)")
        else:
            achieved = flops / kavg / 1e12
            peak = FP32_PEAK_TFLOPS if fp32 else FP64_PEAK_TFLOPS
            peak_src = ("FP32 pipe: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz = 80.5 TFLOP/s nominal (a plain FFMA "
                        "loop measured 74)") if fp32 else ("FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.26, "
                                                           "nominal 1.25 TFLOP/s (not in MEASURED_PEAKS.json; a plain "
                                                           "DFMA loop measured 1.2)")
        mode, precision = wl.precision() if hasattr(wl, "precision") else ("fp64", None)
        cfg = dict(wl.config(h), l2="flushed before every step (256 MiB write, untimed)",
                   parallelism=(f"{world} GPU(s), " + ("LPT shares of one block list" if args.shard == "lpt" and
                                                            world > 1 and isinstance(wl, FmmWorkload) else
                                                            "one independent problem per GPU")), mode=mode,
                   graph_ms_per_step=graph_ms, wall_s=t_wall)
        if precision:
            cfg["precision"] = precision
        cfg.update(wl.extra(res))
        for c in comparisons.values():
            c["speedup_of_this_line"] = value / c["value"] if c["value"] > 0 else None
        if comparisons:
            cfg["comparisons"] = comparisons
        line = {
            "metric": METRIC, "value": value, "unit": wl.unit, "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
            "config": cfg,
            "roofline": {"bound": bound, "kernel": wl.kernel, "achieved": achieved, "peak": peak,
                         "unit": runit, "frac": achieved / peak,
                         "traffic": ncu_traffic(wl.kernel, wl.name),
                         "peak_source": peak_src,
                         ("bytes_per_launch" if bound == "hbm" else "flops_per_launch"): flops,
                         "avg_launch_ms": kavg * 1e3,
                         "hbm_peak_gbs": peaks.get("hbm_gbs")},
            "kernels": {kname: {"ms_total": v[0], "launches": v[1]} for kname, v in prof.items()},
            "gpu_launches": int(launches),
            "launches_per_step": int(launches_per_step),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": wl.unit, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
        }
        if not args.no_cpu_baseline:
            good, n, el, desc = wl.oracle_units(h, args.cpu_budget)
            line["cpu_baseline"] = {"value": good / el, "unit": wl.unit, "cores": cpu_cores_used(), "kind": "oracle",
                                    "sample": f"{desc}; {el:.1f} s on 1 host thread"}
            if isinstance(wl, FmmWorkload) and type(wl).oracle_units is FmmWorkload.oracle_units:
                try:
                    good, n, el, ncpu, desc = wl.oracle_units_allcores(h, args.cpu_budget)
                    line["cpu_baseline_allcores"] = {"value": good / el, "unit": wl.unit, "cores": ncpu,
                                                     "kind": "oracle", "sample": desc}
                except Exception as e:          # the single-thread figure above stands on its own
                    line["cpu_baseline_allcores"] = {"error": f"{type(e).__name__}: {e}"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lib", choices=["lib", "reference"])
    ap.add_argument("--workload", default="fmm", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune-stages", action="store_true",
                    help="FMM batches: pick the schedule of generator sizes by lra_ca_batched_tune_stages (untimed)")
    ap.add_argument("--shard", default="lpt", choices=["lpt", "replicas"],
                    help="batched workloads on several GPUs: LPT shares of one block list, or a replica per GPU")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=90.0, help="seconds of oracle time for --impl reference")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]()
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_lib(args, wl)


if __name__ == "__main__":
    main()
