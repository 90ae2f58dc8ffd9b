"""Benchmark of the C-A CUR library on one or more GPUs of one node.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lib|reference] [--workload NAME]

A step is one pass of the hot path over one synthetic input: the C-A CUR
approximation (strip gathers with the fused multiplier, FP64 maxvol, nucleus,
outputs C, U, R) followed by the sampled a-posteriori residual check of the
result.  Inputs are seeded, synthetic and resident in HBM before the timed
region; L2 is flushed (a 256 MiB write) before every timed step and each step is
timed with CUDA events on the launching stream.  ``e2e`` repeats the same steps
through the same public API from pinned host buffers, copies included.

Under torchrun every rank runs an independent replica (a single LRA does not
shard: its maxvol needs a global argmax per swap) and rank 0 prints one JSON
line with the whole-job throughput (max time over ranks).  ``--impl reference``
times the FP64 CPU oracle on the same workload (rank 0 only).
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


# ------------------------------------------------------------------ workloads
class DenseSpiky:
    """8192 x 8192 FP32, numerical rank 32 (Gaussian factors, s_i = 2^{-i/2},
    1e-6 noise) with 1% of the entries replaced by +-10 spikes; right multiplier
    ARHT (d = 2) or sparse +-1 (4 nonzeros per column); k = 48, 4 C-A loops."""

    def __init__(self, mult: str, n: int = 8192, k: int = 48, sweeps: int = 4, seed: int = 0):
        self.mult, self.n, self.k, self.sweeps, self.seed = mult, n, k, sweeps, seed
        self.name = f"dense{n}_f32_rank32_spikes1pct_{'arht2' if mult == 'arht' else 'sparse4'}_k{k}_s{sweeps}"
        self.q = self.s = 256

    def host(self, rank: int):
        p = li.dense_spiky(self.n, r=32, seed=self.seed + 1000 * rank)
        if self.mult == "arht":
            li.with_arht(p, 2, self.seed + 7)
        else:
            li.with_sparse(p, 4, self.seed + 7)
        I0 = li.initial_rows(self.n, self.k, self.seed + 11)
        Q, S = li.sample_positions(self.n, self.n, self.q, self.s, self.seed + 13)
        return p, I0, Q, S

    def config(self):
        return {"workload": self.name, "m": self.n, "n": self.n, "k": self.k, "sweeps": self.sweeps,
                "multiplier": "ARHT d=2" if self.mult == "arht" else "sparse +-1, 4 nnz/col",
                "input_dtype": "f32", "residual_sample": f"{self.q}x{self.s}"}

    def flops_per_lra(self, swaps: int) -> float:
        """Algorithmic FP64 flops of one C-A run (fma = 2, division = 1): the
        maxvol steps of the FP64 reference, see maxvol_flops()."""
        k, n = self.k, self.n
        f = maxvol_flops(k, n, cold=True)
        f += (2 * self.sweeps - 1) * maxvol_flops(k, n, cold=False)
        f += swaps * (2.0 * k * n + n)
        return f


def maxvol_flops(k: int, n: int, cold: bool) -> float:
    if cold:
        fma = sum((k - 1 - t) * (n - 1 - t) for t in range(k))
    else:
        fma = sum((k - 1 - t) * (n - k) for t in range(k)) + sum((k - 1 - t) ** 2 for t in range(k))
    fma += (n - k) * k * (k - 1) // 2
    div = (n - k) * k + (k * (k - 1) // 2)
    return 2.0 * fma + div


WORKLOADS = {
    "dense8192_arht": lambda: DenseSpiky("arht"),
    "dense8192_sparse": lambda: DenseSpiky("sparse"),
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
        except (OSError, FileNotFoundError):
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
                sm.append(float(f[1])); mx = float(f[2])
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
    """Per-launch DRAM bytes of `kernel` from a committed ncu summary, if it was
    taken on the current sources (profiles/<kernel>__<workload>.txt lines
    'csrc_hash: ...' and 'dram_bytes_per_launch: ...'); else None."""
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


# ------------------------------------------------------------------ oracle arm
def oracle_step(wl, p, I0, Q, S):
    import oracle
    o = oracle.ca_run(p, wl.k, wl.sweeps, I0)
    st = oracle.residual_sample(p, o["C"], o["U"], o["R"], Q, S)
    return o, st


def cpu_baseline(wl, p, I0, Q, S, budget_s: float = 12.0):
    """The oracle as it stands, single-threaded, on whole LRAs until budget_s."""
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle_step(wl, p, I0, Q, S)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 50:
            break
    return {"value": n / el, "unit": "LRA/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} complete LRAs of the same workload (C-A + nucleus + {wl.q}x{wl.s} residual sample), "
                      f"{el:.1f} s, 1 thread"}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p, I0, Q, S = wl.host(0)
    for _ in range(args.warmup):
        oracle_step(wl, p, I0, Q, S)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(wl, p, I0, Q, S)
    el = time.perf_counter() - t0
    v = args.steps / el
    line = {"metric": METRIC, "value": v, "unit": "LRA/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": wl.config(),
            "cpu_baseline": {"value": v, "unit": "LRA/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed LRAs after {args.warmup} warm-up, 1 thread"},
            "e2e": {"value": v, "unit": "LRA/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = "CUR LRAs/s (C-A, FP64 pivots and nucleus)"


# ------------------------------------------------------------------ library arm
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

    p, I0, Q, S = wl.host(rank)
    Wd = torch.from_numpy(p.W).to(dev)
    prob = lra.Problem.dense(Wd)
    mult = (lra.lra_precondition("arht", p.n, p.depth, p.perm, p.dsign) if p.mkind == li.MULT_ARHT
            else lra.lra_precondition("sparse", p.n, p.nnz, p.srow, p.ssign))
    I0d = torch.from_numpy(I0).to(dev)
    Qd, Sd = torch.from_numpy(Q).to(dev), torch.from_numpy(S).to(dev)
    k, sweeps = wl.k, wl.sweeps
    out = lra.lra_ca_run(prob, I0d, k, sweeps, multiplier=mult)
    ws = out["_workspace"]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2

    def step():
        lra.lra_ca_run(prob, I0d, k, sweeps, multiplier=mult, out=out, workspace=ws)
        return lra.lra_residual_sample(prob, out["C"], out["U"], out["R"], Qd, Sd)

    for _ in range(max(args.warmup, 3)):
        stats = step()
    torch.cuda.synchronize()
    info = out["info"].cpu().numpy()
    if info[3] not in (0, 16, 17):
        raise RuntimeError(f"C-A run failed with status {info[3]}")

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = lra.lra_launch_count()
    lra.lra_profile_enable(True)
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        stats = step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    lra.lra_profile_enable(False)
    launches = lra.lra_launch_count() - launches0
    prof = lra.lra_profile_collect()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    t_max = torch.tensor([step_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    total_ms = float(t_max.item())
    value = world * args.steps / (total_ms / 1e3)

    # end to end through the same API from pinned host memory
    Wh = torch.from_numpy(p.W).pin_memory()
    I0h = torch.from_numpy(I0).pin_memory()
    host_out = {key: torch.empty(v.shape, dtype=v.dtype).pin_memory() for key, v in out.items()
                if not key.startswith("_")}
    st_h = torch.empty(5, dtype=torch.float64).pin_memory()
    h2d = Wh.numel() * Wh.element_size() + I0h.numel() * 4
    d2h = sum(v.numel() * v.element_size() for v in host_out.values()) + 40

    def e2e_step():
        Wd.copy_(Wh, non_blocking=True)
        I0d.copy_(I0h, non_blocking=True)
        s = step()
        for key, v in host_out.items():
            v.copy_(out[key], non_blocking=True)
        st_h.copy_(s, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_ms, op=dist.ReduceOp.MAX)
    e2e_value = world * args.steps / (float(e2e_ms.item()) / 1e3)

    if rank == 0:
        info = out["info"].cpu().numpy()
        st = stats.cpu().numpy()
        swaps = int(info[1])
        ca_ms, ca_n = prof.get("ca_kernel", (float("nan"), 0))
        ca_avg_s = ca_ms / max(ca_n, 1) / 1e3
        flops = wl.flops_per_lra(swaps)
        achieved = flops / ca_avg_s / 1e12
        traffic = ncu_traffic("ca_kernel", wl.name)
        peaks = load_peaks()
        line = {
            "metric": METRIC, "value": value, "unit": "LRA/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(wl.config(), l2="flushed before every step (256 MiB write, untimed)",
                           parallelism=f"replicas x{world}", mode="fp64",
                           rank=int(info[0]), swaps=swaps, loops=int(info[2]), status=int(info[3]),
                           rel_fro_err_sampled=float(st[4]), wall_s=t_wall),
            "roofline": {"bound": "alu", "kernel": "ca_kernel", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                         "peak_source": "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz (nominal 1.25 TFLOP/s)",
                         "flops_per_launch": flops, "avg_launch_ms": ca_avg_s * 1e3,
                         "hbm_peak_gbs": peaks.get("hbm_gbs")},
            "kernels": {kname: {"ms_total": v[0], "launches": v[1]} for kname, v in prof.items()},
            "gpu_launches": int(launches),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "LRA/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, p, I0, Q, S)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lib", choices=["lib", "reference"])
    ap.add_argument("--workload", default="dense8192_arht", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]()
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_lib(args, wl)


if __name__ == "__main__":
    main()
