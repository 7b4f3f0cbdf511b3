#!/usr/bin/env python3
"""NNS-EMD throughput on GB300: pairs/s on the colour-transfer workload.

A step is one full NNS-EMD solve (every round of Alg. 1, Sec. III-A) of one
pair: two images' colour histograms, 65,536 points each in d=3 (8 Gaussian
colour clusters, sigma 0.08, clipped to [0,1)), uniform weights, squared
Euclidean ground distance, full sparse plan returned.  Inputs are synthetic
(the paper's seasonal colour-transfer images are not available).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun, one rank per GPU) every rank solves its own
pair (seed = rank): the pairs are independent, so there is no collective on
the data path ("weak" scaling); value = N*K pairs / max-over-ranks time.

Reported on one JSON line (rank 0):
  value / ms_per_step  device time of K solves with inputs resident in HBM
                       (CUDA events on the launching stream; L2 flushed
                       between steps by a 256 MiB write);
  e2e                  the same through nnsemd_solve_host: host (pinned)
                       inputs copied in and the plan copied out every step;
  roofline             the NNS kernel (K1) against the FP32-pipe peak: its
                       algorithmic work is 2d FP32 operations per
                       supplier/consumer pair (d subtractions, d multiply-
                       adds), timed by the library with CUDA events around
                       every K1 launch of the timed steps;
  cpu_baseline         the CPU oracle (single thread) on a bounded sample of
                       the workload, scaled to one full pair by NNS work.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = ("colour-transfer pair: 65,536 x 65,536 points, d=3, 8 Gaussian colour clusters "
            "(sigma 0.08, clipped to [0,1)), uniform weights, squared-Euclidean ground distance, "
            "full sparse plan returned")
METRIC = "NNS-EMD pairs/s at <=1e-3 rel err vs FP64 oracle; fused-kernel % of roofline"
N_POINTS = 65536
D = 3
SM_COUNT = 152
FP32_LANES_PER_SM = 128
ORACLE_SAMPLE_N = 16384        # oracle sample: the same generator at 16,384 points per side
WORK_FILE = os.path.join(ROOT, "tests", "golden", "colour_transfer_oracle.json")
COUNTERS_FILE = os.path.join(ROOT, "profiles", "k_nns_lowd_colour_transfer.json")


# ---------------------------------------------------------------------------
# ranks
# ---------------------------------------------------------------------------

def world():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(backend: str):
    import torch.distributed as dist
    rank, ws, _ = world()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)


def dist_reduce(value: float, op: str, device) -> float:
    """max / sum of a float over ranks (identity with one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def dist_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = max(smax, float(parts[2]))
                except ValueError:
                    continue
                for k, name in enumerate(names):
                    if parts[5 + k].lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample, scaled to one full pair by NNS work)
# ---------------------------------------------------------------------------

def full_pair_work() -> int | None:
    """Sum of m_t * n_t of the full workload, as computed by the oracle
    (tests/golden/make_oracle_values.py writes it)."""
    try:
        with open(WORK_FILE) as fh:
            return int(json.load(fh)["pair_evals"])
    except (OSError, KeyError, ValueError):
        return None


def oracle_sample(full_work: int | None) -> dict:
    import oracle
    from paper_2401_07378_gb300 import workloads
    p = workloads.color_transfer(seed=0, n=ORACLE_SAMPLE_N)
    t0 = time.perf_counter()
    r = oracle.solve_pair(p, "sql2")
    dt = time.perf_counter() - t0
    scale = (full_work / r.pair_evals) if full_work else (N_POINTS / ORACLE_SAMPLE_N) ** 2
    per_pair = dt * scale
    return {"value": 1.0 / per_pair, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle (FP64 mass, FP32 decisions checked against FP64) on one {ORACLE_SAMPLE_N}-point "
                       f"instance of the same generator: {dt:.2f} s for {r.pair_evals} pair evaluations, scaled "
                       f"by NNS work to the full pair ({full_work or 'n^2 ratio'} evaluations)"),
            "seconds": dt}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def source_hash(path: str) -> str:
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()


def measured_traffic() -> float | None:
    """DRAM bytes per K1 launch from the committed ncu capture, if it was
    taken on the current kernel source."""
    try:
        with open(COUNTERS_FILE) as fh:
            c = json.load(fh)
        src = os.path.join(ROOT, "paper_2401_07378_gb300", "csrc", "lowd.cu")
        if c.get("source_sha256") != source_hash(src):
            return None
        return float(c["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def run_ours(args) -> dict | None:
    import numpy as np
    import torch
    from paper_2401_07378_gb300 import nnsemd, workloads

    rank, ws, local = world()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init("nccl")
    pair = workloads.color_transfer(seed=rank)
    x = torch.from_numpy(pair.x).to(dev)
    a = torch.from_numpy(pair.a).to(dev)
    y = torch.from_numpy(pair.y).to(dev)
    b = torch.from_numpy(pair.b).to(dev)
    ctx = nnsemd.Context(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    T = nnsemd.FLAG_TIME_KERNELS

    for _ in range(args.warmup):
        ctx.solve(x, a, y, b, metric="sql2", plan=True)
    torch.cuda.synchronize()
    dist_barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    nns_ms = tail_ms = 0.0
    nns_pairs = nns_launches = launches = 0
    pair_evals = rounds = 0
    cost = None
    for k in range(args.steps):
        flush.zero_()
        starts[k].record()
        res = ctx.solve(x, a, y, b, metric="sql2", plan=True, flags=T)
        ends[k].record()
        s = res.stats
        nns_ms += s["nns_kernel_ms"]
        tail_ms += s["tail_kernel_ms"]
        nns_pairs += s["nns_kernel_pairs"]
        nns_launches += s["nns_kernel_launches"]
        launches += s["kernel_launches"]
        pair_evals, rounds, cost = s["pair_evals"], s["rounds"], res.cost
    torch.cuda.synchronize()
    dist_barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    max_ms = dist_reduce(total_ms, "max", dev)
    launches_all = int(dist_reduce(float(launches), "sum", dev))

    # end to end through the host entry point (pinned buffers)
    hx = torch.from_numpy(pair.x).pin_memory()
    ha = torch.from_numpy(pair.a).pin_memory()
    hy = torch.from_numpy(pair.y).pin_memory()
    hb = torch.from_numpy(pair.b).pin_memory()
    cap = 2 * N_POINTS - 1
    plan_out = (torch.empty(cap, dtype=torch.int32).pin_memory(), torch.empty(cap, dtype=torch.int32).pin_memory(),
                torch.empty(cap, dtype=torch.float64).pin_memory())
    for _ in range(min(args.warmup, 2)):
        ctx.solve_host(hx, ha, hy, hb, metric="sql2", plan=True, plan_out=plan_out)
    torch.cuda.synchronize()
    dist_barrier()
    e2e_ms = 0.0
    nnz = 0
    for k in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        hres = ctx.solve_host(hx, ha, hy, hb, metric="sql2", plan=True, plan_out=plan_out)
        e1.record()
        torch.cuda.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        nnz = int(hres.plan_f.numel())
        assert hres.cost == cost
    e2e_max = dist_reduce(e2e_ms, "max", dev)
    h2d = sum(t.numel() * t.element_size() for t in (hx, ha, hy, hb))
    d2h = nnz * (4 + 4 + 8) + 8

    if rank != 0:
        ctx.close()
        return None

    pk = peaks()
    clk_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak = SM_COUNT * FP32_LANES_PER_SM * clk_mhz * 1e6 / 1e12          # T FP32-pipe op/s
    per_launch_ops = nns_pairs * 2 * D / max(nns_launches, 1)
    per_launch_s = nns_ms / 1e3 / max(nns_launches, 1)
    achieved = per_launch_ops / per_launch_s / 1e12 if nns_ms > 0 else 0.0
    traffic = measured_traffic()
    value = ws * args.steps / (max_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 distances, f64 mass/cost", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_side": N_POINTS, "d": D, "metric": "sql2",
                   "precision": "fp32", "plan": "full", "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"{ws} independent pairs, one per GPU" if ws > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "kernel": "k_nns_lowd (K1, fused FP32 distance + argmin)",
                     "peak_basis": (f"152 SMs x 128 FP32 lanes x {clk_mhz:.0f} MHz (sm_max_mhz of "
                                    "MEASURED_PEAKS.json); work = 2d FP32-pipe ops per pair"),
                     "launches": nns_launches, "kernel_ms": nns_ms,
                     "share_of_step": nns_ms / total_ms if total_ms else None},
        "tail_kernel_share": tail_ms / total_ms if total_ms else None,
        "e2e": {"value": ws * args.steps / (e2e_max / 1e3), "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_all,
        "rounds_per_pair": rounds, "pair_evals_per_pair": pair_evals, "cost": cost,
        "clocks": clocks,
    }
    if ws == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(full_pair_work() or pair_evals)
        cb.pop("seconds", None)
        line["cpu_baseline"] = cb
    ctx.close()
    return line


def run_reference(args) -> dict | None:
    rank, ws, _ = world()
    if rank != 0:
        return None
    full_work = full_pair_work()
    for _ in range(args.warmup):
        oracle_sample(full_work)
    per_pair = []
    sample = None
    for _ in range(args.steps):
        r = oracle_sample(full_work)
        per_pair.append(1.0 / r["value"])
        sample = r["sample"]
    total = sum(per_pair)
    value = args.steps / total
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (oracle; decisions also in f32)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points_per_side": N_POINTS, "d": D, "metric": "sql2"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
