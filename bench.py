#!/usr/bin/env python3
"""NNS-EMD throughput on GB300 (pairs/s), with a live roofline.

Default workload (the one the headline metric is quoted on): one step is one
full NNS-EMD solve (every round of Alg. 1, Sec. III-A) of a colour-transfer
pair -- two images' colour histograms, 65,536 points each in d=3 (8 Gaussian
colour clusters, sigma 0.08, clipped to [0,1)), uniform weights,
squared-Euclidean ground distance, full sparse plan returned.  Inputs are
synthetic (the paper's seasonal colour-transfer images are not available).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload colour|single|gmm|docs|retrieval] [--precision fp32|bf16|fp16|fp8]

Other workloads (reported by hand, not by the driver):
  single     one 256 x 256 pair in d=2, Euclidean;
  gmm        one 262,144 x 262,144 pair in d=64 (256-component mixture), Euclidean;
  docs       1 query document vs 4,096 documents, word vectors d=300 (batched);
  retrieval  10,000 signature pairs, 256..2,048 descriptors of d=128 (batched).

With N > 1 (torchrun, one rank per GPU): a batched workload (docs,
retrieval) is ONE batch split over the ranks by estimated work (greedy
longest-processing-time on m * n, shard.py), every rank solves its share and
the P costs are all-gathered in pair order ("strong" scaling: the total work
is fixed); a single-pair workload runs one independent pair per rank
(seed = rank, "weak" scaling).  value = all ranks' pairs / max-over-ranks time.

JSON line (rank 0):
  value / ms_per_step  device time of K steps with inputs resident in HBM
                       (CUDA events on the launching stream; L2 flushed by a
                       256 MiB write before every step, outside the events);
  e2e                  the same step end to end: single pairs through
                       nnsemd_solve_host (pinned host inputs copied in and the
                       plan copied out every step); batches with the packed
                       inputs copied in from pinned memory and the P costs
                       read back every step;
  roofline             the dominant kernel against its peak: the FP32 pipe
                       for the CUDA-core NNS kernels (2d FP32 operations per
                       supplier/consumer pair), the tensor pipe for the
                       tcgen05 kernel (2d flops per pair), timed by the
                       library with CUDA events around each launch;
  cpu_baseline         the CPU oracle timed on all host cores: colour, the
                       full pair (the oracle's multi-core twin); docs, every
                       pair; retrieval, a seeded 200-pair subset; single, the
                       pair solved repeatedly (one copy per core); gmm, a
                       8,192-point instance scaled to the full pair;
  accuracy             R of the GPU against the oracle on the same pairs:
                       relative error against the FP64-decision oracle (the
                       metric's "rel err vs FP64 oracle") and against the
                       FP32-decision oracle (whose decisions the kernels
                       take), the pairs checked and the oracle's FP32/FP64
                       near-ties; the run fails (exit 3) above the tolerance
                       (1e-5 for FP32 forms, 1e-3 for reduced precision and
                       learned forms).
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

METRIC = "NNS-EMD pairs/s at <=1e-3 rel err vs FP64 oracle; fused-kernel % of roofline"
FP32_LANES_PER_SM = 128
GMM_SAMPLE_N = 8192            # GMM oracle sample: 8,192 points per side (the full pair is out of reach)
RETRIEVAL_SAMPLE = 200         # retrieval pairs the oracle checks (seeded subset)
TOL_FP32 = 1e-5                # relative error bound of the FP32 forms against the FP64 oracle
TOL_REDUCED = 1e-3             # ... of the reduced-precision and learned forms
WORK_FILE = os.path.join(ROOT, "tests", "golden", "colour_transfer_oracle.json")
COUNTERS_FILE = os.path.join(ROOT, "profiles", "k_nns_lowd_colour_transfer.json")

WORKLOADS = {
    "colour": dict(d=3, desc=("colour-transfer pair: 65,536 x 65,536 points, d=3, 8 Gaussian colour clusters "
                         "(sigma 0.08, clipped to [0,1)), uniform weights, squared-Euclidean ground distance, "
                         "full sparse plan returned"), metric="sql2", precision="fp32", batched=False),
    "single": dict(d=2, desc="single pair: 256 x 256 points, d=2, Uniform[0,1), uniform weights, Euclidean, full plan",
                   metric="l2", precision="fp32", batched=False),
    "gmm": dict(d=64, desc=("GMM pair: 262,144 x 262,144 points, d=64, 256-component mixture (means N(0,4I), "
                      "cov 0.25I), Dirichlet(0.5) weights, Euclidean, full plan; learned candidate proposal "
                      "(MLP 64-256-256-4096 cells, trained on 200 seeded plain runs), BF16 contraction (split "
                      "high/low BF16 parts, BF16X3, top-8 candidates re-ranked in FP32) for the consumers it "
                      "cannot certify"),
                metric="l2", precision="bf16x3", batched=False, proposal="learned", steps=5, rerank_k=8),
    "docs": dict(d=300, desc=("document kNN: 1 query vs 4,096 documents, word vectors d=300 N(0,1) L2-normalised "
                       "(50k vocabulary), lengths LogNormal(ln 60, 0.6) clipped to [20,500], Zipf(1.1) weights, "
                       "Euclidean, BF16 distances + FP32 re-rank, one persistent launch replayed as a CUDA graph"),
                 metric="l2", precision="bf16", batched=True, graph=True, steps=50),
    "retrieval": dict(d=128, desc=("retrieval: 10,000 signature pairs, m, n ~ U{256..2048}, d=128 |N(0,1)| "
                            "L2-normalised x512, Dirichlet(1) weights, Euclidean, FP16 distances + FP32 re-rank, "
                            "autotuned tiles, batched"),
                      metric="l2", precision="fp16", batched=True, autotune=True, steps=5),
}


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
# inputs
# ---------------------------------------------------------------------------

def make_inputs(name: str, rank: int, points: int | None = None, pairs: int | None = None):
    """The workload's synthetic input (seed = rank).  ``points`` / ``pairs``
    shrink it for profiling captures (not for bench lines)."""
    from paper_2401_07378_gb300 import workloads
    if name == "colour":
        return workloads.color_transfer(seed=rank, n=points or 65536)
    if name == "single":
        return workloads.single_pair(seed=rank)
    if name == "gmm":
        return workloads.gmm_pair(seed=rank, n=points or 262144)
    if name == "docs":
        return workloads.doc_knn(seed=rank, num_docs=pairs or 4096)
    if name == "retrieval":
        return workloads.retrieval(seed=rank, num_pairs=pairs or 10000)
    raise ValueError(name)


# ---------------------------------------------------------------------------
# CPU oracle: timing on the host cores and the accuracy of the GPU's R
# ---------------------------------------------------------------------------

def golden_fp64_cost() -> float | None:
    """R of the full colour-transfer pair under FP64 decisions, written by
    tests/golden/make_oracle_values.py (calls only the oracle)."""
    try:
        with open(WORK_FILE) as fh:
            return float(json.load(fh)["fp64"]["cost"])
    except (OSError, KeyError, ValueError):
        return None


def warm_pool(pool):
    """Start every worker of an oracle process pool before any timing."""
    list(pool.map(time.sleep, [0.2] * pool._max_workers))


def retrieval_subset(num_pairs: int) -> list[int]:
    """The seeded subset of retrieval pairs the oracle checks."""
    import numpy as np
    k = min(RETRIEVAL_SAMPLE, num_pairs)
    return sorted(int(p) for p in np.random.default_rng(0).choice(num_pairs, size=k, replace=False))


def oracle_time(name: str, inp, pool=None) -> dict:
    """Time the oracle, as it stands, on the host cores over a bounded sample
    of the workload ``inp``.  Returns the rate (pairs/s), the threads used,
    a description of the sample and the oracle's results (pair index -> R
    under FP32 decisions, and its FP32/FP64 near-ties).  ``pool``: the host
    process pool (oracle.process_pool) of the many-pair samples."""
    import oracle
    from paper_2401_07378_gb300 import workloads
    cores = max(1, oracle.max_threads()) if name in ("colour", "gmm") else pool._max_workers
    metric = WORKLOADS[name]["metric"]
    costs, ties = {}, 0
    t0 = time.perf_counter()
    if name == "colour":
        r = oracle.solve_pair(inp, metric, threads=0)
        dt = time.perf_counter() - t0
        costs[0], ties = r.cost, r.near_ties
        value = 1.0 / dt
        sample = (f"the full pair, solved once by the oracle's multi-core twin on {cores} host threads "
                  f"({dt:.2f} s, {r.rounds} rounds, {r.pair_evals} pair evaluations)")
    elif name == "single":
        done, batch = 0, cores * 8
        while True:
            rs = oracle.solve_many([inp] * batch, metric, pool=pool)
            done += batch
            dt = time.perf_counter() - t0
            if dt > 3.0:
                break
        costs[0], ties = rs[0].cost, rs[0].near_ties
        value = done / dt
        sample = f"the full pair solved {done} times, one copy per host process on {cores} processes, in {dt:.2f} s"
    elif name == "gmm":
        p = workloads.gmm_pair(seed=0, n=GMM_SAMPLE_N)
        r = oracle.solve_pair(p, metric, threads=0)
        dt = time.perf_counter() - t0
        scale = (262144 / GMM_SAMPLE_N) ** 2
        value = 1.0 / (dt * scale)
        sample = (f"one {GMM_SAMPLE_N}-point instance of the same generator on {cores} host threads: {dt:.2f} s "
                  f"for {r.pair_evals} pair evaluations, scaled to 262,144 points by (262144/{GMM_SAMPLE_N})^2 "
                  f"(assumes the NNS work grows as m * n; the oracle's own count on the sample)")
    else:
        ids = list(range(inp.num_pairs)) if name == "docs" else retrieval_subset(inp.num_pairs)
        rs = oracle.solve_many([inp.pair(k) for k in ids], metric, pool=pool)
        dt = time.perf_counter() - t0
        for k, r in zip(ids, rs):
            costs[k] = r.cost
            ties += r.near_ties
        value = len(ids) / dt
        which = "every pair of the batch" if name == "docs" else f"a seeded {len(ids)}-pair subset of the batch"
        sample = f"{which}, one pair per host process on {cores} processes, in {dt:.2f} s"
    return {"value": value, "cores": cores, "sample": sample, "seconds": dt, "costs": costs, "near_ties": ties}


def accuracy(name: str, inp, gpu_costs: dict, orc: dict, tol: float, pool=None) -> dict:
    """Relative error |R_gpu - R_oracle| / R_oracle (Sec. IV-F's definition,
    taken against the oracle) over the pairs the oracle solved, against the
    FP32-decision oracle and against the FP64-decision oracle."""
    import oracle
    metric = WORKLOADS[name]["metric"]
    out = {"pairs_checked": 0, "rel_err_vs_fp32_decision_oracle": None, "rel_err_vs_fp64_oracle": None,
           "oracle_near_ties_fp32_vs_fp64": orc.get("near_ties"), "tolerance": tol}
    if not orc["costs"]:
        out["note"] = ("the oracle cannot solve the full pair in bounded time; parity of this form is tested "
                       "against the oracle at 16,384 points per side (tests/test_gpu_full_size.py)")
        out["ok"] = None
        return out
    ids = sorted(orc["costs"])
    rel = lambda g, o: abs(g - o) / abs(o) if o != 0 else abs(g - o)
    out["pairs_checked"] = len(ids)
    out["rel_err_vs_fp32_decision_oracle"] = max(rel(gpu_costs[k], orc["costs"][k]) for k in ids)
    if name == "colour":
        r64 = {0: golden_fp64_cost()}
        out["fp64_source"] = "tests/golden/colour_transfer_oracle.json (oracle-written, FP64 decisions)"
    elif name == "single":
        r64 = {0: oracle.solve_pair(inp, metric, decide="fp64").cost}
    else:
        pairs = [inp.pair(k) for k in ids]
        r64 = dict(zip(ids, (r.cost for r in oracle.solve_many(pairs, metric, decide="fp64", pool=pool))))
    if all(v is not None for v in r64.values()):
        out["rel_err_vs_fp64_oracle"] = max(rel(gpu_costs[k], r64[k]) for k in ids)
    worst = max(v for v in (out["rel_err_vs_fp32_decision_oracle"], out["rel_err_vs_fp64_oracle"]) if v is not None)
    out["ok"] = bool(worst <= tol)
    return out


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

K1_BEGIN = "// K1: fused FP32 distance + argmin"
K1_END = "// one-CTA solver"


def k1_source_hash() -> str:
    """sha256 over K1's source: its section of lowd.cu (from the K1 banner to
    the next section's) followed by common.cuh, whose helpers it inlines."""
    csrc = os.path.join(ROOT, "paper_2401_07378_gb300", "csrc")
    with open(os.path.join(csrc, "lowd.cu")) as fh:
        text = fh.read()
    begin = text.index(K1_BEGIN)
    part = text[begin:text.index(K1_END, begin)]
    with open(os.path.join(csrc, "common.cuh")) as fh:
        part += fh.read()
    return hashlib.sha256(part.encode()).hexdigest()


def measured_traffic() -> float | None:
    """DRAM bytes per K1 launch from the committed ncu capture, if it was
    taken on the current K1 source."""
    try:
        with open(COUNTERS_FILE) as fh:
            c = json.load(fh)
        if c.get("source_sha256") != k1_source_hash():
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


def roofline(d: int, precision: str, rk: int, pairs: int, launches: int, ms: float, total_ms: float, lowd: bool,
             sms: int) -> dict:
    pk = peaks()
    per_launch_s = ms / 1e3 / max(launches, 1)
    if precision == "fp32":
        clk = float(pk.get("sm_max_mhz", 2070.0))
        peak = sms * FP32_LANES_PER_SM * clk * 1e6 / 1e12
        ops = pairs * 2 * d / max(launches, 1)
        basis = (f"{sms} SMs (the device's multiprocessor count) x 128 FP32 lanes x {clk:.0f} MHz "
                 f"(sm_max_mhz of MEASURED_PEAKS.json); "
                 f"work = 2d FP32-pipe ops per supplier/consumer pair")
        bound = "alu"
        kernel = "k_nns_lowd (K1)" if lowd else "k_nns_f32_tiled"
    else:
        bf16 = float(pk.get("bf16_tflops", 1935.1))
        peak = bf16 * (2.0 if precision == "fp8" else 1.0)
        ops = pairs * 2 * d / max(launches, 1)
        basis = ("measured cuBLAS bf16 burst of MEASURED_PEAKS.json" +
                 (" x 2 (nominal fp8/bf16 ratio)" if precision == "fp8" else "") +
                 "; work = 2d flops per supplier/consumer pair" +
                 (" (the BF16X3 split runs 3 x 2d on the tensor pipe)" if precision == "bf16x3" else ""))
        bound = "tensor"
        kernel = f"k_nns_tc<{precision}> (tcgen05 contraction + top-{8 if 1 <= rk <= 8 else 16} epilogue)"
    achieved = ops / per_launch_s / 1e12 if ms > 0 else 0.0
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None, "traffic": measured_traffic() if lowd else None,
            "kernel": kernel, "peak_basis": basis, "launches": launches, "kernel_ms": ms,
            "share_of_step": ms / total_ms if total_ms else None}




def rerank_k(args) -> int:
    """Reduced-precision candidates re-ranked per consumer (0: the library's 16)."""
    if getattr(args, "rerank_k", None) is not None:
        return args.rerank_k
    return WORKLOADS[args.workload].get("rerank_k", 0)


def bench_config(args, ws: int) -> dict:
    """The workload's `config` (the same dict on both arms)."""
    spec = WORKLOADS[args.workload]
    precision = args.precision or spec["precision"]
    if ws == 1:
        par = "1 GPU"
    elif spec["batched"]:
        par = f"one batch split over {ws} GPUs by estimated work (greedy longest-processing-time), costs all-gathered"
    else:
        par = f"{ws} independent pairs, one per GPU"
    return {"workload": spec["desc"], "name": args.workload, "d": spec["d"], "metric": spec["metric"],
            "precision": precision, "rerank_k": rerank_k(args), "protocol": args.protocol,
            "l2": "flushed before every step (256 MiB write)", "parallelism": par}


def run_ours(args) -> dict | None:
    import numpy as np
    import torch
    from paper_2401_07378_gb300 import nnsemd, shard

    spec = WORKLOADS[args.workload]
    precision = args.precision or spec["precision"]
    metric = spec["metric"]
    proposal = args.proposal or spec.get("proposal", "none")
    rk = rerank_k(args)
    rank, ws, local = world()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init("nccl")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # a batch is one workload split over the ranks; a single pair runs once per rank
    full = make_inputs(args.workload, 0 if spec["batched"] else rank, args.points, args.pairs)
    inp, shares = full, None
    if spec["batched"] and ws > 1:
        shares = shard.partition(shard.pair_work(full.x_off, full.y_off), ws)
        inp = shard.sub_batch(full, shares[rank])
    ctx = nnsemd.Context(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    T = nnsemd.FLAG_TIME_KERNELS
    t = lambda v: torch.from_numpy(v).to(dev)
    x, a, y, b = t(inp.x), t(inp.a), t(inp.y), t(inp.b)
    d = int(full.x.shape[1])
    prop, prop_info = None, None
    if proposal == "learned":
        if args.workload != "gmm":
            raise SystemExit("--proposal learned serves the gmm workload")
        from paper_2401_07378_gb300 import proposal_training
        prop, prop_info = proposal_training.build_gmm_proposal(ctx, d=d)
    costs = None
    if spec["batched"]:
        P = inp.num_pairs
        costs = torch.empty(P, dtype=torch.float64, device=dev)
        bflags = ((nnsemd.FLAG_GRAPH if spec.get("graph") else 0) |
                  (nnsemd.FLAG_AUTOTUNE if spec.get("autotune") else 0))
        step = lambda: ctx.solve_batched(x, a, inp.x_off, y, b, inp.y_off, metric=metric, precision=precision,
                                         rerank_k=rk, costs=costs, stats=True, flags=bflags,
                                         protocol=args.protocol)[1]
        units = P
    else:
        def step():
            r = ctx.solve(x, a, y, b, metric=metric, precision=precision, rerank_k=rk, plan=True, flags=T,
                          proposal=prop, protocol=args.protocol)
            return dict(r.stats, cost=r.cost)
        units = 1

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist_barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    agg = {"nns_kernel_ms": 0.0, "tail_kernel_ms": 0.0, "nns_kernel_pairs": 0, "nns_kernel_launches": 0,
           "kernel_launches": 0, "certified": 0, "fallbacks": 0, "near_ties": 0, "widened": 0}
    last = None
    # the timed steps alone for a profiler started with --profile-from-start off
    torch.cuda.cudart().cudaProfilerStart()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record()
        s = step()
        ends[k].record()
        for key in agg:
            agg[key] += s.get(key, 0) or 0
        last = s
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    dist_barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    total_ms = sum(step_ms)
    max_ms = dist_reduce(total_ms, "max", dev)
    launches_all = int(dist_reduce(float(agg["kernel_launches"]), "sum", dev))
    # every pair's R, in pair order (a split batch is gathered from all ranks)
    if spec["batched"]:
        gpu_costs = (shard.gather_costs(costs, shares, full.num_pairs, rank, dev) if shares is not None
                     else costs.cpu().numpy())
    else:
        gpu_costs = np.array([(last or {}).get("cost")], np.float64)
    total_units = full.num_pairs if spec["batched"] else ws * units

    e2e = None
    if spec["batched"]:
        # the packed batch copied in from pinned host memory, solved, and the
        # P costs read back, every step (separate device buffers, so a
        # captured graph of the device-resident step is not reused here)
        hx, ha = torch.from_numpy(inp.x).pin_memory(), torch.from_numpy(inp.a).pin_memory()
        hy, hb = torch.from_numpy(inp.y).pin_memory(), torch.from_numpy(inp.b).pin_memory()
        dx, da, dy, db = (torch.empty_like(v) for v in (x, a, y, b))
        hcosts = torch.empty(P, dtype=torch.float64).pin_memory()

        def host_step():
            for dv, hv in ((dx, hx), (da, ha), (dy, hy), (db, hb)):
                dv.copy_(hv, non_blocking=True)
            ctx.solve_batched(dx, da, inp.x_off, dy, db, inp.y_off, metric=metric, precision=precision,
                              rerank_k=rk, costs=costs, flags=bflags, protocol=args.protocol)
            hcosts.copy_(costs, non_blocking=True)

        for _ in range(min(args.warmup, 2)):
            host_step()
        torch.cuda.synchronize()
        dist_barrier()
        e2e_ms = 0.0
        for k in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            host_step()
            e1.record()
            torch.cuda.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        e2e_max = dist_reduce(e2e_ms, "max", dev)
        e2e = {"value": args.steps * total_units / (e2e_max / 1e3), "unit": "pairs/s",
               "h2d_bytes_per_step": sum(v.numel() * v.element_size() for v in (hx, ha, hy, hb)),
               "d2h_bytes_per_step": P * 8}
    else:
        hx, ha = torch.from_numpy(inp.x).pin_memory(), torch.from_numpy(inp.a).pin_memory()
        hy, hb = torch.from_numpy(inp.y).pin_memory(), torch.from_numpy(inp.b).pin_memory()
        cap = inp.m + inp.n - 1
        plan_out = (torch.empty(cap, dtype=torch.int32).pin_memory(),
                    torch.empty(cap, dtype=torch.int32).pin_memory(),
                    torch.empty(cap, dtype=torch.float64).pin_memory())
        host_step = lambda: ctx.solve_host(hx, ha, hy, hb, metric=metric, precision=precision, rerank_k=rk,
                                           plan=True, plan_out=plan_out, proposal=prop, protocol=args.protocol)
        for _ in range(min(args.warmup, 2)):
            host_step()
        torch.cuda.synchronize()
        dist_barrier()
        e2e_ms, nnz = 0.0, 0
        for k in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            hres = host_step()
            e1.record()
            torch.cuda.synchronize()
            e2e_ms += e0.elapsed_time(e1)
            nnz = int(hres.plan_f.numel())
        e2e_max = dist_reduce(e2e_ms, "max", dev)
        e2e = {"value": args.steps * total_units / (e2e_max / 1e3), "unit": "pairs/s",
               "h2d_bytes_per_step": sum(v.numel() * v.element_size() for v in (hx, ha, hy, hb)),
               "d2h_bytes_per_step": nnz * (4 + 4 + 8) + 8}

    if rank != 0:
        ctx.close()
        return None

    lowd = d <= 8
    if spec["batched"]:
        # the persistent batched kernel is the step: its NNS work against the
        # FP32 pipe, or the tensor pipe when the contraction runs there
        rl = roofline(d, precision, rk,
                      agg.get("nns_kernel_pairs", 0) or (last or {}).get("pair_evals", 0) * args.steps,
                      args.steps, total_ms, total_ms, lowd, sms)
        if precision == "fp32":
            rl["kernel"] = ("k_batched_lowd" if lowd else
                            "k_batched_hd / k_batched_hd_small (persistent, one pair per CTA)")
        else:
            rl["kernel"] = f"k_batched_tc<{precision}> (persistent, one pair per CTA, tcgen05 NNS per round)"
        rl["traffic"] = None
    elif agg["nns_kernel_launches"] == 0 and agg["tail_kernel_ms"] > 0:
        # a pair small enough for one launch (k_solve_small): that kernel runs
        # every round, so its NNS work over its own time
        rl = roofline(d, precision, rk, (last or {}).get("pair_evals", 0) * args.steps, args.steps,
                      agg["tail_kernel_ms"], total_ms, lowd, sms)
        rl["kernel"] = "k_solve_small (the whole pair in one launch: every round's NNS, grouping, flow, compaction)"
        rl["traffic"] = None
        rl["note"] = "latency-bound: the NNS work is a small part of each round"
    else:
        rl = roofline(d, precision, rk, agg["nns_kernel_pairs"], agg["nns_kernel_launches"], agg["nns_kernel_ms"],
                      total_ms, lowd, sms)
        if prop is not None:
            # the learned step scans candidates only: its rate is the full scan's work over its time
            rl["kernel"] = ("learned NNS step (cell lists, candidate plan, k_lc_keys cell-by-cell exact scan, "
                            "certificate, tensor-core scan + re-rank of the uncertified)")
            rl["note"] = "achieved counts the full scan's 2d ops per pair: an effective rate, not pipe utilisation"
    line = {
        "metric": METRIC, "value": args.steps * total_units / (max_ms / 1e3), "unit": "pairs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if (spec["batched"] and ws > 1) else "weak", "vs_baseline": None,
        "dtype": "f32 distances, f64 mass/cost" if precision == "fp32" else f"{precision} contraction, f32 re-rank, f64 mass/cost",
        "data": "synthetic",
        "config": bench_config(args, ws),
        "roofline": rl,
        "tail_kernel_share": agg["tail_kernel_ms"] / total_ms if total_ms else None,
        "gpu_launches": launches_all,
        "rounds_per_step": (last or {}).get("rounds"), "pair_evals_per_step": (last or {}).get("pair_evals"),
        "certified": agg["certified"], "certified_by_second_tier": agg["widened"], "fallbacks": agg["fallbacks"],
        "near_ties_reduced_precision": agg["near_ties"],
        "cost": float(gpu_costs[0]) if not spec["batched"] else None,
        "proposal": prop_info,
        "clocks": clocks,
    }
    line["e2e"] = e2e
    if args.points or args.pairs:
        line["config"]["reduced_size"] = {"points": args.points, "pairs": args.pairs}
        line["config"]["workload"] += " [REDUCED SIZE: profiling case, not the workload]"
    if prop is not None:
        line["config"]["proposal"] = "learned (trained before timing; training not in the timed region)"
        prop.close()
    if args.workload == "gmm" and not args.no_plain:
        # the plain FP32 form of the same solve on the same GPU, for comparison
        plain = lambda: ctx.solve(x, a, y, b, metric=metric, precision="fp32", plan=True)
        plain()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k_plain = 2
        flush.zero_()
        p0.record()
        for _ in range(k_plain):
            pr = plain()
        p1.record()
        torch.cuda.synchronize()
        line["plain_fp32"] = {"value": k_plain / (p0.elapsed_time(p1) / 1e3), "unit": "pairs/s", "steps": k_plain,
                              "same_cost": pr.cost == (last or {}).get("cost", pr.cost)}
    ctx.close()
    tol = TOL_FP32 if (precision == "fp32" and prop is None) else TOL_REDUCED
    if ws == 1 and not args.no_cpu_baseline and not (args.points or args.pairs):
        import oracle
        with oracle.process_pool() as pool:
            warm_pool(pool)
            orc = oracle_time(args.workload, full, pool)
            acc = accuracy(args.workload, full, dict(enumerate(gpu_costs.tolist())), orc, tol, pool)
        line["cpu_baseline"] = {"value": orc["value"], "unit": "pairs/s", "cores": orc["cores"], "kind": "oracle",
                                "sample": orc["sample"]}
        line["accuracy"] = acc
        line["rel_err_vs_fp64_oracle"] = acc["rel_err_vs_fp64_oracle"]
    return line


def run_reference(args) -> dict | None:
    """The oracle as it stands, timed on the host cores on the same workload
    (each step the bounded sample of oracle_time); rank 0 only."""
    rank, ws, _ = world()
    if rank != 0:
        return None
    import oracle
    name = args.workload
    full = make_inputs(name, 0, args.points, args.pairs)
    with oracle.process_pool() as pool:
        warm_pool(pool)
        for _ in range(args.warmup):
            oracle_time(name, full, pool)
        secs, units, last = 0.0, 0.0, None
        for _ in range(args.steps):
            r = oracle_time(name, full, pool)
            secs += r["seconds"]
            units += r["value"] * r["seconds"]
            last = r
    value = units / secs
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 mass/cost, f32 decisions (the CPU oracle)", "data": "synthetic",
            "config": bench_config(args, 1),
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200 for colour/single, fewer for the larger workloads)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="colour")
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp16", "fp8", "bf16x3"], default=None)
    ap.add_argument("--proposal", choices=["none", "learned"], default=None,
                    help="gmm only (default learned): train a learned candidate proposal before timing")
    ap.add_argument("--no-plain", action="store_true", help="gmm: skip timing the plain FP32 form")
    ap.add_argument("--protocol", choices=["greedy", "random"], default="greedy",
                    help="serving order of a supplier's consumers (Sec. III-A); random uses seed 0")
    ap.add_argument("--points", type=int, default=None,
                    help="colour/gmm: points per side (default the full workload; smaller sizes are for profiling)")
    ap.add_argument("--pairs", type=int, default=None,
                    help="docs/retrieval: number of pairs (default the full workload; smaller is for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rerank-k", type=int, default=None,
                    help="reduced precision: candidates re-ranked per consumer (default: the workload's)")
    args = ap.parse_args(argv)
    if args.steps is None:
        args.steps = WORKLOADS[args.workload].get("steps", 200)
    if args.impl == "reference" and args.protocol != "greedy":
        raise SystemExit("the reference arm times the greedy protocol")
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)
        acc = line.get("accuracy") or {}
        if acc.get("ok") is False:
            print(f"accuracy check failed: {acc}", file=sys.stderr, flush=True)
            sys.exit(3)


if __name__ == "__main__":
    main()
