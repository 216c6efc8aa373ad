#!/usr/bin/env python3
"""Benchmark of the Stream-K GEMM library on the shape-sweep workload.

Workload: 2,000 single BF16 GEMMs, m, n, k each log-uniform in [128, 8192] and
rounded to multiples of 16, inputs N(0,1) (seeded, generated on the device),
FP32 accumulation, BF16 output, alpha = 1, beta = 0 -- a synthetic stand-in for
the paper's 32,824-shape corpus (Section 6), which is not available.

One step runs all 2,000 GEMMs once.  Each step is a CUDA graph of the sk_gemm
launches with a timing event between consecutive GEMMs, so per-GEMM device
times carry no host launch overhead.  Three schedules of the same kernel are
timed: the two-tile Stream-K + data-parallel hybrid chosen by SK_MODE_AUTO
(the headline), data-parallel tiling and basic Stream-K.  `value` is the
geometric mean over shapes of TFLOP/s (2mnk / median per-GEMM time).

`e2e` repeats the headline schedule with, per GEMM, the host->device copy of A
and B from pinned host memory and the device->host copy of C inside the timed
region.  `cpu_baseline` times the FP64 oracle on the host cores on a bounded
sample of the same workload; the same sample checks the GPU outputs.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Geo-mean TFLOP/s & % tensor peak over shape sweep vs DP tiling; p99 latency"
UNIT = "TFLOP/s"
CPU_SAMPLE_SHAPES = 50        # every (2000 / 50)-th shape of the sweep
CPU_FLOPS_PER_SHAPE = 2e9     # oracle work per sampled shape


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--count", type=int, default=None, help="shapes in the sweep (default 2000)")
    ap.add_argument("--variants", default="auto,dp,sk,auto+indep",
                    help="schedules timed on the sweep; the first is the headline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-grouped", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-f8", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--serving-seconds", type=float, default=0.5,
                    help="seconds of Poisson arrivals per serving rate (the serving "
                         "configuration states 60 s; the default keeps the run short)")
    ap.add_argument("--serving-rates", default="2000,5000,20000,40000,50000",
                    help="comma-separated request rates of the serving workload")
    ap.add_argument("--dump-dir", default=None,
                    help="folder for per-shape detail and the clock log (default: "
                         "$SK_BENCH_DUMP_DIR, else a temporary folder)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]),
                "hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0,
                "source": "fallback"}


# DRAM bytes per flop of sk_gemm_kernel over the sweep, from one ncu launch
# list of the sweep's first shapes (dram__bytes_read.sum + dram__bytes_write.sum
# summed over the captured launches, divided by their 2mnk), and the sha256 of
# csrc/sk_kernel.cuh followed by csrc/planner.cpp at that capture.  The
# summary with its command is profiles/sk_gemm_sweep_launches.md.
PROFILED_TRAFFIC = {"dram_bytes_per_flop": 2.169549e-03,
                    "kernel_source_sha256":
                        "a9e83151ebf17b8fb1d37945f5ea29acdc7f7e7993a6ec75536351aadda4757e"}


def profiled_bytes_per_flop():
    """The profiled DRAM bytes per flop, or None when the kernel or planner
    source changed since the capture."""
    import hashlib
    h = hashlib.sha256()
    for f in ("sk_kernel.cuh", "planner.cpp"):
        with open(os.path.join(ROOT, "paper_2301_03598_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != PROFILED_TRAFFIC["kernel_source_sha256"]:
        return None
    return PROFILED_TRAFFIC["dram_bytes_per_flop"]


# Dense BF16 tcgen05 rate of one SM per clock: 8192 flops (the nominal 2.25
# PFLOP/s of a 148-SM part at 1.86 GHz).
FLOP_PER_CLK_PER_SM = 8192


def theoretical_peak(clocks):
    """Clock-derived dense BF16 tensor peak of this GPU: SMs x flops per SM
    per clock x the median SM clock under load (the maximum clock when no
    sample was taken)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    if clocks and clocks.get("sm_mhz"):
        mhz, which = float(clocks["sm_mhz"]), "median SM clock under load"
    else:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz = float(json.load(f)["sm_max_mhz"])
        except Exception:
            mhz = 2070.0
        which = "maximum SM clock"
    return {"tflops": sms * FLOP_PER_CLK_PER_SM * mhz * 1e6 / 1e12, "sms": sms,
            "flop_per_clk_per_sm": FLOP_PER_CLK_PER_SM, "sm_mhz": mhz, "clock": which}


def dump_dir():
    """Where per-shape detail and the clock log go: --dump-dir, else the
    SK_BENCH_DUMP_DIR environment variable, else a fresh temporary folder."""
    global _DUMP_DIR
    if _DUMP_DIR is None:
        import tempfile
        _DUMP_DIR = os.environ.get("SK_BENCH_DUMP_DIR") or tempfile.mkdtemp(prefix="sk_bench_")
        os.makedirs(_DUMP_DIR, exist_ok=True)
    return _DUMP_DIR


_DUMP_DIR = None


def geomean(x):
    x = np.asarray(x, np.float64)
    return float(np.exp(np.mean(np.log(x)))) if x.size else float("nan")


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = os.path.join(dump_dir(), f"clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- workload
from paper_2301_03598_gb300.sweep import (OUT_ELEMS, POOL_ELEMS, Sweep, _al,  # noqa: E402
                                          capture_step, event_overhead_us, reps_for, run_variant)


def make_plans(shapes, variant, ws_holder):
    """Plans of one bench variant: a schedule mode (auto, dp, sk, hybrid), with
    "+indep" the same plans declared to have independent inputs
    (SK_ATTR_INDEPENDENT_INPUTS: every GEMM of the sweep reads operands that no
    other GEMM writes, so a launch's MAC loop may overlap its predecessor)."""
    import torch
    from paper_2301_03598_gb300 import streamk as sk
    mode, _, extra = variant.partition("+")
    plans = [sk.sk_plan(m, n, k, "bf16", "bf16", "bf16", "f32", "row", "col", "row", mode)
             for (m, n, k) in shapes]
    if extra == "indep":
        for p in plans:
            p.set("independent_inputs", 1)
    elif extra:
        raise ValueError(f"unknown variant {variant}")
    need = max([p.get("workspace_bytes") for p in plans] + [4096])
    if ws_holder.get("ws") is None or ws_holder["ws"].numel() < need:
        ws_holder["ws"] = torch.empty(need, dtype=torch.uint8, device="cuda")
        ws_holder.setdefault("keep", []).append(ws_holder["ws"])  # earlier plans still use old
    for p in plans:
        sk.sk_plan_attach_workspace(p, ws_holder["ws"], ws_holder["ws"].numel())
    return plans


def run_e2e(plans, sweep, steps, warmup, barrier):
    """Per GEMM: H2D of A and B from pinned host memory, sk_gemm, D2H of C,
    pipelined over three streams inside one graph per step: the copies of
    GEMM i+1's inputs and of GEMM i-1's output overlap GEMM i, through two
    device buffers of each kind.  A timing event follows each D2H, so a
    GEMM's time is the interval between consecutive results reaching the
    host (for the first, from the step's start)."""
    import torch
    from paper_2301_03598_gb300 import streamk as sk
    shapes = sweep.shapes
    n = len(shapes)
    host_pool = torch.empty(POOL_ELEMS, dtype=torch.bfloat16, pin_memory=True)
    host_pool.copy_(sweep.pool)
    max_ab = max(_al(m * k) + _al(n_ * k) for (m, n_, k) in shapes)
    max_c = max(m * n_ for (m, n_, k) in shapes)
    dev_in = [torch.empty(max_ab, dtype=torch.bfloat16, device="cuda") for _ in range(2)]
    dev_out = [torch.empty(max_c, dtype=torch.bfloat16, device="cuda") for _ in range(2)]
    host_out = torch.empty(max_c, dtype=torch.bfloat16, pin_memory=True)
    h2d = d2h = 0
    main = torch.cuda.Stream()
    s_in, s_gemm, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def capture(count_bytes):
        nonlocal h2d, d2h
        g = torch.cuda.CUDAGraph()
        evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(n + 1)]
        loaded = [torch.cuda.Event() for _ in range(n)]
        done = [torch.cuda.Event() for _ in range(n)]
        copied = [torch.cuda.Event() for _ in range(n)]
        with torch.cuda.graph(g, stream=main):
            evs[0].record(main)
            for st in (s_in, s_gemm, s_out):
                st.wait_stream(main)
            for i in range(n):
                m, n_, k = shapes[i]
                ao, bo, _ = sweep.inst[i][0]
                buf_in, buf_out = dev_in[i % 2], dev_out[i % 2]
                if i >= 2:
                    s_in.wait_event(done[i - 2])      # GEMM i-2 has read this input buffer
                with torch.cuda.stream(s_in):
                    buf_in[:m * k].copy_(host_pool[ao:ao + m * k], non_blocking=True)
                    buf_in[_al(m * k):_al(m * k) + n_ * k].copy_(host_pool[bo:bo + n_ * k],
                                                                non_blocking=True)
                    loaded[i].record(s_in)
                s_gemm.wait_event(loaded[i])
                if i >= 2:
                    s_gemm.wait_event(copied[i - 2])  # D2H i-2 has read this output buffer
                sk.sk_gemm(plans[i], buf_in[:m * k], buf_in[_al(m * k):_al(m * k) + n_ * k],
                           buf_out, 1.0, 0.0, stream=s_gemm)
                done[i].record(s_gemm)
                s_out.wait_event(done[i])
                with torch.cuda.stream(s_out):
                    host_out[:m * n_].copy_(buf_out[:m * n_], non_blocking=True)
                    copied[i].record(s_out)
                    evs[i + 1].record(s_out)
                if count_bytes:
                    h2d += 2 * (m * k + n_ * k)
                    d2h += 2 * m * n_
            for st in (s_in, s_gemm, s_out):
                main.wait_stream(st)
        return g, evs

    graphs = [capture(s == 0) for s in range(steps + 1)]
    for _ in range(max(1, warmup)):
        graphs[0][0].replay()
    torch.cuda.synchronize()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for g, _ in graphs[1:]:
        g.replay()
    t1.record()
    torch.cuda.synchronize()
    barrier()
    per = np.asarray([[evs[i].elapsed_time(evs[i + 1]) for i in range(n)]
                      for _, evs in graphs[1:]])
    for p in plans:
        st, dev = sk.sk_last_error(p)
        if st != sk.SK_OK:
            raise RuntimeError(f"device status {st}/{dev} in the e2e region")
    return t0.elapsed_time(t1), per, h2d, d2h


# ----------------------------------------------------------------------------- oracle legs
def sample_blocks(shapes, count, flops_per_shape, seed):
    """Sampled output blocks (rows r0..r0+R, cols c0..c0+Cn) of every
    (len/count)-th shape, sized to about flops_per_shape of oracle work."""
    rng = np.random.Generator(np.random.PCG64(seed))
    stride = max(1, len(shapes) // count)
    out = []
    for i in range(0, len(shapes), stride)[:count]:
        m, n, k = shapes[i]
        entries = max(1, int(flops_per_shape // (2 * k)))
        R = max(1, min(m, int(math.sqrt(entries))))
        Cn = max(1, min(n, entries // R))
        r0 = int(rng.integers(0, m - R + 1))
        c0 = int(rng.integers(0, n - Cn + 1))
        out.append((i, r0, R, c0, Cn))
    return out


def time_oracle_blocks(blocks, operands, nthreads=0):
    """Time the oracle on each block.  operands[i] = (A_rows64, Bt_cols64).
    Returns per-block (seconds, flops, C64 block, |A||B| block)."""
    import oracle
    res = []
    for (i, r0, R, c0, Cn), (A64, Bt64) in zip(blocks, operands):
        k = A64.shape[1]
        rows = np.repeat(np.arange(R), Cn)
        cols = np.tile(np.arange(Cn), R)
        t = time.perf_counter()
        vals, absv = oracle.gemm_entries(rows, cols, A64, Bt64.T, nthreads=nthreads)
        dt = time.perf_counter() - t
        res.append((dt, 2.0 * k * R * Cn, vals.reshape(R, Cn), absv.reshape(R, Cn)))
    return res


def cpu_baseline_and_parity(shapes, sweep, plans, flops_per_shape):
    """Oracle timing on the host cores plus a full-size sampled parity check of
    the GPU outputs (same plans, same launch configuration)."""
    import torch
    import oracle
    from oracle import rounding
    from paper_2301_03598_gb300 import streamk as sk
    blocks = sample_blocks(shapes, CPU_SAMPLE_SHAPES, flops_per_shape, 2301_03598)
    operands, gpu_blocks = [], []
    for (i, r0, R, c0, Cn) in blocks:
        m, n, k = shapes[i]
        A = sweep.A(i).view(m, k)[r0:r0 + R].cpu().to(torch.float64).numpy()
        Bt = sweep.B(i).view(n, k)[c0:c0 + Cn].cpu().to(torch.float64).numpy()
        operands.append((A, Bt))
        C = torch.empty(m * n, dtype=torch.bfloat16, device="cuda")
        sk.sk_gemm(plans[i], sweep.A(i), sweep.B(i), C, 1.0, 0.0)
        st, dev = sk.sk_last_error(plans[i])
        if st != sk.SK_OK:
            raise RuntimeError(f"device status {st}/{dev} in the parity run")
        gpu_blocks.append(C.view(m, n)[r0:r0 + R, c0:c0 + Cn].cpu().to(torch.float64).numpy())
    threads = oracle.max_threads(0)
    res = time_oracle_blocks(blocks, operands)
    worst, bad, entries = 0.0, 0, 0
    for (blk, (dt, fl, C64, absAB), G) in zip(blocks, res, gpu_blocks):
        k = shapes[blk[0]][2]
        bnd = k * 2.0 ** -22 * absAB + rounding.ulp(C64, "bf16")
        err = np.abs(G - C64)
        worst = max(worst, float(np.max(err / bnd)))
        bad += int(np.sum(err > bnd))
        entries += G.size
    per_shape = [fl / dt / 1e12 for (dt, fl, _, _) in res]
    total_s = sum(r[0] for r in res)
    cpu = {"value": geomean(per_shape), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{len(blocks)} of {len(shapes)} sweep shapes (every "
                     f"{len(shapes) // len(blocks)}th), one output block of about "
                     f"{flops_per_shape:.0e} flops each, FP64 triple loop",
           "aggregate_tflops": sum(r[1] for r in res) / total_s / 1e12, "seconds": total_s}
    parity = {"shapes": len(blocks), "entries": entries, "violations": bad,
              "max_err_over_bound": worst,
              "bound": "k*2^-22*|A||B| + ulp_bf16(C64)"}
    return cpu, parity


# ----------------------------------------------------------------------------- arms
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_replicas(med, total_ms, flops, world, all_reduce_max=None):
    """Whole-job figures of `world` independent replicas (weak scaling): each
    shape's time and the step total are the maxima over ranks (the slowest
    replica sets the pace), and the value is the geo-mean TFLOP/s of those
    times times `world`.  all_reduce_max maps a float64 array to its
    elementwise maximum over ranks.  Returns (med, total_ms, value)."""
    med = np.asarray(med, np.float64)
    if world > 1:
        arr = np.asarray(all_reduce_max(np.append(med, total_ms)), np.float64)
        med, total_ms = arr[:-1], float(arr[-1])
    tflops = np.asarray(flops, np.float64) / (med * 1e-3) / 1e12
    return med, total_ms, geomean(tflops) * world


def reference_arm(args):
    """The oracle as the reference: FP64 CPU GEMM on a bounded sample per step."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2301_03598_gb300 import inputs
    import oracle
    import torch
    shapes = inputs.sweep_shapes(args.count or inputs.SWEEP_COUNT)
    blocks = sample_blocks(shapes, 20, 2.5e8, 7)
    operands = []
    for (i, r0, R, c0, Cn) in blocks:
        m, n, k = shapes[i]
        _, A64 = inputs.host_matrix(R, k, "bf16", "normal", 1000 + i)
        _, B64 = inputs.host_matrix(Cn, k, "bf16", "normal", 2000 + i)
        operands.append((A64, B64))
    for _ in range(args.warmup):
        time_oracle_blocks(blocks[:2], operands[:2])
    per_step = []
    t = time.perf_counter()
    for _ in range(args.steps):
        res = time_oracle_blocks(blocks, operands)
        per_step.append([fl / dt / 1e12 for (dt, fl, _, _) in res])
    elapsed = time.perf_counter() - t
    per_shape = np.median(np.asarray(per_step), axis=0)
    value = geomean(per_shape)
    cores = oracle.max_threads(0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "shape sweep: 2000 BF16 GEMMs, m,n,k log-uniform in "
                               "[128, 8192] (multiples of 16); reference = FP64 oracle on a "
                               "bounded sample", "sample_shapes": len(blocks)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{len(blocks)} sweep shapes, one output block of about "
                                   "2.5e8 flops each, per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def ours_arm(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        barrier = dist.barrier
    else:
        torch.cuda.set_device(0)

        def barrier():
            return None
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_03598_gb300 import inputs
    from paper_2301_03598_gb300 import streamk as sk

    shapes = inputs.sweep_shapes(args.count or inputs.SWEEP_COUNT)
    flops = np.array([2.0 * m * n * k for (m, n, k) in shapes])
    sweep = Sweep(shapes, torch.device("cuda", torch.cuda.current_device()),
                  seed=inputs.SWEEP_SEED + rank)
    ws = {}
    variants = [v for v in args.variants.split(",") if v]
    results = {}
    headline = None
    for v in variants:
        plans = make_plans(shapes, v, ws)
        sampler = ClockSampler(torch.cuda.current_device()) if v == variants[0] else None
        total_ms, step_ms, per, clocks = run_variant(plans, sweep, args.steps, args.warmup,
                                                     barrier, sampler)
        med = np.median(per, axis=0)                         # ms per GEMM
        tflops = flops / (med * 1e-3) / 1e12
        results[v] = {
            "geomean_tflops": geomean(tflops), "min_tflops": float(tflops.min()),
            "max_tflops": float(tflops.max()),
            "aggregate_tflops": float(flops.sum() / (med.sum() * 1e-3) / 1e12),
            "ms_per_step": float(np.mean(step_ms)),
            "p50_us": float(np.percentile(med * 1e3, 50)),
            "p99_us": float(np.percentile(med * 1e3, 99)),
            "_per_shape": tflops, "_med": med, "_plans": plans, "_clocks": clocks,
        }
        if headline is None:
            headline = v
    ev_us = event_overhead_us(torch.cuda.Stream())
    H = results[headline]
    plans = H["_plans"]
    peaks = load_peaks()
    peak = peaks["bf16_tflops_sustained"]

    # whole-job aggregation over replicas: per-shape max time over ranks
    def all_reduce_max(arr):
        import torch.distributed as dist
        t = torch.tensor(arr, dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.cpu().numpy()

    med, total_ms, value = aggregate_replicas(H["_med"], H["ms_per_step"] * args.steps, flops,
                                              world, all_reduce_max)
    tflops = flops / (med * 1e-3) / 1e12

    e2e = None
    if not args.no_e2e:
        e_ms, e_per, h2d, d2h = run_e2e(plans, sweep, args.steps, args.warmup, barrier)
        e_med = np.median(e_per, axis=0)
        e2e = {"value": geomean(flops / (e_med * 1e-3) / 1e12) * world, "unit": UNIT,
               "timing": "one graph per step: per GEMM H2D of A and B from pinned host memory, "
                         "sk_gemm, D2H of C (R = 1), pipelined over three streams with two "
                         "device buffers of each kind; per-GEMM time = interval between "
                         "consecutive D2H completions",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e_ms / args.steps,
               "aggregate_tflops": float(flops.sum() / (e_med.sum() * 1e-3) / 1e12)}

    cpu = parity = None
    if rank == 0 and not args.no_cpu:
        cpu, parity = cpu_baseline_and_parity(shapes, sweep, plans, CPU_FLOPS_PER_SHAPE)

    if rank != 0:
        return
    # per-shape detail for offline analysis
    with open(os.path.join(dump_dir(), "bench_per_shape.json"), "w") as f:
        json.dump({"shapes": shapes,
                   "plans": {v: [[p.get("tile_n"), p.get("grid"), p.get("sk_tiles"),
                                  p.get("mode")] for p in r["_plans"]]
                             for v, r in results.items()},
                   "us": {v: (r["_med"] * 1e3).tolist() for v, r in results.items()}}, f)
    kernel_ms = float(np.sum(H["_med"]))
    bpf = profiled_bytes_per_flop()
    theo = theoretical_peak(H["_clocks"])
    achieved = float(flops.sum() / (kernel_ms * 1e-3) / 1e12)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {
            "workload": "shape sweep: 2000 single BF16 GEMMs, m,n,k log-uniform in [128, 8192] "
                        "rounded to multiples of 16, N(0,1) inputs, FP32 accumulate, BF16 out, "
                        "alpha=1, beta=0",
            "shapes": len(shapes), "schedule": "auto (two-tile Stream-K + DP hybrid)",
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2: a 4 GiB input pool read in order, consecutive GEMMs "
                  "touch disjoint regions",
            "timing": "one CUDA graph per step; each shape runs R times back to back on fresh "
                      "operands (R = 16/8/4/2 by size) between two timing events; per-GEMM "
                      "time = interval / R",
            "event_node_us": ev_us,
        },
        "pct_of_peak": value / world / peak,
        "theoretical_peak": theo,
        "pct_of_theoretical_peak": value / world / theo["tflops"],
        "variants": {v: {kk: vv for kk, vv in r.items() if not kk.startswith("_")}
                     for v, r in results.items()},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (bpf * float(flops.mean())) if bpf is not None else None,
                     "traffic_unit": "DRAM bytes per launch (ncu launch list of the sweep's "
                                     "first shapes, scaled by flops)",
                     "kernel": "sk::sk_gemm_kernel", "peak_kind":
                     f"bf16 sustained ({peaks['source']})"},
        "gpu_launches": int(sum(sweep.reps) * args.steps),
        "e2e": e2e, "cpu_baseline": cpu, "parity": parity,
        "clocks": H["_clocks"],
    }
    if "dp" in results and headline != "dp":
        sp = results[headline]["_per_shape"] / results["dp"]["_per_shape"]
        line["speedup_vs_dp"] = {"avg": float(sp.mean()), "std": float(sp.std()),
                                 "min": float(sp.min()), "max": float(sp.max()),
                                 "geomean": geomean(sp)}
        line["vs_dp_geomean"] = results[headline]["geomean_tflops"] / \
            results["dp"]["geomean_tflops"]
        # where both schedules are the same plan the ratio is run-to-run noise
        # of one plan; the shapes whose plans differ show the planner's choice
        key = lambda p: (p.get("tile_n"), p.get("cluster_m"), p.get("grid"), p.get("sk_tiles"))
        differ = np.array([key(a) != key(b) for a, b in zip(results[headline]["_plans"],
                                                          results["dp"]["_plans"])])
        if differ.any():
            spd = sp[differ]
            line["speedup_vs_dp"]["plans_differ"] = {
                "shapes": int(differ.sum()), "geomean": geomean(spd), "min": float(spd.min()),
                "below_0.95": int((spd < 0.95).sum())}
        same = sp[~differ]
        if same.size:
            line["speedup_vs_dp"]["same_plan_spread"] = {
                "shapes": int(same.size), "min": float(same.min()), "max": float(same.max())}
    if "auto+indep" in results and headline == "auto":
        sp = results["auto+indep"]["_per_shape"] / results["auto"]["_per_shape"]
        line["independent_inputs"] = {
            "what": "the headline's plans with SK_ATTR_INDEPENDENT_INPUTS (opt-in, off by "
                    "default): operand loads and the MAC loop overlap the previous launch, "
                    "C and workspace accesses keep stream order; not the headline",
            "geomean_tflops": results["auto+indep"]["geomean_tflops"],
            "speedup_vs_default": {"geomean": geomean(sp), "min": float(sp.min()),
                                   "max": float(sp.max())}}
    if not args.no_grouped:
        line["grouped"] = run_grouped(max(3, min(args.steps, 10)), args.warmup)
    if not args.no_configs:
        line["config_shapes"] = run_config_shapes(peaks)
    if not args.no_f8:
        line["grouped_e4m3"] = run_grouped_f8(max(3, min(args.steps, 10)), args.warmup)
        line["e4m3_shapes"] = run_f8_shapes(peaks)
    if not args.no_serving:
        line["serving"] = run_serving(
            rates=tuple(int(r) for r in args.serving_rates.split(",") if r),
            seconds=args.serving_seconds)
    print(json.dumps(line), flush=True)


def grouped_schedules(gplan, launch, steps, warmup, stream, flops):
    """The same grouped launch under each schedule of the concatenated
    iteration space, each forced in turn: data-parallel waves, the two-tile
    hybrid (Stream-K over the first (t mod p) + p tiles) and basic Stream-K
    (one even split of all iterations).  Restores the plan's mode."""
    import torch
    from paper_2301_03598_gb300 import streamk as sk
    saved = gplan.get("mode")
    out = {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for name in ("dp", "hybrid", "sk"):
        gplan.set("mode", sk.MODES[name])
        with torch.cuda.stream(stream):
            for _ in range(max(1, warmup)):
                launch()
            ev[0].record(stream)
            for _ in range(steps):
                launch()
            ev[1].record(stream)
        torch.cuda.synchronize()
        st, dstat = sk.sk_grouped_last_error(gplan)
        if st != sk.SK_OK:
            raise RuntimeError(f"grouped {name} status {st}/{dstat}")
        ms = ev[0].elapsed_time(ev[1]) / steps
        info = gplan.info()
        out[name] = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                     "plan": {k: info[k] for k in ("tile_n", "cluster_m", "grid", "tiles",
                                                   "sk_tiles", "workspace_bytes")}}
    gplan.set("mode", saved)
    return out


def run_grouped(steps, warmup):
    """The grouped workload (256 problems, see inputs.grouped_shapes) as one
    autotuned Stream-K launch across all problems (tile width, cluster size,
    schedule and pipeline depth measured; the model's own pick is reported
    beside it), against the same 256 GEMMs as separate launches of the
    single-GEMM path replayed from one CUDA graph.  Inputs are
    device-resident; each problem has its own A, B and C."""
    import torch
    from paper_2301_03598_gb300 import inputs
    from paper_2301_03598_gb300 import streamk as sk
    shapes = inputs.grouped_shapes()
    dev = torch.device("cuda", torch.cuda.current_device())
    As, Bs, Cs = [], [], []
    for i, (m, n, k) in enumerate(shapes):
        As.append(inputs.device_pool(m * k, "bf16", "normal", inputs.GROUPED_SEED + 3 * i, dev).view(m, k))
        Bs.append(inputs.device_pool(n * k, "bf16", "normal", inputs.GROUPED_SEED + 3 * i + 1, dev).view(n, k))
        Cs.append(torch.empty(m, n, dtype=torch.bfloat16, device=dev))
    flops = float(sum(2.0 * m * n * k for m, n, k in shapes))
    stream = torch.cuda.Stream()
    gplan = sk.sk_grouped_plan(shapes, "bf16", "bf16", "auto")
    model_plan = gplan.info()
    tuned_us = sk.sk_grouped_autotune(gplan, As, Bs, Cs, reps=3, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        for _ in range(max(1, warmup)):
            sk.sk_grouped_gemm(gplan, As, Bs, Cs, stream=stream)
        ev[0].record(stream)
        for _ in range(steps):
            sk.sk_grouped_gemm(gplan, As, Bs, Cs, stream=stream)
        ev[1].record(stream)
    torch.cuda.synchronize()
    st, dstat = sk.sk_grouped_last_error(gplan)
    if st != sk.SK_OK:
        raise RuntimeError(f"grouped launch status {st}/{dstat}")
    g_ms = ev[0].elapsed_time(ev[1]) / steps
    ginfo = gplan.info()
    scheds = grouped_schedules(gplan, lambda: sk.sk_grouped_gemm(gplan, As, Bs, Cs, stream=stream),
                               steps, warmup, stream, flops)
    # the same problems as separate plans, one graph of 256 launches per step
    plans = make_plans(shapes, "auto", {})
    ws_keep = [p._workspace for p in plans]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        for p, A, B, C in zip(plans, As, Bs, Cs):
            sk.sk_gemm(p, A, B, C, stream=stream)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            for p, A, B, C in zip(plans, As, Bs, Cs):
                sk.sk_gemm(p, A, B, C)
        for _ in range(max(1, warmup)):
            graph.replay()
        ev[0].record(stream)
        for _ in range(steps):
            graph.replay()
        ev[1].record(stream)
    torch.cuda.synchronize()
    for p in plans:
        st, dstat = sk.sk_last_error(p)
        if st != sk.SK_OK:
            raise RuntimeError(f"separate launch status {st}/{dstat}")
    s_ms = ev[0].elapsed_time(ev[1]) / steps
    del ws_keep
    for p in plans:
        p.destroy()
    gplan.destroy()
    return {
        "workload": "grouped GEMM: 256 problems, m log-uniform in [16, 4096] (multiples of 16), "
                    "n, k uniform from {1024, 2048, 4096, 8192}, BF16 in (a stand-in for the "
                    "FP8-e4m3 inputs of the grouped configuration), FP32 accumulate, BF16 out",
        "problems": len(shapes), "gflop": flops / 1e9,
        "grouped": {"ms": g_ms, "tflops": flops / (g_ms * 1e-3) / 1e12, "launches_per_step": 1,
                    "autotune_best_us": tuned_us,
                    "plan": {k: ginfo[k] for k in ("mode", "tile_n", "cluster_m", "grid", "tiles",
                                                   "sk_tiles", "stages")},
                    "model_plan": {k: model_plan[k] for k in ("mode", "tile_n", "cluster_m",
                                                              "grid", "sk_tiles")}},
        "schedules": scheds,
        "separate": {"ms": s_ms, "tflops": flops / (s_ms * 1e-3) / 1e12,
                     "launches_per_step": len(shapes),
                     "timing": "the 256 single-GEMM launches replayed from one CUDA graph"},
        "speedup": s_ms / g_ms,
    }


def run_grouped_f8(steps, warmup):
    """The grouped workload with E4M3 operands (per-128 x 128-block FP32 scales,
    values N(0,1) before quantisation), BF16 out: one autotuned Stream-K
    launch across the 256 problems against 256 separate sk_gemm_scaled
    launches replayed from one CUDA graph."""
    import torch
    from paper_2301_03598_gb300 import inputs
    from paper_2301_03598_gb300 import streamk as sk
    shapes = inputs.grouped_shapes()
    dev = torch.device("cuda", torch.cuda.current_device())
    As, Bs, SAs, SBs, Cs = [], [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        qa, sa = inputs.device_e4m3_matrix(m, k, inputs.GROUPED_SEED + 3 * i, dev)
        qb, sb = inputs.device_e4m3_matrix(n, k, inputs.GROUPED_SEED + 3 * i + 1, dev)
        As.append(qa)
        Bs.append(qb)
        SAs.append(sa)
        SBs.append(sb)
        Cs.append(torch.empty(m, n, dtype=torch.bfloat16, device=dev))
    flops = float(sum(2.0 * m * n * k for m, n, k in shapes))
    stream = torch.cuda.Stream()
    gplan = sk.sk_grouped_plan(shapes, "e4m3", "bf16", "auto")
    tuned_us = sk.sk_grouped_autotune_scaled(gplan, As, Bs, SAs, SBs, Cs, reps=3, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        for _ in range(max(1, warmup)):
            sk.sk_grouped_gemm_scaled(gplan, As, Bs, SAs, SBs, Cs, stream=stream)
        ev[0].record(stream)
        for _ in range(steps):
            sk.sk_grouped_gemm_scaled(gplan, As, Bs, SAs, SBs, Cs, stream=stream)
        ev[1].record(stream)
    torch.cuda.synchronize()
    st, dstat = sk.sk_grouped_last_error(gplan)
    if st != sk.SK_OK:
        raise RuntimeError(f"grouped e4m3 launch status {st}/{dstat}")
    g_ms = ev[0].elapsed_time(ev[1]) / steps
    ginfo = gplan.info()
    scheds = grouped_schedules(
        gplan, lambda: sk.sk_grouped_gemm_scaled(gplan, As, Bs, SAs, SBs, Cs, stream=stream),
        steps, warmup, stream, flops)
    plans = [sk.sk_plan(m, n, k, "e4m3", "e4m3", "bf16") for m, n, k in shapes]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        for args in zip(plans, As, Bs, SAs, SBs, Cs):
            sk.sk_gemm_scaled(*args, stream=stream)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            for args in zip(plans, As, Bs, SAs, SBs, Cs):
                sk.sk_gemm_scaled(*args)
        for _ in range(max(1, warmup)):
            graph.replay()
        ev[0].record(stream)
        for _ in range(steps):
            graph.replay()
        ev[1].record(stream)
    torch.cuda.synchronize()
    for p in plans:
        st, dstat = sk.sk_last_error(p)
        if st != sk.SK_OK:
            raise RuntimeError(f"separate e4m3 launch status {st}/{dstat}")
    s_ms = ev[0].elapsed_time(ev[1]) / steps
    for p in plans:
        p.destroy()
    gplan.destroy()
    return {
        "workload": "grouped GEMM: the 256 problems of the grouped workload, FP8-e4m3 A and B "
                    "with per-128x128-block FP32 scales (N(0,1) before quantisation), FP32 "
                    "accumulate, BF16 out",
        "problems": len(shapes), "gflop": flops / 1e9,
        "grouped": {"ms": g_ms, "tflops": flops / (g_ms * 1e-3) / 1e12, "launches_per_step": 1,
                    "autotune_best_us": tuned_us,
                    "plan": {k: ginfo[k] for k in ("mode", "tile_n", "grid", "tiles", "sk_tiles",
                                                   "stages")}},
        "schedules": scheds,
        "separate": {"ms": s_ms, "tflops": flops / (s_ms * 1e-3) / 1e12,
                     "launches_per_step": len(shapes),
                     "timing": "the 256 sk_gemm_scaled launches replayed from one CUDA graph"},
        "speedup": s_ms / g_ms,
    }


F8_SHAPES = [(8192, 8192, 8192), (4096, 4096, 4096), (2048, 2048, 8192), (384, 384, 4096),
             (256, 256, 65536)]


SHAPE_ROUNDS = 7


def _shape_reps(m, n, k):
    """Back-to-back launches in one timed replay of a single shape: about a
    millisecond of work for the largest shapes, at least ~150 us for the
    smallest, so the timing events' own cost stays near 1%."""
    fl = 2.0 * m * n * k
    return 32 if fl < 1e10 else 8 if fl < 1e11 else 2


def _graph_times_us(launches, reps, stream, rounds=SHAPE_ROUNDS):
    """Per-launch device time (us) of each callable in `launches`: each is
    captured `reps` times back to back into its own CUDA graph, all graphs are
    replayed once to warm up, then `rounds` times in turn (one replay of each
    per round, between two events on the launching stream), so a drift of the
    clock or power state over the measurement reaches every arm alike.
    Returns the median over rounds per callable."""
    import torch
    graphs = []
    with torch.cuda.stream(stream):
        for fn in launches:
            for _ in range(3):
                fn()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for _ in range(reps):
                    fn()
            graphs.append(g)
        for g in graphs:
            g.replay()
        evs = []
        for _ in range(rounds):
            row = []
            for g in graphs:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.replay()
                e1.record(stream)
                row.append((e0, e1))
            evs.append(row)
    torch.cuda.synchronize()
    out = [float(np.median([evs[r][i][0].elapsed_time(evs[r][i][1]) for r in range(rounds)]))
           * 1e3 / reps for i in range(len(graphs))]
    del graphs
    return out


def run_f8_shapes(peaks):
    """Single E4M3 GEMMs (AUTO plans, BF16 out), each timed as the median over
    rounds of one CUDA-graph replay of back-to-back launches after warm-up
    (_graph_times_us); TFLOP/s against the FP8 peak taken as twice the measured
    BF16 burst peak (the nominal dense ratio)."""
    import torch
    from paper_2301_03598_gb300 import inputs
    from paper_2301_03598_gb300 import streamk as sk
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"peak_tflops": 2.0 * peaks["bf16_tflops"],
           "peak_kind": "2 x bf16 burst (" + peaks["source"] + ")",
           "timing": f"median of {SHAPE_ROUNDS} graph replays of back-to-back launches", "shapes": []}
    stream = torch.cuda.Stream()
    for (m, n, k) in F8_SHAPES:
        qa, sa = inputs.device_e4m3_matrix(m, k, 77, dev)
        qb, sb = inputs.device_e4m3_matrix(n, k, 78, dev)
        C = torch.empty(m, n, dtype=torch.bfloat16, device=dev)
        plan = sk.sk_plan(m, n, k, "e4m3", "e4m3", "bf16")
        reps = _shape_reps(m, n, k)
        (us,) = _graph_times_us(
            [lambda: sk.sk_gemm_scaled(plan, qa, qb, sa, sb, C, stream=stream)], reps, stream)
        st, dstat = sk.sk_last_error(plan)
        if st != sk.SK_OK:
            raise RuntimeError(f"e4m3 {m}x{n}x{k} status {st}/{dstat}")
        tf = 2.0 * m * n * k / (us * 1e-6) / 1e12
        info = plan.info()
        out["shapes"].append({"m": m, "n": n, "k": k, "us": us, "tflops": tf, "reps": reps,
                              "frac_of_peak": tf / out["peak_tflops"],
                              "plan": {x: info[x] for x in ("mode", "grid", "tiles", "sk_tiles")}})
        plan.destroy()
        del qa, qb, sa, sb, C
    return out


CONFIG_SHAPES = [("single GEMM, FP16 in U[-1,1], FP32 out, beta = 0", "f16", "f32", 0.0,
                  [(384, 384, 4096)]),
                 ("extreme shapes, BF16 in N(0,1), BF16 out, beta = 0.5 with random C", "bf16",
                  "bf16", 0.5, [(8192, 8192, 8192), (256, 256, 65536), (8192, 128, 4096),
                                (1536, 1536, 1536)])]


def run_config_shapes(peaks):
    """The single-GEMM and extreme-shape workloads under each schedule (DP
    tiling, basic Stream-K at the modelled grid, the two-tile hybrid, AUTO).
    The four plans of a shape are timed together by _graph_times_us: one CUDA
    graph of back-to-back launches each (no host launch cost between them),
    replayed in turn over several rounds after warm-up, median per plan, on the
    same operands (only 8192^3's exceed the L2).  TFLOP/s against the measured
    BF16 burst peak and against the shape's attainable roofline
    min(peak, AI x HBM bandwidth), AI = flops / (A + B read, C read if beta != 0,
    C written)."""
    import torch
    from paper_2301_03598_gb300 import inputs
    from paper_2301_03598_gb300 import streamk as sk
    dev = torch.device("cuda", torch.cuda.current_device())
    peak, bw = peaks["bf16_tflops"], peaks["hbm_gbs"]
    out = {"peak_tflops": peak, "peak_kind": "bf16 burst (" + peaks["source"] + ")",
           "hbm_gbs": bw, "l2": "operands reused across the timed launches; only 8192^3 "
                               "exceeds the L2",
           "timing": f"median of {SHAPE_ROUNDS} rounds, each one graph replay of back-to-back "
                     "launches per schedule in turn", "configs": []}
    stream = torch.cuda.Stream()
    modes = ("dp", "sk", "hybrid", "auto")
    for what, ab, c_type, beta, shapes in CONFIG_SHAPES:
        dist = "uniform" if ab == "f16" else "normal"
        rows = []
        for (m, n, k) in shapes:
            A = inputs.device_pool(m * k, ab, dist, 91, dev).view(m, k)
            B = inputs.device_pool(n * k, ab, dist, 92, dev).view(n, k)
            C = (inputs.device_pool(m * n, c_type, "normal", 93, dev).view(m, n) if beta
                 else torch.zeros(m, n, dtype=inputs.DTYPES[c_type], device=dev))
            flops = 2.0 * m * n * k
            cb = C.element_size() * m * n
            nbytes = A.element_size() * (m * k + n * k) + cb * (2 if beta else 1)
            attainable = min(peak, flops / nbytes * bw / 1e3)
            reps = _shape_reps(m, n, k)
            row = {"m": m, "n": n, "k": k, "gflop": flops / 1e9, "mbytes": nbytes / 1e6,
                   "attainable_tflops": attainable, "reps": reps, "modes": {}}
            plans = [sk.sk_plan(m, n, k, ab, ab, c_type, mode=mode) for mode in modes]
            times = _graph_times_us(
                [lambda p=p: sk.sk_gemm(p, A, B, C, 1.0, beta, stream=stream) for p in plans],
                reps, stream)
            for mode, plan, us in zip(modes, plans, times):
                st, dstat = sk.sk_last_error(plan)
                if st != sk.SK_OK:
                    raise RuntimeError(f"{m}x{n}x{k} {mode} status {st}/{dstat}")
                tf = flops / (us * 1e-6) / 1e12
                info = plan.info()
                row["modes"][mode] = {"us": us, "tflops": tf, "frac_of_peak": tf / peak,
                                      "frac_of_attainable": tf / attainable,
                                      "plan": {x: info[x] for x in (
                                          "mode", "tile_n", "cluster_m", "grid", "tiles",
                                          "sk_tiles")}}
                plan.destroy()
            rows.append(row)
            del A, B, C
        out["configs"].append({"workload": what, "shapes": rows})
    return out


def _plain_launches(sk, launch, plans, arrivals, pick):
    """One launch per request at its arrival time on one stream; returns the
    arrival-to-completion latencies (us) and the wall time of the run."""
    import collections
    import torch
    s = torch.cuda.Stream()
    for j in range(8):   # warm the launch path
        launch(j % len(plans), j % 2, s)
    torch.cuda.synchronize()
    pend, lats = collections.deque(), []
    t0 = time.perf_counter()
    for a_t, (j, d) in zip(arrivals, pick):
        while True:
            now = time.perf_counter() - t0
            while pend and pend[0][0].query():
                lats.append((now - pend.popleft()[1]) * 1e6)
            if now >= a_t:
                break
        launch(j, d, s)
        ev = torch.cuda.Event()
        ev.record(s)
        pend.append((ev, a_t))
    while pend:
        now = time.perf_counter() - t0
        while pend and pend[0][0].query():
            lats.append((now - pend.popleft()[1]) * 1e6)
    wall = time.perf_counter() - t0
    for pair in plans:
        for p in pair:
            st, dev_st = sk.sk_last_error(p)
            if st != sk.SK_OK or dev_st != 0:
                raise RuntimeError(f"plain launch status {st}, device status {dev_st}")
    return np.array(lats), wall


def run_serving(rates=(2000, 5000, 20000, 40000, 50000), seconds=0.5, seed=2301_03598 + 5, slots=4,
                max_batch=64):
    """The serving workload: requests arrive as a Poisson process at each rate
    for `seconds`, each a GEMM drawn from 64 shapes (48 from the shape sweep's
    distribution, 16 from the grouped workload's), half of them BF16 and half
    block-scaled E4M3 (chosen per request), FP32 accumulate, BF16 out.  The
    continuous-batching server (batches of up to 64 requests of one input
    type, 4 concurrent launch slots, 64 GB admission budget) against two
    baselines: the same server with batches of one on one slot, and plain
    launches, one `sk_gemm` / `sk_gemm_scaled` per request on arrival from
    plans made per shape beforehand, on one stream, completion seen by
    polling an event recorded after each launch.  Latency: arrival to
    observed completion."""
    import torch
    from paper_2301_03598_gb300 import inputs
    from paper_2301_03598_gb300 import streamk as sk
    rng = np.random.default_rng(seed)
    sw, gr = inputs.sweep_shapes(), inputs.grouped_shapes()
    shapes = [sw[i] for i in rng.choice(len(sw), 48, replace=False)] + \
             [gr[i] for i in rng.choice(len(gr), 16, replace=False)]
    dev = torch.device("cuda", torch.cuda.current_device())
    ops = []
    for i, (m, n, k) in enumerate(shapes):
        qa, sa = inputs.device_e4m3_matrix(m, k, seed + 3 * i + 2, dev)
        qb, sb = inputs.device_e4m3_matrix(n, k, seed + 3 * i + 3, dev)
        ops.append((inputs.device_pool(m * k, "bf16", "normal", seed + 3 * i, dev).view(m, k),
                    inputs.device_pool(n * k, "bf16", "normal", seed + 3 * i + 1, dev).view(n, k),
                    qa, qb, sa, sb, torch.empty(m, n, dtype=torch.bfloat16, device=dev)))
    flops = np.array([2.0 * m * n * k for m, n, k in shapes])
    plans = [(sk.sk_plan(m, n, k, "bf16", "bf16", "bf16"), sk.sk_plan(m, n, k, "e4m3", "e4m3", "bf16"))
             for m, n, k in shapes]

    def submit(srv, j, d):
        A, B, qa, qb, sa, sb, C = ops[j]
        return srv.submit(A, B, C) if d == 0 else srv.submit_scaled(qa, qb, sa, sb, C)

    def launch(j, d, stream):
        A, B, qa, qb, sa, sb, C = ops[j]
        if d == 0:
            sk.sk_gemm(plans[j][0], A, B, C, stream=stream)
        else:
            sk.sk_gemm_scaled(plans[j][1], qa, qb, sa, sb, C, stream=stream)

    out = {"workload": "Poisson arrivals of single GEMMs, shapes drawn from 48 shapes of the "
                       "sweep distribution and 16 of the grouped workload's, half BF16 and half "
                       "FP8-e4m3 with per-128x128-block FP32 scales, FP32 accumulate, BF16 out",
           "seconds_per_rate": seconds, "rates": {}}
    for rate in rates:
        n_req = int(rate * seconds)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
        pick = list(zip(rng.integers(0, len(shapes), size=n_req).tolist(),
                        rng.integers(0, 2, size=n_req).tolist()))
        req_flops = float(sum(flops[j] for j, _ in pick))
        res = {}
        for name, mb, ns in (("server", max_batch, slots), ("per_request", 1, 1)):
            srv = sk.sk_server_create("bf16", "bf16", max_batch=mb, slots=ns,
                                      hbm_budget_bytes=64 << 30)
            try:
                # warm the launch path: every shape and input type once, alone
                # (the plain arm below plans every shape before timing too)
                for j in range(len(shapes)):
                    for d in (0, 1):
                        srv.wait(submit(srv, j, d))
                torch.cuda.synchronize()
                tickets = []
                t0 = time.perf_counter()
                for a_t, (j, d) in zip(arrivals, pick):
                    while time.perf_counter() - t0 < a_t:
                        pass
                    tickets.append(submit(srv, j, d))
                lats = []
                for t in tickets:
                    st, lat = srv.wait(t)
                    if st != sk.SK_OK:
                        raise RuntimeError(f"served request status {st}")
                    lats.append(lat)
                wall = time.perf_counter() - t0
                stats = srv.stats()
            finally:
                srv.destroy()
            lats = np.array(lats)
            # throughput over the span from the first arrival to the last
            # completion (arrival + latency), the same for every arm; `wall`
            # also holds the harness's wait calls after the last submission
            span = float(np.max(arrivals + lats * 1e-6))
            res[name] = {"p50_us": float(np.percentile(lats, 50)),
                         "p99_us": float(np.percentile(lats, 99)),
                         "mean_us": float(lats.mean()),
                         "requests_per_s": n_req / span,
                         "tflops": req_flops / span / 1e12,
                         "harness_wall_s": wall,
                         "batches": stats["batches"] - 2 * len(shapes),
                         "largest_batch": stats["max_batch"]}
        lats, wall = _plain_launches(sk, launch, plans, arrivals, pick)
        span = float(np.max(arrivals + lats * 1e-6))   # completions come in arrival order
        res["plain_launch"] = {"p50_us": float(np.percentile(lats, 50)),
                               "p99_us": float(np.percentile(lats, 99)),
                               "mean_us": float(lats.mean()),
                               "requests_per_s": n_req / span,
                               "tflops": req_flops / span / 1e12,
                               "harness_wall_s": wall}
        res["p99_speedup"] = res["per_request"]["p99_us"] / res["server"]["p99_us"]
        res["p99_speedup_vs_plain"] = res["plain_launch"]["p99_us"] / res["server"]["p99_us"]
        out["rates"][str(rate)] = res
    out["throughput"] = ("requests / (last completion - first arrival); completion = arrival + "
                         "latency, so all arms count the same span")
    for pair in plans:
        for p in pair:
            p.destroy()
    return out


def main():
    global _DUMP_DIR
    args = parse_args()
    if args.dump_dir:
        _DUMP_DIR = args.dump_dir
        os.makedirs(_DUMP_DIR, exist_ok=True)
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
