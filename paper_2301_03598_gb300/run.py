"""Run GEMMs through the C ABI from the command line.

    python -m paper_2301_03598_gb300.run M N K [--mode auto] [--reps 20] ...
    python -m paper_2301_03598_gb300.run --sweep 120 [--mode auto]
    python -m paper_2301_03598_gb300.run --grouped 32 [--dtype e4m3] [--mode auto]

The first form plans one problem, runs it ``--reps`` times back to back on the
current stream and prints the plan and the mean time per GEMM (CUDA events,
after ``--warmup`` untimed runs).  The second runs the first N shapes of the
2,000-shape log-uniform BF16 sweep once each, every shape on operands of its
own, and prints the total time.  The third runs the first N problems of the
grouped workload as one grouped launch, ``--reps`` times.  All end by reading
the plan's status and exit non-zero on any error, so they serve as the
command under a profiler.
Operands are seeded Philox normals on the device; with ``--dtype e4m3`` they
are quantised to E4M3 with one FP32 scale per 128 x 128 block and run through
``sk_gemm_scaled``.
"""
from __future__ import annotations

import argparse
import json
import sys

import torch

from . import inputs
from . import streamk as sk


def _operands(m, n, k, ab, c, seed, device):
    C = torch.zeros(m, n, dtype=inputs.DTYPES[c], device=device)
    if ab == "e4m3":
        A, sA = inputs.device_e4m3_matrix(m, k, seed, device)
        B, sB = inputs.device_e4m3_matrix(n, k, seed + 1, device)
        return A, B, C, (sA, sB)
    A = inputs.device_pool(m * k, ab, "normal", seed, device).view(m, k)
    B = inputs.device_pool(n * k, ab, "normal", seed + 1, device).view(n, k)
    return A, B, C, None


def _gemm(plan, A, B, C, scales, args):
    if scales is None:
        sk.sk_gemm(plan, A, B, C, args.alpha, args.beta)
    else:
        sk.sk_gemm_scaled(plan, A, B, scales[0], scales[1], C, args.alpha, args.beta)


def _plan(m, n, k, args):
    p = sk.sk_plan(m, n, k, args.dtype, args.dtype, args.out, mode=args.mode)
    for name in ("tile_n", "grid", "cluster_m", "raster_group"):
        v = getattr(args, name)
        if v:
            p.set(name, v)
    return p


def _check(plan):
    st, dev = sk.sk_last_error(plan)
    if st != sk.SK_OK:
        raise sk.StreamKError(st, f"sk_gemm (device status {dev})")


def run_one(args, device):
    m, n, k = args.shape
    A, B, C, sc = _operands(m, n, k, args.dtype, args.out, args.seed, device)
    plan = _plan(m, n, k, args)
    for _ in range(args.warmup):
        _gemm(plan, A, B, C, sc, args)
    s = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    e0.record(s)
    for _ in range(args.reps):
        _gemm(plan, A, B, C, sc, args)
    e1.record(s)
    torch.cuda.synchronize(device)
    _check(plan)
    us = e0.elapsed_time(e1) * 1e3 / max(1, args.reps)
    info = plan.info()
    print(json.dumps({"m": m, "n": n, "k": k, "us_per_gemm": us,
                      "tflops": 2.0 * m * n * k / us / 1e6 if us > 0 else None,
                      "plan": {key: info[key] for key in (
                          "mode", "tile_n", "grid", "ctas", "cluster_m", "tiles",
                          "iters_per_tile", "sk_tiles", "dp_tiles", "raster_group")}}))


def run_sweep(args, device):
    shapes = inputs.sweep_shapes()[: args.sweep]
    plans, ops = [], []
    for i, (m, n, k) in enumerate(shapes):
        plans.append(_plan(m, n, k, args))
        ops.append(_operands(m, n, k, args.dtype, args.out, args.seed + 2 * i, device))
    for _ in range(args.warmup):
        for p, (A, B, C, sc) in zip(plans, ops):
            _gemm(p, A, B, C, sc, args)
    s = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    e0.record(s)
    for p, (A, B, C, sc) in zip(plans, ops):
        _gemm(p, A, B, C, sc, args)
    e1.record(s)
    torch.cuda.synchronize(device)
    for p in plans:
        _check(p)
    flops = sum(2.0 * m * n * k for m, n, k in shapes)
    ms = e0.elapsed_time(e1)
    print(json.dumps({"shapes": len(shapes), "ms": ms, "flops": flops,
                      "tflops": flops / ms / 1e9 if ms > 0 else None}))


def run_grouped(args, device):
    shapes = inputs.grouped_shapes()[: args.grouped]
    ops = [_operands(m, n, k, args.dtype, args.out, args.seed + 2 * i, device)
           for i, (m, n, k) in enumerate(shapes)]
    plan = sk.sk_grouped_plan(shapes, args.dtype, args.out, args.mode)
    As, Bs, Cs = [o[0] for o in ops], [o[1] for o in ops], [o[2] for o in ops]

    def launch():
        if args.dtype == "e4m3":
            sk.sk_grouped_gemm_scaled(plan, As, Bs, [o[3][0] for o in ops], [o[3][1] for o in ops],
                                      Cs)
        else:
            sk.sk_grouped_gemm(plan, As, Bs, Cs)

    for _ in range(args.warmup):
        launch()
    s = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    e0.record(s)
    for _ in range(args.reps):
        launch()
    e1.record(s)
    torch.cuda.synchronize(device)
    st, dev = sk.sk_grouped_last_error(plan)
    if st != sk.SK_OK:
        raise sk.StreamKError(st, f"sk_grouped_gemm (device status {dev})")
    us = e0.elapsed_time(e1) * 1e3 / max(1, args.reps)
    flops = sum(2.0 * m * n * k for m, n, k in shapes)
    print(json.dumps({"problems": len(shapes), "us_per_launch": us,
                      "tflops": flops / us / 1e6 if us > 0 else None, "plan": plan.info()}))
    plan.destroy()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("shape", nargs="*", type=int, help="M N K")
    ap.add_argument("--sweep", type=int, default=0, help="run the first N sweep shapes")
    ap.add_argument("--grouped", type=int, default=0,
                    help="run the first N grouped-workload problems as one grouped launch")
    ap.add_argument("--mode", default="auto", choices=sorted(sk.MODES))
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "f16", "e4m3"])
    ap.add_argument("--out", default="bf16", choices=["bf16", "f16", "f32"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--tile-n", dest="tile_n", type=int, default=0)
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--cluster-m", dest="cluster_m", type=int, default=0)
    ap.add_argument("--raster-group", dest="raster_group", type=int, default=0)
    ap.add_argument("--alpha", type=float, default=1.0)
    ap.add_argument("--beta", type=float, default=0.0)
    ap.add_argument("--seed", type=int, default=2301_03598)
    args = ap.parse_args(argv)
    if not args.sweep and not args.grouped and len(args.shape) != 3:
        ap.error("give M N K, --sweep N or --grouped N")
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    device = torch.device("cuda", torch.cuda.current_device())
    if args.sweep:
        run_sweep(args, device)
    elif args.grouped:
        run_grouped(args, device)
    else:
        run_one(args, device)
    return 0


if __name__ == "__main__":
    sys.exit(main())
