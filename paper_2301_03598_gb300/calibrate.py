"""Recalibrate the planner's time model on this GPU.

    python -m paper_2301_03598_gb300.calibrate measure --out DIR [--count N]
    python -m paper_2301_03598_gb300.calibrate fit DIR/calibration.json

The model SK_MODE_AUTO ranks its candidates by is Appendix A.1's
time_CTA = a + b*[split] + c*iterations + d*(peers - 1), extended by e per tile
segment and f, the shortest period of consecutive whole tiles (the library's
sk_model_time).  Its six terms are constants per tile configuration, fitted to
measurements of the kernel they plan for.

measure (GPU): times every shape of the 2,000-shape BF16 sweep under every
fixed plan -- each tile configuration (BLK_N 64, 128 and 256 on single CTAs,
128 and 256 on CTA pairs) with each schedule (data-parallel tiling, the two-tile
hybrid, basic Stream-K at the model's grid size, the one-tile hybrid) -- through
the benchmark's harness (one CUDA graph per step, operands larger than L2, a
timing event between shapes), and writes the per-shape median times with the
plans to DIR/calibration.json.

fit (host only): fits the six terms of each configuration by least squares on
the log-time ratio of model to measurement, evaluating the model through
sk_model_time, and reports for the built-in and the fitted terms how close the
model's pick among the measured plans comes to the fastest of them per shape
(the geo-mean ratio AUTO is judged by).  It prints the fitted terms as the
initialiser lines of model_coefficients (csrc/planner.cpp).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

CONFIGS = [(64, 1), (128, 1), (256, 1), (128, 2), (256, 2)]
MODES = ["dp", "hybrid", "sk", "hybrid1"]
SPLIT_MARGIN = 0.10  # kSplitMargin of the planner


def considered(m, n, tile_n, cluster_m):
    """The configurations AUTO ranks for a shape (planner.cpp describe)."""
    if tile_n == 256 and n <= 128:
        return False
    if cluster_m == 2 and m <= 128:
        return False
    return True


def measure(args):
    import torch
    from . import inputs
    from . import streamk as sk
    from .sweep import Sweep, run_variant
    shapes = inputs.sweep_shapes(args.count)
    dev = torch.device("cuda", torch.cuda.current_device())
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sweep = Sweep(shapes, dev, seed=inputs.SWEEP_SEED)
    out = {"num_sms": num_sms, "shapes": shapes, "device": torch.cuda.get_device_name(dev),
           "steps": args.steps, "warmup": args.warmup, "plans": {}}
    keep = []
    for tn, cm in CONFIGS:
        for mode in MODES:
            plans = []
            for (m, n, k) in shapes:
                p = sk.sk_plan(m, n, k, "bf16", "bf16", "bf16", "f32", "row", "col", "row", mode)
                p.set("tile_n", tn)
                p.set("cluster_m", cm)
                plans.append(p)
            need = max([p.get("workspace_bytes") for p in plans] + [4096])
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
            keep.append(ws)  # the plans write into it until they are destroyed
            for p in plans:
                sk.sk_plan_attach_workspace(p, ws, ws.numel())
            _, _, per, _ = run_variant(plans, sweep, args.steps, args.warmup, lambda: None)
            med = np.median(per, axis=0) * 1e3  # per-GEMM ms -> us
            infos = [p.info() for p in plans]
            out["plans"][f"{mode}/{tn}x{cm}"] = {
                "us": [float(v) for v in med],
                "plan": [[i["mode"], i["grid"], i["sk_tiles"], i["dp_tiles"], i["workspace_bytes"]]
                         for i in infos]}
            print(f"{mode}/{tn}x{cm}: geo-mean "
                  f"{math.exp(np.mean(np.log([2.0 * a * b * c / t / 1e6 for (a, b, c), t in zip(shapes, med)]))):.1f}"
                  " TFLOP/s", flush=True)
            for p in plans:
                p.destroy()
            torch.cuda.synchronize()
    os.makedirs(args.out, exist_ok=True)
    path = os.path.join(args.out, "calibration.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path)


def _model(sk, shape, key, plan, num_sms, coef):
    m, n, k = shape
    mode, cfg = key.split("/")
    tn, cm = (int(v) for v in cfg.split("x"))
    grid = plan[1] if mode == "sk" else 0
    return sk.sk_model_time(m, n, k, mode, tile_n=tn, grid=grid, num_sms=num_sms, cluster_m=cm,
                            coef=coef)


def pick_quality(sk, data, coefs, modes):
    """Geo-mean over shapes of t(model's pick among the measured plans of
    `modes`) / t(fastest of them), and the count of shapes whose pick is more
    than 5% slower than the fastest data-parallel plan."""
    shapes, num_sms, plans = data["shapes"], data["num_sms"], data["plans"]
    ratios, worse_than_dp = [], 0
    for i, (m, n, k) in enumerate(shapes):
        best_t, pick, pick_t, best_dp = math.inf, None, None, math.inf
        for key, rec in plans.items():
            mode, cfg = key.split("/")
            tn, cm = (int(v) for v in cfg.split("x"))
            if not considered(m, n, tn, cm) or mode not in modes:
                continue
            t = rec["us"][i]
            best_t = min(best_t, t)
            if mode == "dp":
                best_dp = min(best_dp, t)
            us = _model(sk, (m, n, k), key, rec["plan"][i], num_sms, coefs[cfg])
            if rec["plan"][i][4] > 0:
                us *= 1.0 + SPLIT_MARGIN
            if pick is None or us < pick:
                pick, pick_t = us, t
        ratios.append(pick_t / best_t)
        worse_than_dp += pick_t > 1.05 * best_dp
    return math.exp(float(np.mean(np.log(ratios)))), worse_than_dp


def fit(args):
    from scipy.optimize import least_squares
    from . import streamk as sk
    with open(args.data) as f:
        data = json.load(f)
    shapes, num_sms, plans = data["shapes"], data["num_sms"], data["plans"]
    modes = [md for md in MODES if args.with_hybrid1 or md != "hybrid1"]
    builtin = {f"{tn}x{cm}": sk.sk_model_coefficients(tn, cm) for tn, cm in CONFIGS}
    fitted = {}
    for tn, cm in CONFIGS:
        cfg = f"{tn}x{cm}"
        rows = []
        for md in modes:
            rec = plans[f"{md}/{cfg}"]
            for i, (m, n, k) in enumerate(shapes):
                if considered(m, n, tn, cm):
                    rows.append(((m, n, k), f"{md}/{cfg}", rec["plan"][i], rec["us"][i]))

        def resid(c):
            return np.array([math.log(_model(sk, s, key, p, num_sms, list(c)) / t)
                             for s, key, p, t in rows])

        x0 = np.array(builtin[cfg])
        r = least_squares(resid, x0, bounds=(1e-3, np.inf), x_scale=x0, diff_step=1e-3)
        fitted[cfg] = [float(v) for v in r.x]
        rms0 = float(np.sqrt(np.mean(resid(x0) ** 2)))
        rms1 = float(np.sqrt(np.mean(r.fun ** 2)))
        print(f"{cfg}: {len(rows)} measurements, rms log error {rms0:.3f} -> {rms1:.3f}", flush=True)
    q0 = pick_quality(sk, data, builtin, modes)
    q1 = pick_quality(sk, data, fitted, modes)
    print(f"pick / best measured plan, geo-mean: built-in {q0[0]:.4f} ({q0[1]} shapes > 5% behind DP),"
          f" fitted {q1[0]:.4f} ({q1[1]} shapes > 5% behind DP)")
    names = {"64x1": "k64x1", "128x1": "k128x1", "256x1": "k256x1", "128x2": "k128x2",
             "256x2": "k256x2"}
    for cfg, c in fitted.items():
        print(f"  static const double {names[cfg]}[kModelTerms] = "
              f"{{{c[0]:.3f}, {c[1]:.3f}, {c[2]:.4f}, {c[3]:.3f}, {c[4]:.3f}, {c[5]:.3f}}};")
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"builtin": builtin, "fitted": fitted, "pick_quality": {
                "builtin": q0[0], "fitted": q1[0]}}, f, indent=1)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("measure", help="time the sweep under every fixed plan (GPU)")
    a.add_argument("--out", required=True)
    a.add_argument("--count", type=int, default=2000)
    a.add_argument("--steps", type=int, default=3)
    a.add_argument("--warmup", type=int, default=2)
    b = sub.add_parser("fit", help="fit the model terms to a measurement (host only)")
    b.add_argument("data")
    b.add_argument("--out", default=None, help="write the fitted terms as JSON")
    b.add_argument("--with-hybrid1", action="store_true",
                   help="also fit on the one-tile hybrid's measurements")
    args = ap.parse_args(argv)
    return measure(args) if args.cmd == "measure" else fit(args)


if __name__ == "__main__":
    sys.exit(main())
