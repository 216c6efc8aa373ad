"""Device-side harness of the shape sweep: seeded operands larger than L2, one
CUDA graph per step with a timing event between shapes, per-GEMM device times.

Shared by bench.py (the benchmark) and paper_2301_03598_gb300.calibrate (the
planner's model recalibration), so both time GEMMs the same way.
"""
from __future__ import annotations

import numpy as np

POOL_ELEMS = 1 << 31          # 4 GiB of BF16 inputs on the device
OUT_ELEMS = 1 << 30           # 2 GiB of BF16 outputs (reused round-robin)


def reps_for(m, n, k):
    """Back-to-back repetitions of one shape inside a step: enough that the
    ~4 us cost of the graph's timing events is spread over them."""
    fl = 2.0 * m * n * k
    return 16 if fl < 1e9 else 8 if fl < 1e10 else 4 if fl < 1e11 else 2


class Sweep:
    """Device-resident inputs and outputs of the shape sweep.  Every GEMM
    instance (shape, repetition) reads its own slices of a 4 GiB input pool,
    allocated in order with wrap-around, so consecutive GEMMs never share
    operands and the pool is far larger than L2."""

    def __init__(self, shapes, device, seed):
        import torch
        from paper_2301_03598_gb300 import inputs
        self.shapes = shapes
        self.device = device
        self.reps = [reps_for(*s) for s in shapes]
        self.pool = inputs.device_pool(POOL_ELEMS, "bf16", "normal", seed, device)
        self.out = torch.empty(OUT_ELEMS, dtype=torch.bfloat16, device=device)
        self.inst = []          # per shape: list of (a_off, b_off, c_off)
        cur = cur_c = 0
        for (m, n, k), R in zip(shapes, self.reps):
            lst = []
            for _ in range(R):
                need = _al(m * k) + _al(n * k)
                if cur + need > POOL_ELEMS:
                    cur = 0
                if cur_c + _al(m * n) > OUT_ELEMS:
                    cur_c = 0
                lst.append((cur, cur + _al(m * k), cur_c))
                cur += need
                cur_c += _al(m * n)
            self.inst.append(lst)

    def A(self, i, r=0):
        m, n, k = self.shapes[i]
        o = self.inst[i][r][0]
        return self.pool[o:o + m * k]

    def B(self, i, r=0):
        m, n, k = self.shapes[i]
        o = self.inst[i][r][1]
        return self.pool[o:o + n * k]

    def C(self, i, r=0):
        m, n, k = self.shapes[i]
        o = self.inst[i][r][2]
        return self.out[o:o + m * n]


def _al(x):
    return (x + 127) // 128 * 128  # 256-byte aligned slices


def capture_step(plans, sweep, stream):
    """A CUDA graph of one step: every shape of the sweep, each run R times
    back to back on fresh operands, with a timing event between shapes."""
    import torch
    from paper_2301_03598_gb300 import streamk as sk
    g = torch.cuda.CUDAGraph()
    evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(len(plans) + 1)]
    with torch.cuda.graph(g, stream=stream):
        evs[0].record()
        for i, p in enumerate(plans):
            for r in range(sweep.reps[i]):
                sk.sk_gemm(p, sweep.A(i, r), sweep.B(i, r), sweep.C(i, r), 1.0, 0.0)
            evs[i + 1].record()
    return g, evs


def event_overhead_us(stream, count=200):
    """Device time of one timing-event node in a graph (measured, reported)."""
    import torch
    g = torch.cuda.CUDAGraph()
    evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(count + 1)]
    with torch.cuda.graph(g, stream=stream):
        for e in evs:
            e.record()
    g.replay()
    torch.cuda.synchronize()
    return evs[0].elapsed_time(evs[-1]) * 1e3 / count


def run_variant(plans, sweep, steps, warmup, barrier, sampler=None):
    """Returns (total_ms, per-step device ms, per_gemm_ms[steps][n])."""
    import torch
    from paper_2301_03598_gb300 import streamk as sk
    n = len(plans)
    stream = torch.cuda.Stream()
    g, evs = capture_step(plans, sweep, stream)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    for p in plans:
        st, dev = sk.sk_last_error(p)
        if st != sk.SK_OK:
            raise RuntimeError(f"device status {st}/{dev} during warm-up")
    barrier()
    if sampler:
        sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    per, step_ms = [], []
    t0.record()
    for _ in range(steps):
        g.replay()
        torch.cuda.synchronize()   # read this step's per-shape events
        per.append([evs[i].elapsed_time(evs[i + 1]) / sweep.reps[i] for i in range(n)])
        step_ms.append(evs[0].elapsed_time(evs[-1]))
    t1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    for p in plans:
        st, dev = sk.sk_last_error(p)
        if st != sk.SK_OK:
            raise RuntimeError(f"device status {st}/{dev} in the timed region")
    return t0.elapsed_time(t1), step_ms, np.asarray(per), clocks
