"""The 256-problem grouped workload at full size (m log-uniform in [16, 4096],
n and k from {1024, 2048, 4096, 8192}), on the operands and in the launch
configurations that bench.py times: one grouped launch with the AUTO plan for
BF16, and the AUTO and the autotuned plan for E4M3 with per-128 x 128-block
scales.  Every problem is checked against the FP64 oracle on seeded sampled
entries plus entries along its tile edges (rows and columns 0, 127, 128, 255,
256 and the last), where Stream-K seams, ragged tiles and problem boundaries
are."""
import numpy as np
import pytest
import torch

import oracle
from oracle import e4m3
from paper_2301_03598_gb300 import inputs
from paper_2301_03598_gb300 import streamk as sk

from gemm_check import bound, check_bound

pytestmark = pytest.mark.gpu

EDGES = (0, 127, 128, 255, 256)


def _entries(m, n, rng, samples=24, per_edge=4):
    rows = list(rng.integers(0, m, samples))
    cols = list(rng.integers(0, n, samples))
    for r in sorted({*EDGES, m - 1} & set(range(m))):
        rows += [r] * per_edge
        cols += list(rng.integers(0, n, per_edge))
    for c in sorted({*EDGES, n - 1} & set(range(n))):
        rows += list(rng.integers(0, m, per_edge))
        cols += [c] * per_edge
    return np.array(rows, np.int64), np.array(cols, np.int64)


def _take(t, idx):
    return t[torch.from_numpy(idx).to(t.device)].cpu()


def _check_problem(i, shape, C, rows, cols, want, absAB, what):
    m, n, k = shape
    got = inputs.widen(C[torch.from_numpy(rows).to(C.device),
                         torch.from_numpy(cols).to(C.device)].cpu())
    check_bound(got, want, bound(k, 1.0, 0.0, absAB, want, None, "bf16"),
                f"{what} problem {i} ({m}x{n}x{k})")


def test_grouped_bf16_full_workload():
    shapes = inputs.grouped_shapes()
    dev = torch.device("cuda", torch.cuda.current_device())
    As, Bs, Cs = [], [], []
    for i, (m, n, k) in enumerate(shapes):
        As.append(inputs.device_pool(m * k, "bf16", "normal", inputs.GROUPED_SEED + 3 * i,
                                     dev).view(m, k))
        Bs.append(inputs.device_pool(n * k, "bf16", "normal", inputs.GROUPED_SEED + 3 * i + 1,
                                     dev).view(n, k))
        Cs.append(torch.full((m, n), float("nan"), dtype=torch.bfloat16, device=dev))
    plan = sk.sk_grouped_plan(shapes, "bf16", "bf16", "auto")
    try:
        sk.sk_grouped_gemm(plan, As, Bs, Cs)
        st, dstat = sk.sk_grouped_last_error(plan)
        assert st == sk.SK_OK, (sk.sk_status_string(st), dstat)
        info = plan.info()
    finally:
        plan.destroy()
    rng = np.random.Generator(np.random.PCG64(17))
    for i, (m, n, k) in enumerate(shapes):
        rows, cols = _entries(m, n, rng)
        ur, ri = np.unique(rows, return_inverse=True)
        uc, ci = np.unique(cols, return_inverse=True)
        want, absAB = oracle.gemm_entries(ri, ci, inputs.widen(_take(As[i], ur)),
                                          inputs.widen(_take(Bs[i], uc)).T)
        _check_problem(i, (m, n, k), Cs[i], rows, cols, want, absAB,
                       f"bf16 grouped {info['mode']} g={info['grid']}")


def test_grouped_e4m3_full_workload_auto_and_autotuned():
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
    rng = np.random.Generator(np.random.PCG64(19))
    expected = []
    for i, (m, n, k) in enumerate(shapes):
        rows, cols = _entries(m, n, rng)
        ur, ri = np.unique(rows, return_inverse=True)
        uc, ci = np.unique(cols, return_inverse=True)
        want, absAB = e4m3.gemm_entries_rows(
            ri, ci, _take(As[i], ur).numpy(), _take(SAs[i], ur // 128).numpy(),
            _take(Bs[i], uc).numpy(), _take(SBs[i], uc // 128).numpy())
        expected.append((rows, cols, want, absAB))
    plan = sk.sk_grouped_plan(shapes, "e4m3", "bf16", "auto")
    try:
        for tuned in (False, True):
            if tuned:
                sk.sk_grouped_autotune_scaled(plan, As, Bs, SAs, SBs, Cs, reps=2)
            for C in Cs:
                C.fill_(float("nan"))
            sk.sk_grouped_gemm_scaled(plan, As, Bs, SAs, SBs, Cs)
            st, dstat = sk.sk_grouped_last_error(plan)
            assert st == sk.SK_OK, (sk.sk_status_string(st), dstat)
            info = plan.info()
            what = f"e4m3 grouped {'autotuned ' if tuned else ''}{info['mode']} g={info['grid']}"
            for i, (shape, (rows, cols, want, absAB)) in enumerate(zip(shapes, expected)):
                _check_problem(i, shape, Cs[i], rows, cols, want, absAB, what)
    finally:
        plan.destroy()
