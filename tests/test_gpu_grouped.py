"""Grouped GEMM on the GPU through the C ABI: every problem of one persistent
launch against the FP64 oracle, and the device schedule against the oracle's
grouped Stream-K schedule."""
import pytest
import torch

from oracle import schedule as S
from paper_2301_03598_gb300 import streamk as sk

from gemm_check import Problem

pytestmark = pytest.mark.gpu

# dense operands need rows of a multiple of 16 bytes: k a multiple of 8 (16-bit inputs)
GROUP = [(300, 500, 704), (128, 128, 4096), (1000, 200, 128), (64, 520, 1024), (17, 1000, 304),
         (777, 96, 2000)]


def _run(shapes, mode, c_type="bf16", beta=0.0, attrs=None, trace=False, seed=0, reps=1):
    probs = [Problem(m, n, k, "bf16", c_type, "normal", seed=seed + 13 * i, beta=beta)
             for i, (m, n, k) in enumerate(shapes)]
    plan = sk.sk_grouped_plan(shapes, "bf16", c_type, mode)
    try:
        for key, v in (attrs or {}).items():
            plan.set(key, v)
        As = [p.A.cuda() for p in probs]
        Bs = [p.B.cuda() for p in probs]
        outs = []
        recs = None
        for _ in range(reps):
            Cs = [p.Cin.clone().cuda() for p in probs]
            alphas = [1.0 + 0.25 * (i % 3) for i in range(len(shapes))]
            betas = [beta] * len(shapes)
            if trace:
                tr = torch.full((plan.get("trace_ints"),), -7, dtype=torch.int32, device="cuda")
                sk.sk_grouped_gemm_traced(plan, As, Bs, Cs, alphas, betas, tr)
            else:
                sk.sk_grouped_gemm(plan, As, Bs, Cs, alphas, betas)
            st, dev = sk.sk_grouped_last_error(plan)
            assert st == sk.SK_OK, (sk.sk_status_string(st), dev)
            outs.append([c.cpu() for c in Cs])
            if trace:
                recs = _decode_grouped(tr.cpu().tolist(), plan.get("ctas"), plan.get("trace_cap"))
        return probs, outs, alphas, plan.info(), recs
    finally:
        plan.destroy()


def _decode_grouped(vals, ctas, cap):
    out = []
    stride = sk.TRACE_HEADER + cap * sk.TRACE_RECORD
    for x in range(ctas):
        base = x * stride
        for r in range(vals[base]):
            o = base + sk.TRACE_HEADER + r * sk.TRACE_RECORD
            f = vals[o:o + sk.TRACE_FIELDS]
            # (cta, problem, tile, tm, tn, kb0, kb1, role, peer_first, peer_last)
            out.append((f[0], vals[o + 9]) + tuple(f[1:]))
    return out


@pytest.mark.parametrize("mode", ["auto", "dp", "sk", "hybrid"])
@pytest.mark.parametrize("tile_n,cluster_m", [(128, 1), (256, 1), (128, 2), (256, 2)])
def test_grouped_matches_oracle(mode, tile_n, cluster_m):
    probs, outs, alphas, info, _ = _run(GROUP, mode, "bf16", 0.0,
                                        {"tile_n": tile_n, "cluster_m": cluster_m}, seed=5)
    assert info["cluster_m"] == cluster_m and info["ctas"] == cluster_m * info["grid"]
    for p, C, al in zip(probs, outs[0], alphas):
        p.check(C, al, 0.0, f"grouped {mode} bn={tile_n} cm={cluster_m} {p.m}x{p.n}x{p.k}")


@pytest.mark.parametrize("c_type", ["f32", "f16"])
def test_grouped_beta_and_output_types(c_type):
    probs, outs, alphas, info, _ = _run(GROUP, "sk", c_type, 0.5, {"grid": 40}, seed=9)
    for p, C, al in zip(probs, outs[0], alphas):
        p.check(C, al, 0.5, f"grouped beta {c_type} {p.m}x{p.n}x{p.k}")


@pytest.mark.parametrize("mode,attrs", [("sk", {"grid": 23}), ("hybrid", {"tile_n": 128}),
                                        ("auto", {}), ("dp", {"tile_n": 256}),
                                        ("sk", {"tile_n": 256, "cluster_m": 2, "grid": 23}),
                                        ("hybrid", {"tile_n": 128, "cluster_m": 2}),
                                        ("dp", {"tile_n": 256, "cluster_m": 2})])
def test_grouped_device_schedule_matches_oracle(mode, attrs):
    probs, outs, alphas, info, recs = _run(GROUP, mode, "bf16", 0.0, attrs, trace=True, seed=2)
    cm = info["cluster_m"]
    oprobs = [S.Problem(m, n, k, 128 * cm, info["tile_n"], info["tile_k"]) for (m, n, k) in GROUP]
    ctas = S.grouped_schedule(oprobs, info["grid"], info["sk_tiles"])
    units = S.grouped_trace(oprobs, ctas, [min(p.tiles_m, 16 // cm) for p in oprobs])
    assert recs == S.grouped_cluster_trace(units, cm)
    for p, C, al in zip(probs, outs[0], alphas):
        p.check(C, al, 0.0, f"traced grouped {mode}")


def test_grouped_relaunch_with_new_buffers_and_graph_replay():
    shapes = GROUP[:4]
    probs = [Problem(m, n, k, "bf16", "bf16", "normal", seed=31 + i) for i, (m, n, k) in enumerate(shapes)]
    plan = sk.sk_grouped_plan(shapes, "bf16", "bf16", "sk")
    try:
        As = [p.A.cuda() for p in probs]
        Bs = [p.B.cuda() for p in probs]
        for rep in range(2):   # fresh outputs: the problem table is re-encoded
            Cs = [torch.zeros(p.m, p.n, dtype=torch.bfloat16, device="cuda") for p in probs]
            sk.sk_grouped_gemm(plan, As, Bs, Cs)
            assert sk.sk_grouped_last_error(plan)[0] == sk.SK_OK
            for p, C in zip(probs, Cs):
                p.check(C.cpu(), 1.0, 0.0, f"relaunch {rep}")
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            sk.sk_grouped_gemm(plan, As, Bs, Cs, stream=s)   # table already current
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                sk.sk_grouped_gemm(plan, As, Bs, Cs, stream=s)
        for _ in range(3):
            for C in Cs:
                C.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert sk.sk_grouped_last_error(plan)[0] == sk.SK_OK
            for p, C in zip(probs, Cs):
                p.check(C.cpu(), 1.0, 0.0, "graph replay")
    finally:
        plan.destroy()


@pytest.mark.parametrize("cluster_m,grid", [(1, 36), (2, 18)])
def test_grouped_single_problem_equals_gemm_bitwise(cluster_m, grid):
    """A group of one problem runs the same schedule as the single-GEMM path
    with the same tile configuration and grid, so the results are bitwise
    equal (single CTAs and CTA pairs)."""
    m, n, k = 384, 384, 4096
    p = Problem(m, n, k, "bf16", "f32", "normal", seed=77)
    A, B = p.A.cuda(), p.B.cuda()
    plan = sk.sk_plan(m, n, k, "bf16", "bf16", "f32", mode="sk")
    gplan = sk.sk_grouped_plan([(m, n, k)], "bf16", "f32", "sk")
    try:
        plan.set("tile_n", 128)
        plan.set("cluster_m", cluster_m)
        plan.set("grid", grid)
        gplan.set("tile_n", 128)
        gplan.set("cluster_m", cluster_m)
        gplan.set("grid", grid)
        C1 = torch.zeros(m, n, dtype=torch.float32, device="cuda")
        C2 = torch.zeros(m, n, dtype=torch.float32, device="cuda")
        sk.sk_gemm(plan, A, B, C1)
        sk.sk_grouped_gemm(gplan, [A], [B], [C2])
        assert sk.sk_last_error(plan)[0] == sk.SK_OK and sk.sk_grouped_last_error(gplan)[0] == sk.SK_OK
        assert torch.equal(C1, C2)
    finally:
        plan.destroy()
        gplan.destroy()


def test_grouped_autotune_keeps_a_correct_configuration():
    shapes = GROUP
    probs = [Problem(m, n, k, "bf16", "bf16", "normal", seed=50 + i) for i, (m, n, k) in enumerate(shapes)]
    plan = sk.sk_grouped_plan(shapes, "bf16", "bf16", "auto")
    try:
        As = [p.A.cuda() for p in probs]
        Bs = [p.B.cuda() for p in probs]
        Cs = [torch.zeros(p.m, p.n, dtype=torch.bfloat16, device="cuda") for p in probs]
        us = sk.sk_grouped_autotune(plan, As, Bs, Cs, reps=2)
        info = plan.info()
        assert us > 0 and info["tile_n"] in (64, 128, 256)
        for C in Cs:
            C.zero_()
        sk.sk_grouped_gemm(plan, As, Bs, Cs)
        assert sk.sk_grouped_last_error(plan)[0] == sk.SK_OK
        for p, C in zip(probs, Cs):
            p.check(C.cpu(), 1.0, 0.0, "grouped autotuned")
    finally:
        plan.destroy()
