"""SK_ATTR_INDEPENDENT_INPUTS: launches whose operands no earlier kernel in the
stream writes load them and run their MAC loop while the previous kernel
finishes; C and the fixup workspace keep stream order.  Checked against the
oracle: back-to-back launches of one split plan (its workspace reused by
consecutive launches), a chain accumulating into one C (each launch reads the
C its predecessor wrote), and a stream of mixed-shape independent GEMMs.
"""
import numpy as np
import pytest
import torch

from gemm_check import Problem
from paper_2301_03598_gb300 import inputs
from paper_2301_03598_gb300 import streamk as sk

pytestmark = pytest.mark.gpu


def plan_for(m, n, k, c_type, mode, attrs):
    p = sk.sk_plan(m, n, k, "bf16", "bf16", c_type, mode=mode)
    for key, v in attrs.items():
        p.set(key, v)
    p.set("independent_inputs", 1)
    assert p.get("independent_inputs") == 1
    return p


@pytest.mark.parametrize("m,n,k,mode,attrs", [
    (384, 384, 4096, "sk", {"tile_n": 64, "grid": 100}),
    (384, 384, 4096, "sk", {"tile_n": 128, "grid": 148}),
    (1000, 1000, 1000, "auto", {}),
    (2432, 1024, 256, "hybrid", {"tile_n": 128}),
])
def test_back_to_back_split_launches_share_the_workspace(m, n, k, mode, attrs):
    prob = Problem(m, n, k, "bf16", "f32", "normal", seed=61)
    plan = plan_for(m, n, k, "f32", mode, attrs)
    try:
        A, B = prob.A.cuda(), prob.B.cuda()
        outs = [torch.zeros((m, n), dtype=torch.float32, device="cuda") for _ in range(12)]
        for C in outs:
            sk.sk_gemm(plan, A, B, C, 1.0, 0.0)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
        for C in outs[1:]:
            assert torch.equal(C, outs[0])
        prob.check(outs[0].cpu(), 1.0, 0.0, f"independent {mode} {attrs}")
    finally:
        plan.destroy()


def test_chain_accumulating_into_one_c_keeps_order():
    """C_{j+1} = A_j B_j + 1 * C_j on one stream: each launch reads the C its
    predecessor wrote, so the C accesses must wait even though the operand
    loads do not."""
    m, n, k = 512, 384, 1536
    probs = [Problem(m, n, k, "bf16", "f32", "normal", seed=70 + j) for j in range(6)]
    plan = plan_for(m, n, k, "f32", "sk", {"tile_n": 64, "grid": 120})
    try:
        C = torch.zeros((m, n), dtype=torch.float32, device="cuda")
        ops = [(p.A.cuda(), p.B.cuda()) for p in probs]
        for A, B in ops:
            sk.sk_gemm(plan, A, B, C, 1.0, 1.0)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
        parts = [p.oracle(1.0, 0.0) for p in probs]     # (C64, |A||B|) per launch
        want = sum(c64 for c64, _ in parts)
        absab = sum(ab for _, ab in parts)
        got = inputs.widen(C.cpu())
        # six FP32 sums of k terms plus the five FP32 adds of the chain
        tol = 6 * k * 2.0 ** -22 * absab + 2.0 ** -20 * np.abs(want) + 1e-30
        assert np.all(np.abs(got - want) <= tol)
    finally:
        plan.destroy()


def test_stream_of_independent_mixed_gemms():
    shapes = [(128, 128, 128), (592, 192, 7312), (1024, 640, 256), (272, 720, 128),
              (3000, 200, 896), (128, 8192, 512), (2048, 2048, 1024), (256, 256, 8192)]
    probs, plans, outs = [], [], []
    try:
        for i, (m, n, k) in enumerate(shapes):
            probs.append(Problem(m, n, k, "bf16", "bf16", "normal", seed=80 + i))
            plans.append(plan_for(m, n, k, "bf16", "auto", {}))
        ops = [(p.A.cuda(), p.B.cuda()) for p in probs]
        for rep in range(3):
            for p, plan, (A, B) in zip(probs, plans, ops):
                C = torch.zeros((p.m, p.n), dtype=torch.bfloat16, device="cuda")
                sk.sk_gemm(plan, A, B, C, 1.0, 0.0)
                outs.append((p, C))
        torch.cuda.synchronize()
        for plan in plans:
            assert sk.sk_last_error(plan)[0] == sk.SK_OK
        for p, C in outs:
            p.check(C.cpu(), 1.0, 0.0, f"independent stream {p.m}x{p.n}x{p.k}")
    finally:
        for plan in plans:
            plan.destroy()
