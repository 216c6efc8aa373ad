"""The allocation-free entry point sk_gemm_noalloc, for callers that cannot
allocate device memory (plugins handed buffers by a host framework that owns
the pool, latency-critical serving loops where a cudaMalloc would synchronise
the device, processes held to a device-memory quota).

It must give the same results as the plan-based sk_gemm, within the tolerance
the parity tests use (k * 2^-22 * |alpha| |A||B| + 2^-22 |beta C| + one output
ulp), on two calls in a row -- the second call finds the first call's leftovers
in the shared scratch -- and the two calls must agree bit for bit (the fixup
adds partials in a fixed order, so stale flags or partials would show).  The
same holds for the call captured in a CUDA graph after a first eager call.
This file is collected last on purpose.
"""
import pytest
import torch

from gemm_check import Problem, bound, check_bound
from paper_2301_03598_gb300 import inputs
from paper_2301_03598_gb300 import streamk as sk

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,a_type,c_type,mode,alpha,beta", [
    (384, 384, 4096, "f16", "f32", "sk", 1.0, 0.0),       # nine tiles split over many CTAs
    (1000, 776, 1104, "bf16", "bf16", "hybrid", 1.5, 0.5),
    (2432, 1024, 256, "bf16", "bf16", "auto", 1.0, 0.0),   # t >= SM count: two-tile hybrid
])
def test_noalloc_matches_sk_gemm_twice(m, n, k, a_type, c_type, mode, alpha, beta):
    prob = Problem(m, n, k, a_type, c_type, "normal", seed=31, beta=beta)
    A, B = prob.A.cuda(), prob.B.cuda()
    # reference: the existing plan-based entry point, same schedule (BLK_N = 128)
    plan = sk.sk_plan(m, n, k, a_type, a_type, c_type, "f32", "row", "col", "row", mode)
    try:
        plan.set("tile_n", 128)
        C_ref = prob.Cin.clone().cuda()
        sk.sk_gemm(plan, A, B, C_ref, alpha, beta)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
    finally:
        plan.destroy()
    C64, absAB = prob.oracle(alpha, beta)
    tol = bound(k, alpha, beta, absAB, C64, inputs.widen(prob.Cin), c_type)
    ref = inputs.widen(C_ref.cpu())
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    outs = []
    for call in range(2):
        C = prob.Cin.clone().cuda()
        sk.sk_gemm_noalloc(m, n, k, a_type, c_type, A, k, B, k, C, n, alpha, beta, mode,
                           device_status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0, f"call {call}: device status {int(status.item())}"
        got = inputs.widen(C.cpu())
        check_bound(got, ref, tol, f"noalloc call {call} vs sk_gemm")
        check_bound(got, C64, tol, f"noalloc call {call} vs oracle")
        outs.append(C.cpu())
    assert torch.equal(outs[0], outs[1]), "the second call differs from the first"


def test_noalloc_k0_scales_c_twice():
    """k = 0: C = beta * C (no MAC loop), against sk_gemm, on two calls."""
    m, n = 300, 272
    prob = Problem(m, n, 0, "bf16", "bf16", "normal", seed=32, beta=0.5)
    plan = sk.sk_plan(m, n, 0, "bf16", "bf16", "bf16", "f32", "row", "col", "row", "auto")
    dummy = torch.zeros(16, dtype=torch.bfloat16, device="cuda")
    try:
        C_ref = prob.Cin.clone().cuda()
        sk.sk_gemm(plan, dummy, dummy, C_ref, 1.0, 0.5)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
    finally:
        plan.destroy()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        C = prob.Cin.clone().cuda()
        sk.sk_gemm_noalloc(m, n, 0, "bf16", "bf16", dummy, 0, dummy, 0, C, n, 1.0, 0.5, "auto",
                           device_status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(C.cpu(), C_ref.cpu()), f"call {call}"


@pytest.mark.parametrize("m,n,k,mode", [(384, 384, 4096, "sk"), (1000, 776, 1104, "hybrid")])
def test_noalloc_captured_in_a_graph_matches_eager(m, n, k, mode):
    """The documented use under stream capture: one eager call first (it sets
    the device up), then the call captured into a CUDA graph; two replays
    must reproduce the eager result bit for bit (split schedules: the
    captured memsets clear the scratch's flags before every replay)."""
    prob = Problem(m, n, k, "bf16", "f32", "normal", seed=33, beta=0.5)
    A, B = prob.A.cuda(), prob.B.cuda()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    C_eager = prob.Cin.clone().cuda()
    sk.sk_gemm_noalloc(m, n, k, "bf16", "f32", A, k, B, k, C_eager, n, 1.0, 0.5, mode,
                       device_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    C = prob.Cin.clone().cuda()
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            sk.sk_gemm_noalloc(m, n, k, "bf16", "f32", A, k, B, k, C, n, 1.0, 0.5, mode,
                               device_status=status, stream=stream)
    for replay in range(2):
        C.copy_(prob.Cin.cuda())
        status.fill_(-1)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0, f"replay {replay}"
        assert torch.equal(C, C_eager), f"replay {replay} differs from the eager call"
    C64, absAB = prob.oracle(1.0, 0.5)
    tol = bound(k, 1.0, 0.5, absAB, C64, inputs.widen(prob.Cin), "f32")
    check_bound(inputs.widen(C_eager.cpu()), C64, tol, f"noalloc eager {mode}")
    del graph


def test_noalloc_rejects_bad_arguments():
    A = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    with pytest.raises(sk.StreamKError) as e:
        sk.sk_gemm_noalloc(128, 128, 64, "bf16", "f32", A, 60, A, 64, C, 128)   # lda < k
    assert e.value.status == sk.SK_ERR_INVALID
    with pytest.raises(sk.StreamKError) as e:
        sk.sk_gemm_noalloc(128, 128, 64, "bf16", "f32", A.data_ptr() + 2, 64, A, 64, C, 128)
    assert e.value.status == sk.SK_ERR_INVALID
