"""One plan, one workspace: a launch of a plan on a second stream while its
previous launch still runs on the first returns SK_ERR_BUSY and enqueues
nothing; launches on the same stream, and on another stream once the previous
launch has finished, are accepted.  The first stream is held busy by a
bounded device sleep queued ahead of the GEMM, so nothing waits for long.
"""
import pytest
import torch

from gemm_check import Problem
from paper_2301_03598_gb300 import streamk as sk

pytestmark = pytest.mark.gpu

SLEEP_CYCLES = 40_000_000  # about 20 ms at 2 GHz


@pytest.mark.parametrize("mode", ["sk", "dp"])
def test_plan_launch_on_second_stream_while_running_is_busy(mode):
    m, n, k = 1024, 768, 2048
    prob = Problem(m, n, k, "bf16", "f32", "normal", seed=41)
    plan = sk.sk_plan(m, n, k, "bf16", "bf16", "f32", mode=mode)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    A, B = prob.A.cuda(), prob.B.cuda()
    C1 = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    C2 = torch.full((m, n), 7.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    try:
        with torch.cuda.stream(s1):
            torch.cuda._sleep(SLEEP_CYCLES)
        sk.sk_gemm(plan, A, B, C1, 1.0, 0.0, stream=s1)
        with pytest.raises(sk.StreamKError) as e:
            sk.sk_gemm(plan, A, B, C2, 1.0, 0.0, stream=s2)
        assert e.value.status == sk.SK_ERR_BUSY
        # the same stream is ordered behind the running launch: accepted
        sk.sk_gemm(plan, A, B, C1, 1.0, 0.0, stream=s1)
        s1.synchronize()
        assert torch.all(C2 == 7.0), "the refused launch wrote C"
        # the previous launch has finished: another stream may launch now
        sk.sk_gemm(plan, A, B, C2, 1.0, 0.0, stream=s2)
        s2.synchronize()
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
        prob.check(C1.cpu(), 1.0, 0.0, f"{mode} on the first stream")
        prob.check(C2.cpu(), 1.0, 0.0, f"{mode} on the second stream")
    finally:
        torch.cuda.synchronize()
        plan.destroy()


def test_grouped_plan_launch_on_second_stream_while_running_is_busy():
    ms, ns, ks = [256, 384], [256, 512], [512, 256]
    probs = [Problem(m, n, k, "bf16", "bf16", "normal", seed=42 + i)
             for i, (m, n, k) in enumerate(zip(ms, ns, ks))]
    plan = sk.sk_grouped_plan(list(zip(ms, ns, ks)), "bf16", "bf16", "auto")
    As = [p.A.cuda() for p in probs]
    Bs = [p.B.cuda() for p in probs]
    Cs = [torch.zeros((p.m, p.n), dtype=torch.bfloat16, device="cuda") for p in probs]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    try:
        with torch.cuda.stream(s1):
            torch.cuda._sleep(SLEEP_CYCLES)
        sk.sk_grouped_gemm(plan, As, Bs, Cs, stream=s1)
        with pytest.raises(sk.StreamKError) as e:
            sk.sk_grouped_gemm(plan, As, Bs, Cs, stream=s2)
        assert e.value.status == sk.SK_ERR_BUSY
        s1.synchronize()
        sk.sk_grouped_gemm(plan, As, Bs, Cs, stream=s2)
        s2.synchronize()
        assert sk.sk_grouped_last_error(plan)[0] == sk.SK_OK
        for p, C in zip(probs, Cs):
            p.check(C.cpu(), 1.0, 0.0, "grouped after busy")
    finally:
        torch.cuda.synchronize()
        plan.destroy()
