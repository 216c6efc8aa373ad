"""The serving loop (continuous batching over grouped Stream-K launches):
every request's result against the FP64 oracle, alone and in a mix."""
import pytest
import torch

from paper_2301_03598_gb300 import streamk as sk

from gemm_check import Problem, bound, check_bound
from paper_2301_03598_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(300, 500, 704), (128, 128, 4096), (1000, 200, 128), (64, 520, 1024), (17, 1000, 304),
          (777, 96, 2000), (256, 256, 8192), (2048, 384, 512), (33, 33, 64), (512, 1536, 1536)]


def _requests(seed=0, c_type="bf16", beta=0.0):
    probs = [Problem(m, n, k, "bf16", c_type, "normal", seed=seed + 5 * i, beta=beta)
             for i, (m, n, k) in enumerate(SHAPES)]
    dev = [(p.A.cuda(), p.B.cuda()) for p in probs]
    return probs, dev


def _run(server, probs, dev, alone, alpha=1.0, beta=0.0):
    Cs = [p.Cin.clone().cuda() for p in probs]
    if alone:
        for (A, B), C in zip(dev, Cs):
            st, lat = server.wait(server.submit(A, B, C, alpha, beta))
            assert st == sk.SK_OK and lat > 0
    else:
        tickets = [server.submit(A, B, C, alpha, beta) for (A, B), C in zip(dev, Cs)]
        for t in tickets:
            st, lat = server.wait(t)
            assert st == sk.SK_OK and lat > 0
    torch.cuda.synchronize()
    return [C.cpu() for C in Cs]


@pytest.mark.parametrize("c_type,beta", [("bf16", 0.0), ("f32", 0.5)])
def test_server_results_match_oracle(c_type, beta):
    probs, dev = _requests(seed=1, c_type=c_type, beta=beta)
    with sk.sk_server_create("bf16", c_type, max_batch=8, slots=2) as server:
        outs = _run(server, probs, dev, alone=False, alpha=1.25, beta=beta)
        st = server.stats()
        assert st["completed"] == len(SHAPES) and st["queued"] == 0 and st["batches"] >= 2
    for p, C in zip(probs, outs):
        p.check(C, 1.25, beta, f"served {p.m}x{p.n}x{p.k}")


def test_server_result_same_alone_and_in_the_mix():
    """Each request alone (its own batch) and in a mix (batched with others,
    its tiles scheduled with theirs): both within the oracle bound, and within
    twice the bound of each other."""
    probs, dev = _requests(seed=2, c_type="f32")
    with sk.sk_server_create("bf16", "f32", max_batch=16, slots=2) as server:
        alone = _run(server, probs, dev, alone=True)
        mixed = _run(server, probs, dev, alone=False)
        assert server.stats()["max_batch"] > 1
    for p, a, b in zip(probs, alone, mixed):
        C64, absAB = p.oracle(1.0, 0.0)
        bd = bound(p.k, 1.0, 0.0, absAB, C64, inputs.widen(p.Cin), "f32")
        check_bound(inputs.widen(a), C64, bd, "alone")
        check_bound(inputs.widen(b), C64, bd, "mixed")
        check_bound(inputs.widen(a), inputs.widen(b), 2 * bd, "alone vs mixed")


def test_server_budget_limits_batches():
    probs, dev = _requests(seed=3)
    with sk.sk_server_create("bf16", "bf16", max_batch=16, slots=1, hbm_budget_bytes=1) as server:
        outs = _run(server, probs, dev, alone=False)
        st = server.stats()
        assert st["max_batch"] == 1 and st["batches"] == len(SHAPES)
    for p, C in zip(probs, outs):
        p.check(C, 1.0, 0.0, "budget-limited")


def test_server_mixed_bf16_and_e4m3_requests():
    """BF16 and block-scaled E4M3 requests interleaved: batches take one input
    type each, and every result matches its oracle."""
    from test_gpu_f8 import F8Problem
    probs, dev = _requests(seed=4)
    f8 = [F8Problem(m, n, k, "bf16", seed=40 + i, scale_spread=(i % 2 == 0))
          for i, (m, n, k) in enumerate(SHAPES) if k % 16 == 0]
    f8dev = [(p.qA.cuda(), p.qB.cuda(), p.sA.cuda(), p.sB.cuda()) for p in f8]
    Cs = [p.Cin.clone().cuda() for p in probs]
    C8 = [p.Cin.clone().cuda() for p in f8]
    with sk.sk_server_create("bf16", "bf16", max_batch=8, slots=2) as server:
        tickets = []
        for i in range(max(len(probs), len(f8))):
            if i < len(probs):
                tickets.append(server.submit(dev[i][0], dev[i][1], Cs[i]))
            if i < len(f8):
                A, B, sA, sB = f8dev[i]
                tickets.append(server.submit_scaled(A, B, sA, sB, C8[i]))
        for t in tickets:
            st, _ = server.wait(t)
            assert st == sk.SK_OK
        assert server.stats()["completed"] == len(tickets)
    torch.cuda.synchronize()
    for p, C in zip(probs, Cs):
        p.check(C.cpu(), 1.0, 0.0, f"served bf16 {p.m}x{p.n}x{p.k}")
    for p, C in zip(f8, C8):
        p.check(C.cpu(), 1.0, 0.0, f"served e4m3 {p.m}x{p.n}x{p.k}")


def test_server_same_shape_on_concurrent_slots():
    """Lone requests of one Stream-K-split shape on two slots at once: each slot
    runs its own plan and fixup workspace, so every result stays exact."""
    p = Problem(384, 384, 4096, "bf16", "f32", "normal", seed=6)
    A, B = p.A.cuda(), p.B.cuda()
    Cs = [torch.zeros(384, 384, dtype=torch.float32, device="cuda") for _ in range(40)]
    with sk.sk_server_create("bf16", "f32", max_batch=1, slots=2) as server:
        tickets = [server.submit(A, B, C) for C in Cs]
        for t in tickets:
            st, _ = server.wait(t)
            assert st == sk.SK_OK
        assert server.stats()["batches"] == len(Cs)
    torch.cuda.synchronize()
    C64, absAB = p.oracle(1.0, 0.0)
    bd = bound(p.k, 1.0, 0.0, absAB, C64, inputs.widen(p.Cin), "f32")
    first = Cs[0].cpu()
    for C in Cs:
        check_bound(inputs.widen(C.cpu()), C64, bd, "concurrent slots")
        assert torch.equal(C.cpu(), first)   # one plan per slot: the same schedule


def test_server_many_slots_split_launches():
    """Eight slots and lone requests of split-schedule shapes: split launches
    on different slots run one at a time, so none of their waits runs out."""
    shapes = [(384, 384, 4096), (256, 256, 8192), (128, 1000, 3072)]
    probs = [Problem(m, n, k, "bf16", "f32", "normal", seed=70 + i) for i, (m, n, k) in enumerate(shapes)]
    dev = [(p.A.cuda(), p.B.cuda()) for p in probs]
    outs = [[torch.zeros(p.m, p.n, dtype=torch.float32, device="cuda") for _ in range(12)] for p in probs]
    with sk.sk_server_create("bf16", "f32", max_batch=1, slots=8) as server:
        tickets = []
        for r in range(12):
            for (A, B), Cs in zip(dev, outs):
                tickets.append(server.submit(A, B, Cs[r]))
        for t in tickets:
            st, _ = server.wait(t)
            assert st == sk.SK_OK
    torch.cuda.synchronize()
    for p, Cs in zip(probs, outs):
        C64, absAB = p.oracle(1.0, 0.0)
        bd = bound(p.k, 1.0, 0.0, absAB, C64, inputs.widen(p.Cin), "f32")
        for C in Cs:
            check_bound(inputs.widen(C.cpu()), C64, bd, f"8 slots {p.m}x{p.n}x{p.k}")
