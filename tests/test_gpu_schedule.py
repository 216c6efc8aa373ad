"""The schedule the GPU executed, recorded by the kernel itself, against the
oracle's CPU model of Algorithm 5 and the hybrids of Section 5.2: every record
(CTA, tile, tile coordinates, k-range, role, peer range) must match exactly.
Also the failure path of the fixup's bounded Wait.
"""
import pytest
import torch

from gemm_check import Problem, hybrid_shape, num_sms
from oracle import schedule as S
from paper_2301_03598_gb300 import streamk as sk

pytestmark = pytest.mark.gpu


def model_trace(info, m, n, k):
    prob = S.Problem(m, n, k, info["tile_m"], info["tile_n"], info["tile_k"])
    assert prob.tiles == info["tiles"] and prob.iters_per_tile == info["iters_per_tile"]
    sched = S.persistent_schedule(prob, info["grid"], info["sk_tiles"], info["raster_group"])
    return S.cluster_trace(sched, info["cluster_m"])


@pytest.mark.parametrize("m,n,k,mode,attrs", [
    (384, 384, 4096, "sk", {"grid": 148}),
    (384, 384, 4096, "sk", {"grid": 36}),
    (384, 384, 4096, "auto", {}),
    (896, 384, 128 * 16, "sk", {"grid": 4}),
    (19 * 128, 2048, 256, "hybrid", {"tile_n": 128, "raster_group": 4}),
    (19 * 128, 2048, 512, "hybrid1", {"tile_n": 128}),
    (38 * 128, 2048, 192, "hybrid", {"tile_n": 256}),
    (2048, 2048, 128, "dp", {"tile_n": 256, "raster_group": 3}),
    (1000, 1000, 1000, "auto", {}),
    ("2p+8", 1024, 256, "hybrid", {"tile_n": 128, "raster_group": 5}),
    ("2p+8", 2048, 192, "hybrid", {"tile_n": 256}),
    ("2p+8", 1024, 320, "hybrid1", {"tile_n": 128}),
    # 128 x 64 tiles
    (384, 384, 4096, "sk", {"tile_n": 64, "grid": 100}),
    ("2p+8", 512, 256, "hybrid", {"tile_n": 64, "raster_group": 3}),
    (1000, 1000, 1000, "auto", {"tile_n": 64}),
    (640, 200, 3000, "sk", {"tile_n": 64}),
    # CTA pairs (clusters of 2 along M sharing B by multicast)
    (4096, 4096, 512, "hybrid", {"tile_n": 256, "cluster_m": 2}),
    (1000, 3000, 640, "sk", {"tile_n": 256, "cluster_m": 2}),
    (384, 384, 4096, "sk", {"tile_n": 128, "cluster_m": 2, "grid": 30}),
    (2432, 2048, 192, "dp", {"tile_n": 256, "cluster_m": 2, "raster_group": 3}),
])
def test_device_trace_matches_model(m, n, k, mode, attrs):
    if m == "2p+8":
        m = 128 * hybrid_shape(num_sms(), 2, 8)
    prob = Problem(m, n, k, "bf16", "bf16", "normal", seed=21)
    (C,), info, recs = prob.run(1.0, 0.0, mode, plan_attrs=attrs, trace=True)
    want = model_trace(info, m, n, k)
    assert sorted(recs) == sorted(want)
    # and per CTA, in processing order
    assert recs == want
    # the hybrid's owners have exactly one peer (Section 5.2)
    if info["mode"] == sk.MODES["hybrid"] and info["sk_tiles"] > info["num_sms"] // info["cluster_m"]:
        assert all(r[8] - r[7] == 0 for r in recs if r[6] == S.ROLE_OWNER)
    prob.check(C, 1.0, 0.0, f"traced {mode}")


def test_fixup_wait_times_out_and_context_survives():
    """A CTA withholds its Signal; the owner's bounded Wait must expire, the
    kernel must return, the status must say so, and the GPU must stay usable."""
    prob = Problem(384, 384, 4096, "bf16", "f32", "normal", seed=22)
    plan = sk.sk_plan(384, 384, 4096, "bf16", "bf16", "f32", mode="sk")
    try:
        plan.set("grid", 36)
        plan.set("timeout_ns", 50_000_000)   # 50 ms
        # find a CTA whose first segment is a partial (it has an owner waiting)
        info = plan.info()
        model = model_trace(info, 384, 384, 4096)
        victim = next(r[0] for r in model if r[6] == S.ROLE_PARTIAL)
        plan.set("debug_skip_signal", victim)
        A, B = prob.A.cuda(), prob.B.cuda()
        C = torch.zeros((384, 384), dtype=torch.float32, device="cuda")
        sk.sk_gemm(plan, A, B, C, 1.0, 0.0)
        st, dev = sk.sk_last_error(plan)
        assert st == sk.SK_ERR_TIMEOUT and dev in (2, 3)
        # the status is cleared once read, and a normal launch works again
        plan.set("debug_skip_signal", -1)
        sk.sk_gemm(plan, A, B, C, 1.0, 0.0)
        st, dev = sk.sk_last_error(plan)
        assert st == sk.SK_OK and dev == 0
        prob.check(C.cpu(), 1.0, 0.0, "after timeout")
    finally:
        plan.destroy()
