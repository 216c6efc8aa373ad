"""GPU parity: the CUDA Stream-K path against the FP64 oracle, element by
element, within the bound stated in gemm_check (k * 2^-22 * |alpha| |A||B| +
2^-22 |beta C| + one output ulp), through the C ABI.

Sizes span several tiles and ragged edges in m, n and k; schedules cover
data-parallel (Algorithm 2), basic Stream-K (Algorithm 5) at several grid
sizes, and both hybrids of Section 5.2.
"""
import numpy as np
import pytest
import torch

from gemm_check import Problem, hybrid_shape, num_sms
from oracle import schedule as S
from paper_2301_03598_gb300 import streamk as sk

pytestmark = pytest.mark.gpu


# The single-GEMM workload of the paper's strong-scaling regime: m = n = 384,
# k = 4096 (nine 128x128 tiles), FP16 A row-major / B column-major, U[-1, 1],
# FP32 C, alpha = 1, beta = 0.
@pytest.mark.parametrize("mode,attrs", [
    ("auto", {}),
    ("dp", {}),
    ("sk", {"grid": 9}),      # g = t: data-parallel through the Stream-K path
    ("sk", {"grid": 18}),
    ("sk", {"grid": 36}),     # g = 4t: fixed-split s = 4
    ("sk", {"grid": 100}),
    ("sk", {"grid": 148}),
    ("hybrid", {}),
    ("hybrid1", {}),
    ("sk", {"tile_n": 64, "grid": 18}),    # 128 x 64 tiles: g = t, data-parallel
    ("sk", {"tile_n": 64, "grid": 100}),
    ("dp", {"tile_n": 64}),
])
def test_config_384_fp16_fp32(mode, attrs):
    prob = Problem(384, 384, 4096, "f16", "f32", "uniform", seed=1)
    (C,), info, _ = prob.run(1.0, 0.0, mode, plan_attrs=attrs)
    prob.check(C, 1.0, 0.0, f"384x384x4096 {mode} {attrs} g={info['grid']}")


@pytest.mark.parametrize("m,n,k,tile_n", [
    (129, 255, 80, 128), (200, 136, 1000, 128), (16, 16, 16, 128), (1, 8, 8, 128),
    (130, 300, 72, 256), (257, 513, 64, 256), (127, 1, 8, 128), (128, 128, 64, 128),
    (300, 40, 2000, 128), (64, 520, 136, 256),
    (129, 255, 80, 64), (200, 136, 1000, 64), (1, 8, 8, 64), (300, 40, 2000, 64),
    (65, 72, 264, 64), (384, 200, 520, 64),
])
@pytest.mark.parametrize("mode", ["dp", "sk", "hybrid"])
def test_ragged_shapes(m, n, k, tile_n, mode):
    lda = (k + 7) // 8 * 8
    prob = Problem(m, n, k, "bf16", "f32", "normal", seed=m + n + k, lda=lda, ldb=lda)
    (C,), info, _ = prob.run(1.0, 0.0, mode, plan_attrs={"tile_n": tile_n})
    prob.check(C, 1.0, 0.0, f"{m}x{n}x{k} bn={tile_n} {mode} g={info['grid']}")


@pytest.mark.parametrize("a_type,c_type", [("bf16", "bf16"), ("bf16", "f16"), ("f16", "f16"),
                                           ("f16", "bf16"), ("bf16", "f32"), ("f16", "f32")])
@pytest.mark.parametrize("tile_n", [64, 128, 256])
def test_dtypes_alpha_beta(a_type, c_type, tile_n):
    prob = Problem(272, 528, 1088, a_type, c_type, "normal", seed=3, beta=0.5)
    (C,), info, _ = prob.run(1.5, 0.5, "sk", plan_attrs={"tile_n": tile_n, "grid": 60})
    prob.check(C, 1.5, 0.5, f"{a_type}->{c_type} bn={tile_n}")


@pytest.mark.parametrize("tile_n", [64, 128, 256])
def test_two_tile_hybrid_with_dp_waves(tile_n):
    # t = 2p + 8 tiles (rounded to whole tile rows): w = 2 full waves plus a
    # partial one; the two-tile hybrid puts (t mod p) + p tiles in the
    # Stream-K region and one full data-parallel wave after it.
    p = num_sms()
    tiles_m = hybrid_shape(p, 2, 8)
    n = 8 * tile_n
    prob = Problem(tiles_m * 128, n, 256, "bf16", "bf16", "normal", seed=4, beta=0.5)
    (C,), info, _ = prob.run(1.0, 0.5, "hybrid", plan_attrs={"tile_n": tile_n, "cluster_m": 1})
    t = tiles_m * 8
    want = S.hybrid_regions(t, p, S.HYBRID_TWO_TILE)
    assert info["tiles"] == t and (info["sk_tiles"], info["dp_tiles"]) == want
    assert want[0] > p and want[1] == p
    prob.check(C, 1.0, 0.5, f"two-tile hybrid bn={tile_n}")


def test_one_tile_hybrid_with_dp_waves():
    p = num_sms()
    tiles_m = hybrid_shape(p, 2, 8)
    prob = Problem(tiles_m * 128, 1024, 512, "bf16", "bf16", "normal", seed=5)
    (C,), info, _ = prob.run(1.0, 0.0, "hybrid1", plan_attrs={"tile_n": 128})
    want = S.hybrid_regions(tiles_m * 8, p, S.HYBRID_ONE_TILE)
    assert (info["sk_tiles"], info["dp_tiles"]) == want and 0 < want[0] < p
    prob.check(C, 1.0, 0.0, "one-tile hybrid")


@pytest.mark.parametrize("m,n,k,mode,attrs", [
    (4096, 4096, 1024, "hybrid", {}),
    (1000, 1000, 1000, "sk", {"grid": 50}),
    (1152, 2000, 520, "dp", {}),           # odd number of 128-row blocks: the last pair is half empty
    (130, 520, 4096, "sk", {"grid": 20}),
    (384, 384, 4096, "sk", {"tile_n": 128, "grid": 30}),
    (2944, 1536, 136, "auto", {}),
    (1000, 1000, 1000, "sk", {"tile_n": 128, "grid": 50}),   # 128-deep iterations, ragged k tail
    (520, 640, 192, "dp", {"tile_n": 128}),                  # last iteration: one k-block, one empty
])
@pytest.mark.parametrize("c_type", ["bf16", "f32"])
def test_cta_pairs(m, n, k, mode, attrs, c_type):
    prob = Problem(m, n, k, "bf16", c_type, "normal", seed=m + k, beta=0.5 if c_type == "f32" else 0.0)
    beta = 0.5 if c_type == "f32" else 0.0
    attrs = dict({"tile_n": 256}, **attrs)
    attrs["cluster_m"] = 2
    (C,), info, _ = prob.run(1.0, beta, mode, plan_attrs=attrs)
    assert info["cluster_m"] == 2 and info["ctas"] == 2 * info["grid"]
    prob.check(C, 1.0, beta, f"pairs {m}x{n}x{k} {mode} g={info['grid']}")


def test_column_major_c():
    prob = Problem(200, 328, 512, "bf16", "f32", "normal", seed=6, beta=-1.0)
    (C,), _, _ = prob.run(0.75, -1.0, "sk", c_layout="col", plan_attrs={"grid": 40})
    prob.check(C, 0.75, -1.0, "column-major C")


@pytest.mark.parametrize("tile_n", [64, 128])
def test_run_to_run_bitwise_determinism(tile_n):
    prob = Problem(384, 384, 4096, "bf16", "f32", "normal", seed=7)
    outs, info, _ = prob.run(1.0, 0.0, "sk", plan_attrs={"grid": 148, "tile_n": tile_n}, reps=3)
    assert info["workspace_bytes"] > 0
    for C in outs[1:]:
        assert torch.equal(C, outs[0])
    prob.check(outs[0], 1.0, 0.0, "determinism")


def test_sk_with_g_equal_t_is_bitwise_dp():
    # Section 4: with g equal to the number of tiles Stream-K behaves exactly
    # like the data-parallel decomposition -- the same MMA sequence per tile.
    prob = Problem(384, 640, 1024, "bf16", "f32", "normal", seed=8)
    (C_dp,), i1, _ = prob.run(1.0, 0.0, "dp", plan_attrs={"tile_n": 128, "cluster_m": 1})
    (C_sk,), i2, _ = prob.run(1.0, 0.0, "sk", plan_attrs={"tile_n": 128, "cluster_m": 1, "grid": 15})
    assert i1["tiles"] == 15 and i2["grid"] == 15 and i2["workspace_bytes"] == 0
    assert torch.equal(C_dp, C_sk)
    (C_dp,), i1, _ = prob.run(1.0, 0.0, "dp", plan_attrs={"tile_n": 64})
    (C_sk,), i2, _ = prob.run(1.0, 0.0, "sk", plan_attrs={"tile_n": 64, "grid": 30})
    assert i1["tiles"] == 30 and i2["grid"] == 30 and i2["workspace_bytes"] == 0
    assert torch.equal(C_dp, C_sk)


def test_k_zero_scales_c():
    prob = Problem(100, 72, 0, "bf16", "f32", "normal", seed=9, beta=0.5, lda=8, ldb=8)
    (C,), _, _ = prob.run(2.0, 0.5)
    want = prob.Cin.to(torch.float64) * 0.5
    assert torch.equal(C.to(torch.float64), want)


def test_empty_output_is_noop():
    from paper_2301_03598_gb300 import streamk as sk
    plan = sk.sk_plan(0, 64, 64, "bf16", "bf16", "bf16")
    try:
        sk.sk_gemm(plan, 0, 0, 0, 1.0, 0.0)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
    finally:
        plan.destroy()


def test_shared_workspace_between_plans():
    from paper_2301_03598_gb300 import streamk as sk
    p1 = Problem(384, 384, 2048, "bf16", "f32", "normal", seed=10)
    p2 = Problem(256, 640, 4096, "bf16", "f32", "normal", seed=11)
    plans = [sk.sk_plan(p.m, p.n, p.k, "bf16", "bf16", "f32", mode="sk") for p in (p1, p2)]
    try:
        need = max(pl.get("workspace_bytes") for pl in plans)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        ws.fill_(0xA5)  # garbage: attach must clear the flags
        for pl in plans:
            sk.sk_plan_attach_workspace(pl, ws, need)
        for _ in range(2):
            for pl, p in zip(plans, (p1, p2)):
                C = torch.zeros((p.m, p.n), dtype=torch.float32, device="cuda")
                sk.sk_gemm(pl, p.A.cuda(), p.B.cuda(), C, 1.0, 0.0)
                assert sk.sk_last_error(pl)[0] == sk.SK_OK
                p.check(C.cpu(), 1.0, 0.0, "shared workspace")
    finally:
        for pl in plans:
            pl.destroy()


def test_invalid_arguments_on_device():
    from paper_2301_03598_gb300 import streamk as sk
    plan = sk.sk_plan(128, 128, 64, "bf16", "bf16", "f32")
    try:
        A = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
        C = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
        with pytest.raises(sk.StreamKError) as e:
            sk.sk_gemm(plan, A.data_ptr() + 2, A, C, 1.0, 0.0)   # misaligned A
        assert e.value.status == sk.SK_ERR_INVALID
        with pytest.raises(sk.StreamKError):
            sk.sk_gemm(plan, A, 0, C, 1.0, 0.0)                  # null B
        with pytest.raises(sk.StreamKError):
            plan.set("lda", 60)                                  # below k
        with pytest.raises(sk.StreamKError):
            plan.set("tile_n", 192)
    finally:
        plan.destroy()
    with pytest.raises(sk.StreamKError) as e:
        sk.sk_plan(64, 64, 64, "bf16", "f16", "f32")               # mixed input types
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    with pytest.raises(sk.StreamKError):
        sk.sk_plan(64, 64, 64, a_layout="col")


def _sampled_check(m, n, k, alpha, beta, mode, seed, attrs=None, samples=4096):
    """A full-size GEMM on the device, checked on a seeded sample of entries plus
    whole rows and columns along tile edges (where Stream-K seams and ragged
    tiles are), against the oracle computed entry by entry."""
    import numpy as np
    import oracle
    from gemm_check import bound, check_bound
    from paper_2301_03598_gb300 import inputs, streamk as sk
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    A = torch.randn(m, k, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(n, k, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.randn(m, n, device="cuda", generator=g).to(torch.bfloat16)
    Cin = C.clone()
    plan = sk.sk_plan(m, n, k, "bf16", "bf16", "bf16", "f32", "row", "col", "row", mode)
    try:
        for key, v in (attrs or {}).items():
            plan.set(key, v)
        info = plan.info()
        sk.sk_gemm(plan, A, B, C, alpha, beta)
        st, dev = sk.sk_last_error(plan)
        assert st == sk.SK_OK, (st, dev)
    finally:
        plan.destroy()
    rng = np.random.Generator(np.random.PCG64(seed))
    rows = list(rng.integers(0, m, size=samples))
    cols = list(rng.integers(0, n, size=samples))
    for r in sorted({0, 127, 128, 255, 256, m - 1} & set(range(m))):   # seams along m
        cs = rng.integers(0, n, size=64)
        rows += [r] * len(cs)
        cols += list(cs)
    for c in sorted({0, 127, 128, 255, 256, n - 1} & set(range(n))):   # seams along n
        rs = rng.integers(0, m, size=64)
        rows += list(rs)
        cols += [c] * len(rs)
    rows = np.array(rows, np.int64)
    cols = np.array(cols, np.int64)
    ur, ri = np.unique(rows, return_inverse=True)
    uc, ci = np.unique(cols, return_inverse=True)
    A64 = inputs.widen(A[torch.from_numpy(ur).cuda()].cpu())
    B64 = inputs.widen(B[torch.from_numpy(uc).cuda()].cpu())
    C64in = inputs.widen(Cin[torch.from_numpy(ur).cuda()][:, torch.from_numpy(uc).cuda()].cpu())
    want, absAB = oracle.gemm_entries(ri, ci, A64, B64.T, alpha, beta, C64in)
    got = inputs.widen(C.cpu())[rows, cols]
    cin = C64in[ri, ci]
    check_bound(got, want, bound(k, alpha, beta, absAB, want, cin, "bf16"),
                f"{m}x{n}x{k} {mode} sampled ({info['mode']}, tile_n {info['tile_n']}, g {info['grid']})")


# The extreme-quantisation workloads at full size: BF16 in, FP32 accumulate,
# BF16 out, alpha = 1, beta = 0.5 with random C (sampled entries).
@pytest.mark.parametrize("m,n,k", [(8192, 8192, 8192), (256, 256, 65536), (8192, 128, 4096),
                                   (1536, 1536, 1536), (1664, 1664, 1664)])
@pytest.mark.parametrize("mode", ["auto", "dp", "sk"])
def test_extreme_shapes_full_size_sampled(m, n, k, mode):
    _sampled_check(m, n, k, 1.0, 0.5, mode, seed=m * 7 + k)


@pytest.mark.parametrize("m,n,k,attrs", [(8192, 8192, 8192, {"cluster_m": 2}),
                                         (4096, 4096, 4096, {"cluster_m": 2, "raster_group": 4})])
def test_large_pairs_full_size_sampled(m, n, k, attrs):
    _sampled_check(m, n, k, 1.0, 0.5, "hybrid", seed=11, attrs=attrs)


@pytest.mark.parametrize("m,n,k,tile_n", [(129, 255, 80, 128), (300, 40, 2000, 128),
                                          (64, 520, 136, 256), (1000, 777, 520, 256)])
@pytest.mark.parametrize("c_type", ["bf16", "f32"])
@pytest.mark.parametrize("mode", ["dp", "sk"])
def test_coalesced_store_path(m, n, k, tile_n, c_type, mode):
    """SK_ATTR_STORE = 2: the epilogue writes C with coalesced stores from its
    staging buffer (clipped at the ragged edges) instead of TMA stores."""
    prob = Problem(m, n, k, "bf16", c_type, "normal", seed=m + 3 * k, beta=0.5)
    (C,), info, _ = prob.run(1.0, 0.5, mode, plan_attrs={"tile_n": tile_n, "store": 2})
    prob.check(C, 1.0, 0.5, f"store=2 {m}x{n}x{k} bn={tile_n} {mode}")


@pytest.mark.parametrize("m,n,k", [(1000, 3000, 712), (384, 384, 4096), (4096, 128, 1024)])
def test_autotune_keeps_a_correct_configuration(m, n, k):
    """sk_plan_autotune times every configuration and keeps one; the plan then
    computes the right result with it."""
    prob = Problem(m, n, k, "bf16", "bf16", "normal", seed=m + k)
    plan = sk.sk_plan(m, n, k, "bf16", "bf16", "bf16")
    try:
        A, B = prob.A.cuda(), prob.B.cuda()
        C = torch.zeros(m, n, dtype=torch.bfloat16, device="cuda")
        us = sk.sk_plan_autotune(plan, A, B, C, reps=3)
        info = plan.info()
        assert us > 0 and info["tile_n"] in (64, 128, 256) and info["cluster_m"] in (1, 2)
        assert info["mode"] in (sk.MODES["dp"], sk.MODES["hybrid"], sk.MODES["sk"])
        C.zero_()
        sk.sk_gemm(plan, A, B, C, 1.0, 0.0)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
        prob.check(C.cpu(), 1.0, 0.0, f"autotuned {m}x{n}x{k} {info['tile_n']}/{info['cluster_m']}")
    finally:
        plan.destroy()


@pytest.mark.parametrize("tile_n,cluster_m", [(64, 1), (128, 1), (256, 1), (128, 2), (256, 2)])
@pytest.mark.parametrize("stages", [2, 3])
def test_pipeline_stage_counts(tile_n, cluster_m, stages):
    """A ring cycled through fewer stages than it holds (SK_ATTR_STAGES, the
    autotuner's pipeline-depth choice) computes the same GEMM."""
    m, n, k = 1000, 1000, 1000
    prob = Problem(m, n, k, "bf16", "bf16", "normal", seed=90 + stages)
    attrs = {"tile_n": tile_n, "cluster_m": cluster_m, "stages": stages}
    (C,), info, _ = prob.run(1.0, 0.0, "sk", plan_attrs=attrs)
    prob.check(C, 1.0, 0.0, f"stages={stages} bn={tile_n} cm={cluster_m}")
    plan = sk.sk_plan(m, n, k, "bf16", "bf16", "bf16", mode="sk")
    try:
        plan.set("tile_n", tile_n)
        plan.set("cluster_m", cluster_m)
        full = plan.get("stages")
        plan.set("stages", stages)
        assert plan.get("stages") == stages and full >= 3
        with pytest.raises(sk.StreamKError):
            plan.set("stages", full + 1)
    finally:
        plan.destroy()


@pytest.mark.parametrize("tile_n,cluster_m", [(64, 1), (128, 1), (256, 1), (128, 2), (256, 2)])
@pytest.mark.parametrize("c_type,beta", [("bf16", 0.0), ("f32", 0.5)])
def test_fewer_ring_stages_bitwise_many_tiles(tile_n, cluster_m, c_type, beta):
    """A ring cycled through one stage fewer than it holds, on a data-parallel
    plan with several tiles per unit, a ragged edge and (BLK_N = 64, 16-bit C)
    the split epilogue: the result matches the oracle and, the schedule being
    the same, equals the full ring's bit for bit."""
    m, n, k = 4000, 2600, 256
    prob = Problem(m, n, k, "bf16", c_type, "normal", seed=131 + tile_n + cluster_m, beta=beta)
    base = {"tile_n": tile_n, "cluster_m": cluster_m}
    plan = sk.sk_plan(m, n, k, "bf16", "bf16", c_type, mode="dp")
    try:
        plan.set("tile_n", tile_n)
        plan.set("cluster_m", cluster_m)
        full = plan.get("stages")
        assert plan.info()["tiles"] > plan.info()["grid"]
    finally:
        plan.destroy()
    (C_full,), _, _ = prob.run(1.5, beta, "dp", plan_attrs=base)
    (C_alt,), info, _ = prob.run(1.5, beta, "dp", plan_attrs=dict(base, stages=full - 1))
    assert info["mode"] == sk.MODES["dp"]
    prob.check(C_alt, 1.5, beta, f"ring of full-1 stages bn={tile_n} cm={cluster_m} {c_type}")
    assert torch.equal(C_alt, C_full), "fewer ring stages changed the result"
