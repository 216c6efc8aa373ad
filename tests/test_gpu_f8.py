"""Block-scaled E4M3 GEMMs on the GPU through the C ABI (sk_gemm_scaled,
sk_grouped_gemm_scaled) against the FP64 oracle on the same codes and scales.

Bound per element (gemm_check.bound with |A||B| of the dequantized operands):
every k-block's products are exact in FP32 and summed by the tensor cores in
FP32, then scaled (one rounding) and added to the FP32 running sum (one
rounding per k-block), and Stream-K partials are added in FP32, all within
k * 2^-22 relative to sum |a||b| for k >= 16."""
import numpy as np
import pytest
import torch

from oracle import e4m3
from paper_2301_03598_gb300 import inputs
from paper_2301_03598_gb300 import streamk as sk

from gemm_check import bound, check_bound

pytestmark = pytest.mark.gpu


class F8Problem:
    def __init__(self, m, n, k, c_type="bf16", seed=0, beta=0.0, dist="normal",
                 scale_spread=False):
        self.m, self.n, self.k, self.c_type = m, n, k, c_type
        self.qA, self.sA = inputs.host_e4m3_matrix(m, k, dist, seed * 7 + 1)
        self.qB, self.sB = inputs.host_e4m3_matrix(n, k, dist, seed * 7 + 2)
        if scale_spread:
            # exact powers of two per block, 2^-8 .. 2^8: a scale taken from
            # the wrong block is off by orders of magnitude
            g = np.random.Generator(np.random.PCG64(seed + 99))
            self.sA = self.sA * torch.from_numpy(np.exp2(g.integers(-8, 9, self.sA.shape)).astype(np.float32))
            self.sB = self.sB * torch.from_numpy(np.exp2(g.integers(-8, 9, self.sB.shape)).astype(np.float32))
        if beta != 0.0:
            self.Cin, _ = inputs.host_matrix(m, n, c_type, dist, seed * 7 + 3)
        else:
            self.Cin = torch.zeros((m, n), dtype=inputs.DTYPES[c_type])

    def oracle(self, alpha, beta):
        Cin64 = inputs.widen(self.Cin)
        return e4m3.gemm(self.qA.numpy(), self.sA.numpy(), self.qB.numpy(), self.sB.numpy(),
                         alpha, beta, Cin64 if beta != 0.0 else None)

    def run(self, alpha=1.0, beta=0.0, mode="auto", attrs=None, reps=1, c_layout="row"):
        plan = sk.sk_plan(self.m, self.n, self.k, "e4m3", "e4m3", self.c_type, "f32", "row",
                          "col", c_layout, mode)
        try:
            for key, v in (attrs or {}).items():
                plan.set(key, v)
            A, B = self.qA.cuda(), self.qB.cuda()
            sA, sB = self.sA.cuda(), self.sB.cuda()
            outs = []
            for _ in range(reps):
                C = self.Cin.clone().cuda() if c_layout == "row" else self.Cin.t().contiguous().cuda()
                sk.sk_gemm_scaled(plan, A, B, sA, sB, C, alpha, beta)
                st, dev = sk.sk_last_error(plan)
                assert st == sk.SK_OK, (sk.sk_status_string(st), dev)
                out = C.cpu()
                outs.append(out if c_layout == "row" else out.t().contiguous())
            return outs, plan.info()
        finally:
            plan.destroy()

    def check(self, C, alpha, beta, what=""):
        C64, absAB = self.oracle(alpha, beta)
        b = bound(self.k, alpha, beta, absAB, C64, inputs.widen(self.Cin), self.c_type)
        return check_bound(inputs.widen(C), C64, b, what)


SHAPES = [(384, 384, 4096), (300, 260, 1008), (129, 1000, 144), (16, 128, 16), (1000, 520, 2048),
          (1, 1, 16)]


@pytest.mark.parametrize("mode", ["auto", "dp", "sk", "hybrid"])
@pytest.mark.parametrize("shape", SHAPES)
def test_f8_matches_oracle(shape, mode):
    p = F8Problem(*shape, seed=3)
    outs, info = p.run(1.0, 0.0, mode, {"cluster_m": 1, "tile_n": 128})
    assert info["tile_n"] == 128 and info["tile_k"] == 256 and info["cluster_m"] == 1
    p.check(outs[0], 1.0, 0.0, f"e4m3 {shape} {mode}")


def _modelled_width(m, n, k, num_sms):
    """The width (128 or 256) whose AUTO schedule has the smaller modelled
    time, the rule an AUTO E4M3 plan follows: E4M3 rows are planned as 16-bit
    rows of k/2, a split schedule carries the planner's 10% margin, and a tie
    keeps 128."""
    best = {}
    for tn in (128, 256):
        if tn == 256 and n <= 128:
            continue
        info = sk.sk_plan_describe(m, n, k // 2, "auto", tile_n=tn, cluster_m=1, num_sms=num_sms)
        us = sk.sk_model_time(m, n, k // 2, "auto", tile_n=tn, num_sms=num_sms, cluster_m=1)
        best[tn] = us * (1.10 if info["workspace_bytes"] > 0 else 1.0)
    return min(best, key=lambda t: (best[t], t))


@pytest.mark.parametrize("shape", [(384, 384, 4096), (1000, 1100, 2048), (2048, 2048, 1024),
                                   (129, 1000, 144)])
def test_f8_auto_width_follows_the_model(shape):
    p = F8Problem(*shape, seed=18)
    outs, info = p.run(1.0, 0.0, "auto")
    assert info["cluster_m"] == 1
    assert info["tile_n"] == _modelled_width(*shape, info["num_sms"])
    assert info["tile_k"] == (256 if info["tile_n"] == 128 else 128)
    p.check(outs[0], 1.0, 0.0, f"e4m3 auto width {shape} ({info['tile_n']})")


@pytest.mark.parametrize("mode,grid", [("dp", 0), ("sk", 0), ("sk", 37), ("hybrid", 0)])
@pytest.mark.parametrize("shape", [(1000, 520, 2048), (384, 384, 4096), (129, 1000, 144)])
def test_f8_cta_pairs(shape, mode, grid):
    # 256 x 128 tiles on CTA pairs (two-SM E4M3 MMAs), ragged rows and k
    p = F8Problem(*shape, seed=12, scale_spread=True)
    attrs = {"cluster_m": 2}
    if grid:
        attrs["grid"] = grid
    outs, info = p.run(1.0, 0.0, mode, attrs)
    assert info["cluster_m"] == 2
    p.check(outs[0], 1.0, 0.0, f"e4m3 pair {shape} {mode} g={grid}")


@pytest.mark.parametrize("mode,grid", [("dp", 0), ("sk", 0), ("sk", 37), ("hybrid", 0)])
@pytest.mark.parametrize("shape", [(1000, 520, 2048), (384, 384, 4096), (129, 1000, 144),
                                   (300, 260, 1008), (16, 128, 16), (1, 1, 16)])
def test_f8_wide_tiles(shape, mode, grid):
    # 128 x 256 tiles on single CTAs (one k-block of 128 per MAC-loop
    # iteration, two 256-column product buffers): ragged rows, columns and k
    p = F8Problem(*shape, seed=14, scale_spread=True)
    attrs = {"tile_n": 256}
    if grid:
        attrs["grid"] = grid
    outs, info = p.run(1.0, 0.0, mode, attrs)
    assert info["tile_n"] == 256 and info["tile_k"] == 128 and info["cluster_m"] == 1
    p.check(outs[0], 1.0, 0.0, f"e4m3 wide {shape} {mode} g={grid}")


@pytest.mark.parametrize("c_type,layout", [("f32", "row"), ("f16", "row"), ("bf16", "col"),
                                           ("f32", "col")])
def test_f8_wide_tiles_output_types_and_beta(c_type, layout):
    p = F8Problem(520, 600, 1024, c_type=c_type, seed=15, beta=0.5)
    outs, info = p.run(1.5, 0.5, "sk", {"tile_n": 256, "grid": 41}, c_layout=layout)
    assert info["tile_n"] == 256
    p.check(outs[0], 1.5, 0.5, f"e4m3 wide beta {c_type} {layout}")


def test_f8_wide_tiles_bitwise_reproducible():
    p = F8Problem(640, 768, 8192, seed=16)
    outs, _ = p.run(1.0, 0.0, "sk", {"tile_n": 256, "grid": 100}, reps=3)
    assert all(torch.equal(outs[0], o) for o in outs[1:])
    p.check(outs[0], 1.0, 0.0, "e4m3 wide reproducible")


def test_f8_autotune_single_plan():
    # the autotuner ranks 128-wide tiles (single CTAs and pairs) and 256-wide
    # tiles (single CTAs); whatever it keeps must still match the oracle
    p = F8Problem(1000, 1100, 2048, seed=17, scale_spread=True)
    plan = sk.sk_plan(p.m, p.n, p.k, "e4m3", "e4m3", "bf16")
    try:
        A, B, sA, sB = p.qA.cuda(), p.qB.cuda(), p.sA.cuda(), p.sB.cuda()
        C = torch.empty(p.m, p.n, dtype=torch.bfloat16, device="cuda")
        us = sk.sk_plan_autotune_scaled(plan, A, B, sA, sB, C, reps=2)
        assert us > 0.0
        info = plan.info()
        assert info["tile_n"] in (128, 256)
        assert info["tile_n"] == 128 or info["cluster_m"] == 1
        C.fill_(float("nan"))
        sk.sk_gemm_scaled(plan, A, B, sA, sB, C)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
        out = C.cpu()
    finally:
        plan.destroy()
    p.check(out, 1.0, 0.0, f"e4m3 autotuned ({info['tile_n']}, {info['cluster_m']})")


@pytest.mark.parametrize("tile_n,mode,grid", [(128, "sk", 90), (256, "sk", 61), (256, "hybrid", 0)])
def test_f8_independent_inputs_back_to_back(tile_n, mode, grid):
    # SK_ATTR_INDEPENDENT_INPUTS: the MAC loop may overlap the previous launch,
    # while C and the shared fixup workspace keep stream order
    p = F8Problem(700, 900, 3072, seed=19, scale_spread=True)
    plan = sk.sk_plan(p.m, p.n, p.k, "e4m3", "e4m3", "f32", mode=mode)
    try:
        plan.set("tile_n", tile_n)
        if grid:
            plan.set("grid", grid)
        plan.set("independent_inputs", 1)
        A, B, sA, sB = p.qA.cuda(), p.qB.cuda(), p.sA.cuda(), p.sB.cuda()
        outs = [torch.zeros(p.m, p.n, dtype=torch.float32, device="cuda") for _ in range(8)]
        for C in outs:
            sk.sk_gemm_scaled(plan, A, B, sA, sB, C)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
        assert plan.info()["tile_n"] == tile_n
        for C in outs[1:]:
            assert torch.equal(C, outs[0])
        first = outs[0].cpu()
    finally:
        plan.destroy()
    p.check(first, 1.0, 0.0, f"e4m3 independent {tile_n} {mode}")


@pytest.mark.parametrize("tile_n", [128, 256])
def test_f8_independent_inputs_chain_into_one_c(tile_n):
    # C_{j+1} = A_j B_j + C_j: each launch reads the C its predecessor wrote
    m, n, k = 520, 640, 1024
    probs = [F8Problem(m, n, k, "f32", seed=40 + j) for j in range(4)]
    plan = sk.sk_plan(m, n, k, "e4m3", "e4m3", "f32", mode="sk")
    try:
        plan.set("tile_n", tile_n)
        plan.set("grid", 77)
        plan.set("independent_inputs", 1)
        C = torch.zeros(m, n, dtype=torch.float32, device="cuda")
        ops = [(q.qA.cuda(), q.qB.cuda(), q.sA.cuda(), q.sB.cuda()) for q in probs]
        for A, B, sA, sB in ops:
            sk.sk_gemm_scaled(plan, A, B, sA, sB, C, 1.0, 1.0)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
        got = inputs.widen(C.cpu())
    finally:
        plan.destroy()
    parts = [q.oracle(1.0, 0.0) for q in probs]
    want = sum(c for c, _ in parts)
    absab = sum(ab for _, ab in parts)
    # four FP32 block-scaled sums within k * 2^-22 |A||B| each, plus the chain's FP32 adds
    tol = 4 * k * 2.0 ** -22 * absab + 2.0 ** -20 * np.abs(want) + 1e-30
    assert np.all(np.abs(got - want) <= tol)


@pytest.mark.parametrize("grid", [7, 40, 143])
def test_f8_split_tiles_with_spread_scales(grid):
    # 9 tiles of 16 iterations (two k-blocks of 128 each) over g CTAs: every
    # tile split, owners fix up
    p = F8Problem(384, 384, 4096, seed=5, scale_spread=True)
    outs, info = p.run(1.0, 0.0, "sk", {"cluster_m": 1, "grid": grid})
    assert info["grid"] == grid
    p.check(outs[0], 1.0, 0.0, f"e4m3 spread scales g={grid}")


@pytest.mark.parametrize("c_type", ["f32", "f16", "bf16"])
def test_f8_alpha_beta_output_types(c_type):
    p = F8Problem(520, 300, 1024, c_type=c_type, seed=7, beta=0.5)
    outs, _ = p.run(1.5, 0.5, "hybrid")
    p.check(outs[0], 1.5, 0.5, f"e4m3 beta {c_type}")


def test_f8_column_major_c_and_uniform_values():
    p = F8Problem(260, 390, 656, seed=8, dist="uniform", scale_spread=True)
    outs, _ = p.run(1.0, 0.0, "sk", {"grid": 33}, c_layout="col")
    p.check(outs[0], 1.0, 0.0, "e4m3 column-major C")


def test_f8_bitwise_reproducible():
    p = F8Problem(640, 384, 8192, seed=9)
    outs, _ = p.run(1.0, 0.0, "sk", {"cluster_m": 1, "grid": 100}, reps=3)
    assert all(torch.equal(outs[0], o) for o in outs[1:])
    p.check(outs[0], 1.0, 0.0, "e4m3 reproducible")


def test_f8_entry_point_contract():
    plan = sk.sk_plan(256, 256, 256, "e4m3", "e4m3", "bf16")
    try:
        A = torch.zeros(256, 256, dtype=torch.uint8, device="cuda")
        C = torch.zeros(256, 256, dtype=torch.bfloat16, device="cuda")
        s = torch.ones(2, 2, dtype=torch.float32, device="cuda")
        with pytest.raises(sk.StreamKError) as e:
            sk.sk_gemm(plan, A, A, C)                    # scales are required
        assert e.value.status == sk.SK_ERR_INVALID
        with pytest.raises(sk.StreamKError) as e:
            plan.set("tile_n", 64)
        assert e.value.status == sk.SK_ERR_UNSUPPORTED
        # 256-wide E4M3 tiles run on single CTAs only
        plan.set("tile_n", 256)
        with pytest.raises(sk.StreamKError) as e:
            plan.set("cluster_m", 2)
        assert e.value.status == sk.SK_ERR_UNSUPPORTED
        plan.set("tile_n", 128)
        plan.set("cluster_m", 2)
        with pytest.raises(sk.StreamKError) as e:
            plan.set("tile_n", 256)
        assert e.value.status == sk.SK_ERR_UNSUPPORTED
        plan.set("cluster_m", 1)
        assert plan.info()["tile_n"] == 128 and plan.info()["cluster_m"] == 1
        sk.sk_gemm_scaled(plan, A, A, s, s, C)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
        assert float(C.float().abs().max()) == 0.0
    finally:
        plan.destroy()
    plan16 = sk.sk_plan(128, 128, 128, "bf16", "bf16", "bf16")
    try:
        X = torch.zeros(128, 128, dtype=torch.bfloat16, device="cuda")
        s = torch.ones(1, 1, dtype=torch.float32, device="cuda")
        with pytest.raises(sk.StreamKError) as e:
            sk.sk_gemm_scaled(plan16, X, X, s, s, X)     # 16-bit plans take no scales
        assert e.value.status == sk.SK_ERR_INVALID
    finally:
        plan16.destroy()


@pytest.mark.parametrize("mode,attrs", [("auto", {}), ("sk", {"tile_n": 128, "grid": 151}),
                                        ("dp", {"tile_n": 128}), ("sk", {"tile_n": 256})])
def test_f8_large_sampled_entries(mode, attrs):
    # 4096 x 4096 x 8192 on device-drawn operands: 4,096 sampled outputs plus
    # entries along tile edges (Stream-K seams, ragged-free but split tiles)
    m, n, k = 4096, 4096, 8192
    qA, sA = inputs.device_e4m3_matrix(m, k, 31, "cuda")
    qB, sB = inputs.device_e4m3_matrix(n, k, 32, "cuda")
    C = torch.full((m, n), float("nan"), dtype=torch.bfloat16, device="cuda")
    plan = sk.sk_plan(m, n, k, "e4m3", "e4m3", "bf16", mode=mode)
    try:
        for key, v in attrs.items():
            plan.set(key, v)
        sk.sk_gemm_scaled(plan, qA, qB, sA, sB, C)
        assert sk.sk_last_error(plan)[0] == sk.SK_OK
        info = plan.info()
    finally:
        plan.destroy()
    if mode == "auto":
        assert info["tile_n"] == 256  # a wave or more of 128 x 256 tiles
    g = np.random.Generator(np.random.PCG64(5))
    rows, cols = list(g.integers(0, m, 4096)), list(g.integers(0, n, 4096))
    for e in (0, 127, 128, 2047, 2048, m - 1):
        rows += [e] * 64 + list(g.integers(0, m, 64))
        cols += list(g.integers(0, n, 64)) + [e] * 64
    rows, cols = np.array(rows, np.int64), np.array(cols, np.int64)
    want, absAB = e4m3.gemm_entries(rows, cols, qA.cpu().numpy(), sA.cpu().numpy(),
                                    qB.cpu().numpy(), sB.cpu().numpy())
    got = C.cpu()[torch.from_numpy(rows), torch.from_numpy(cols)]
    b = bound(k, 1.0, 0.0, absAB, want, None, "bf16")
    check_bound(inputs.widen(got), want, b,
                f"e4m3 4096x4096x8192 sampled ({info['mode']}, g {info['grid']})")


GROUP = [(300, 500, 704), (128, 128, 4096), (1000, 200, 128), (64, 520, 1024), (17, 1000, 304),
         (777, 96, 2000)]


def _grouped(shapes, mode, c_type="bf16", beta=0.0, attrs=None, seed=0, autotune=False):
    probs = [F8Problem(m, n, k, c_type, seed=seed + 13 * i, beta=beta, scale_spread=(i % 2 == 1))
             for i, (m, n, k) in enumerate(shapes)]
    plan = sk.sk_grouped_plan(shapes, "e4m3", c_type, mode)
    try:
        for key, v in (attrs or {}).items():
            plan.set(key, v)
        As = [p.qA.cuda() for p in probs]
        Bs = [p.qB.cuda() for p in probs]
        SAs = [p.sA.cuda() for p in probs]
        SBs = [p.sB.cuda() for p in probs]
        if autotune:
            scratch = [torch.empty(p.m, p.n, dtype=inputs.DTYPES[c_type], device="cuda")
                       for p in probs]
            sk.sk_grouped_autotune_scaled(plan, As, Bs, SAs, SBs, scratch, reps=2)
        Cs = [p.Cin.clone().cuda() for p in probs]
        alphas = [1.0 + 0.25 * (i % 3) for i in range(len(shapes))]
        sk.sk_grouped_gemm_scaled(plan, As, Bs, SAs, SBs, Cs, alphas, [beta] * len(shapes))
        st, dev = sk.sk_grouped_last_error(plan)
        assert st == sk.SK_OK, (sk.sk_status_string(st), dev)
        return probs, [c.cpu() for c in Cs], alphas, plan.info()
    finally:
        plan.destroy()


@pytest.mark.parametrize("mode,attrs", [("auto", {}), ("dp", {}), ("sk", {"grid": 29}),
                                        ("hybrid", {}), ("dp", {"tile_n": 256}),
                                        ("sk", {"tile_n": 256, "grid": 31}),
                                        ("hybrid", {"tile_n": 256})])
def test_f8_grouped_matches_oracle(mode, attrs):
    probs, outs, alphas, info = _grouped(GROUP, mode, attrs=attrs, seed=4)
    assert info["tile_n"] == attrs.get("tile_n", 128)
    for p, C, al in zip(probs, outs, alphas):
        p.check(C, al, 0.0, f"e4m3 grouped {mode} {p.m}x{p.n}x{p.k}")


def test_f8_grouped_beta_f32_and_autotune():
    probs, outs, alphas, info = _grouped(GROUP, "auto", "f32", 0.5, seed=6, autotune=True)
    for p, C, al in zip(probs, outs, alphas):
        p.check(C, al, 0.5, f"e4m3 grouped autotuned {p.m}x{p.n}x{p.k}")
