"""The C-ABI library without a GPU: it loads, exports every function the
header declares, and its host planner agrees with the oracle's schedule model
(hybrid regions of Section 5.2, grid-size model of Appendix A.1)."""
import ctypes

import pytest

from oracle import schedule as S
from paper_2301_03598_gb300 import build, streamk as sk


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def test_exports_every_header_function():
    names = sk.header_functions()
    assert {"sk_plan", "sk_gemm", "sk_plan_destroy", "sk_last_error"} <= set(names)
    lib = ctypes.CDLL(build.LIB)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings():
    assert sk.sk_status_string(sk.SK_OK) == "SK_OK"
    assert sk.sk_status_string(sk.SK_ERR_TIMEOUT) == "SK_ERR_TIMEOUT"
    assert sk.sk_status_string(99) == "SK_ERR_UNKNOWN"


@pytest.mark.parametrize("case", [(256, 3584, 8192, 108), (1024, 1024, 1024, 64),
                                  (128, 128, 16384, 8)])
def test_grid_model_reproduces_fig7(case):
    m, n, k, g = case
    assert sk.sk_grid_model(m, n, k, 128, 128, 32, 108, (0, 20, 1, 8)) == g


@pytest.mark.parametrize("m,n,k", [(384, 384, 4096), (3000, 200, 128), (128, 128, 65536),
                                   (1536, 1536, 1536), (8192, 128, 4096)])
@pytest.mark.parametrize("coef", [(0, 20, 1, 8), (3, 1, 2, 5), (0, 5, 1, 5)])
def test_grid_model_matches_oracle(m, n, k, coef):
    prob = S.Problem(m, n, k, 128, 128, 64)
    assert sk.sk_grid_model(m, n, k, 128, 128, 64, 148, coef) == \
        S.best_grid_size(prob, 148, *coef)


@pytest.mark.parametrize("t_m,t_n,ipt", [(19, 16, 4), (3, 3, 64), (64, 32, 128), (13, 12, 2),
                                         (38, 8, 3), (12, 12, 24), (2, 2, 1024)])
@pytest.mark.parametrize("p", [148, 132, 4])
def test_hybrid_regions_match_oracle(t_m, t_n, ipt, p):
    m, n, k = t_m * 128, t_n * 128, ipt * 128   # BLK_N = 128 plans iterate BLK_K = 128
    t = t_m * t_n
    for mode, variant in (("hybrid", S.HYBRID_TWO_TILE), ("hybrid1", S.HYBRID_ONE_TILE)):
        d = sk.sk_plan_describe(m, n, k, mode, tile_n=128, cluster_m=1, num_sms=p)
        sk_tiles, dp_tiles = S.hybrid_regions(t, p, variant)
        assert (d["sk_tiles"], d["dp_tiles"]) == (sk_tiles, dp_tiles)
        assert d["tiles"] == t and d["iters_per_tile"] == ipt
        if 0 < sk_tiles < t:
            assert d["grid"] == p
    d = sk.sk_plan_describe(m, n, k, "dp", tile_n=128, cluster_m=1, num_sms=p)
    assert d["sk_tiles"] == 0 and d["grid"] == min(t, p) and d["workspace_bytes"] == 0


def test_describe_config_shapes():
    d = sk.sk_plan_describe(384, 384, 4096, "sk", tile_n=128, cluster_m=1)
    assert (d["tile_n"], d["tile_k"], d["tiles"], d["iters_per_tile"]) == (128, 128, 9, 32)
    assert d["mode_name"] == "sk" and 9 <= d["grid"] <= 148 and d["workspace_bytes"] > 0
    d = sk.sk_plan_describe(8192, 8192, 8192, "hybrid", tile_n=256, cluster_m=1)
    assert (d["tile_n"], d["tiles"], d["mode_name"]) == (256, 2048, "hybrid")
    assert d["sk_tiles"] == 2048 % 148 + 148 and d["dp_tiles"] % 148 == 0
    # CTA pairs: 256 x 256 units on p = 74 pairs
    d = sk.sk_plan_describe(8192, 8192, 8192, "hybrid", tile_n=256, cluster_m=2)
    assert (d["cluster_m"], d["tile_m"], d["tiles"], d["ctas"]) == (2, 256, 1024, 148)
    assert d["sk_tiles"] == 1024 % 74 + 74 and d["dp_tiles"] % 74 == 0
    d = sk.sk_plan_describe(128 * 37, 256, 64, "hybrid", tile_n=256, cluster_m=1)
    assert d["mode_name"] == "hybrid" and d["sk_tiles"] == 37   # below one wave: basic Stream-K


@pytest.mark.parametrize("m,n,k", [(384, 384, 4096), (4096, 128, 4096), (8192, 8192, 8192),
                                   (8192, 8192, 128), (128, 8192, 1024), (1000, 3000, 700),
                                   (256, 256, 65536), (8192, 128, 4096), (1536, 1536, 1536)])
def test_auto_configuration_is_a_candidate(m, n, k):
    """With tile width and cluster size left open the planner returns one of
    the fixed-configuration plans: BLK_N 256 only for n > 128, CTA pairs only
    for m > 128 and BLK_N >= 128."""
    d = sk.sk_plan_describe(m, n, k, num_sms=152)
    assert d["tile_n"] in ((64, 128, 256) if n > 128 else (64, 128))
    assert d["cluster_m"] in ((1, 2) if m > 128 and d["tile_n"] > 64 else (1,))
    fixed = sk.sk_plan_describe(m, n, k, tile_n=d["tile_n"], cluster_m=d["cluster_m"], num_sms=152)
    assert fixed == d
    # a fixed tile width leaves only the cluster size open, and vice versa
    for tn in ((64, 128, 256) if n > 128 else (64, 128)):
        assert sk.sk_plan_describe(m, n, k, tile_n=tn, num_sms=152)["tile_n"] == tn
    assert sk.sk_plan_describe(m, n, k, cluster_m=1, num_sms=152)["cluster_m"] == 1
    assert sk.sk_plan_describe(m, n, k, cluster_m=2, num_sms=152)["tile_n"] in (128, 256)


def test_narrow_tiles_run_on_single_ctas():
    """BLK_N = 64 (128 x 64 tiles, two 64-deep k-blocks per iteration) is planned
    on single CTAs; asking for it with CTA pairs is unsupported."""
    d = sk.sk_plan_describe(384, 384, 4096, "sk", tile_n=64, num_sms=152)
    assert (d["tile_m"], d["tile_n"], d["tile_k"], d["cluster_m"]) == (128, 64, 128, 1)
    assert (d["tiles_m"], d["tiles_n"], d["iters_per_tile"]) == (3, 6, 32)
    assert d["workspace_bytes"] == 4096 * 32 + d["ctas"] * 128 * 64 * 4 or d["workspace_bytes"] == 0
    with pytest.raises(sk.StreamKError) as e:
        sk.sk_plan_describe(384, 384, 4096, "sk", tile_n=64, cluster_m=2, num_sms=152)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    prob = S.Problem(384, 384, 4096, 128, 64, 128)
    sched = S.persistent_schedule(prob, d["grid"], d["sk_tiles"], d["raster_group"])
    assert max(len(c) for c in sched.ctas) <= d["max_segments"]


@pytest.mark.parametrize("m,n,k,mode", [(8192, 8192, 1024, "hybrid"), (4096, 2048, 512, "sk"),
                                        (3000, 2000, 700, "auto"), (2000, 4000, 256, "dp")])
def test_cluster_units_match_oracle(m, n, k, mode):
    d = sk.sk_plan_describe(m, n, k, mode, tile_n=256, cluster_m=2, num_sms=152)
    assert d["cluster_m"] == 2 and d["tile_m"] == 256 and d["ctas"] == 2 * d["grid"]
    prob = S.Problem(m, n, k, 256, 256, 64)
    assert d["tiles"] == prob.tiles and d["grid"] <= 76
    if d["mode_name"] == "hybrid":
        assert (d["sk_tiles"], d["dp_tiles"]) == S.hybrid_regions(prob.tiles, 76, S.HYBRID_TWO_TILE)
    sched = S.persistent_schedule(prob, d["grid"], d["sk_tiles"], d["raster_group"])
    assert max(len(c) for c in sched.ctas) <= d["max_segments"]
    tr = S.cluster_trace(sched, 2)
    assert {r[0] for r in tr} <= set(range(d["ctas"]))
    if d["workspace_bytes"]:
        assert d["workspace_bytes"] >= d["ctas"] * 128 * 256 * 4


def test_max_segments_bounds_every_cta():
    for (m, n, k, mode, g) in [(384, 384, 4096, "sk", 148), (19 * 128, 2048, 256, "hybrid", 0),
                               (1000, 3000, 64, "auto", 0), (128, 128, 64 * 7, "sk", 5)]:
        d = sk.sk_plan_describe(m, n, k, mode, tile_n=128, grid=g, cluster_m=1)
        prob = S.Problem(m, n, k, 128, 128, d["tile_k"])
        sched = S.persistent_schedule(prob, d["grid"], d["sk_tiles"], d["raster_group"])
        assert max(len(c) for c in sched.ctas) <= d["max_segments"]


def test_describe_rejects_bad_arguments():
    with pytest.raises(sk.StreamKError) as e:
        sk.sk_plan_describe(-1, 8, 8)
    assert e.value.status == sk.SK_ERR_INVALID
    with pytest.raises(sk.StreamKError) as e:
        sk.sk_plan_describe(8, 8, 8, tile_n=96)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    with pytest.raises(sk.StreamKError):
        sk.sk_plan_describe(8, 8, 8, mode=9)
    with pytest.raises(sk.StreamKError):
        sk.sk_grid_model(0, 8, 8, 128, 128, 64, 148, (0, 1, 1, 1))


def test_plan_without_device_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sk.StreamKError) as e:
        sk.sk_plan(128, 128, 128)
    assert e.value.status in (sk.SK_ERR_CUDA, sk.SK_ERR_DEVICE)


def test_model_coefficients_per_configuration():
    for tn, cm in [(64, 1), (128, 1), (256, 1), (128, 2), (256, 2)]:
        c = sk.sk_model_coefficients(tn, cm)
        assert len(c) == 6 and all(v > 0 for v in c), (tn, cm, c)
    with pytest.raises(sk.StreamKError) as e:
        sk.sk_model_coefficients(64, 2)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED


@pytest.mark.parametrize("coef", [(1.0, 2.0, 3.0, 4.0, 5.0, 6.0), (4.0, 3.0, 0.25, 0.5, 0.1, 1.5)])
def test_model_time_closed_forms(coef):
    a, b, c, d, e, f = coef
    # data-parallel, one full wave: a + max(c * ipt, f) + e
    assert sk.sk_model_time(1024, 1024, 1024, "dp", tile_n=128, cluster_m=1, num_sms=152,
                            coef=coef) == pytest.approx(a + max(c * 8, f) + e)
    # two waves of 64 tiles on 32 units (ipt = 8): a + 2 * max(c * 8, f) + 2 e
    assert sk.sk_model_time(1024, 1024, 1024, "dp", tile_n=128, cluster_m=1, num_sms=32,
                            coef=coef) == pytest.approx(a + 2 * max(c * 8, f) + 2 * e)
    # basic Stream-K of one 128 x 128 tile with ipt = 32 over g = 4: shares of 8
    # iterations, 4 contributors, split: a + b + 8 c + 3 d + e * segs, where a
    # share of q = 8 < ipt touches at most ceil((q + 1) / ipt) + 1 = 2 segments
    assert sk.sk_model_time(128, 128, 4096, "sk", tile_n=128, cluster_m=1, grid=4, num_sms=152,
                            coef=coef) == pytest.approx(a + b + 8 * c + 3 * d + 2 * e)
    # k = 128 (ipt = 1): every iteration of a share is a whole tile and takes
    # the tile period, so the hybrid over all 225 tiles on 152 units prices
    # like two data-parallel waves
    hyb = sk.sk_model_time(544, 5712, 128, "hybrid", tile_n=128, cluster_m=1, num_sms=152,
                           coef=coef)
    info = sk.sk_plan_describe(544, 5712, 128, "hybrid", tile_n=128, cluster_m=1, num_sms=152)
    assert info["iters_per_tile"] == 1 and info["sk_tiles"] == info["tiles"] == 225
    assert hyb == pytest.approx(a + 2 * max(c, f) + e * (-(-2 // 1) + 1))


@pytest.mark.parametrize("m,n,k", [(384, 384, 4096), (544, 5712, 128), (1000, 776, 1104),
                                   (592, 192, 7312), (4016, 304, 6736), (8192, 8192, 8192),
                                   (256, 256, 65536), (3000, 200, 128)])
def test_auto_is_the_argmin_of_the_exported_model(m, n, k):
    """AUTO's pick has the smallest modelled time (splits raised by the 10%
    margin) among the fixed candidates it ranks."""
    p = 152
    margin = lambda info, us: us * (1.1 if info["workspace_bytes"] > 0 else 1.0)  # noqa: E731
    auto = sk.sk_plan_describe(m, n, k, "auto", num_sms=p)
    best = margin(auto, sk.sk_model_time(m, n, k, "auto", num_sms=p))
    for tn in (64, 128, 256):
        for cm in (1, 2):
            if tn == 64 and cm == 2:
                continue
            if cm == 2 and m <= 128:
                continue
            if tn == 256 and n <= 128:
                continue
            for mode in ("dp", "hybrid"):
                info = sk.sk_plan_describe(m, n, k, mode, tile_n=tn, cluster_m=cm, num_sms=p)
                us = sk.sk_model_time(m, n, k, mode, tile_n=tn, cluster_m=cm, num_sms=p)
                assert best <= margin(info, us) + 1e-9, (mode, tn, cm)
