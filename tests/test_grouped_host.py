"""Grouped GEMM schedule (Stream-K across problems), without a GPU: the
oracle's grouped schedule is pinned by coverage and by reducing to the
single-problem schedules; the library's host planner must reproduce it."""
import random

import numpy as np
import pytest

from oracle import schedule as S
from paper_2301_03598_gb300 import streamk as sk


def _problems(shapes, tile_n, tile_k):
    return [S.Problem(m, n, k, 128, tile_n, tile_k) for (m, n, k) in shapes]


def _groups(large=True):
    rng = random.Random(2301_03598)
    yield [(300, 500, 700), (128, 128, 4096), (1000, 200, 128), (64, 2048, 1024)]
    yield [(128, 128, 128)]
    yield [(int(np.exp(rng.uniform(np.log(16), np.log(1024)))), rng.choice([128, 256, 512]),
            rng.choice([128, 256, 1024])) for _ in range(24)]
    if large:
        yield [(8192, 1024, 2048), (16, 4096, 1024), (4096, 8192, 8192)]
        # shaped like the grouped workload: m log-uniform in [16, 4096], n, k from {1024..8192}
        yield [(int(np.exp(rng.uniform(np.log(16), np.log(4096)))),
                rng.choice([1024, 2048, 4096, 8192]), rng.choice([1024, 2048, 4096, 8192]))
               for _ in range(64)]


@pytest.mark.parametrize("g", [1, 7, 16, 152])
def test_oracle_grouped_covers_every_iteration_once(g):
    for shapes in _groups(large=False):
        probs = _problems(shapes, 128, 128)
        t = sum(p.tiles for p in probs)
        for sk_tiles in (0, t, t // 2):
            ctas = S.grouped_schedule(probs, g, sk_tiles)
            seen = {}
            for x, segs in enumerate(ctas):
                for s in segs:
                    for i in range(s.local_iter, s.local_iter_end):
                        key = (s.problem, s.tile_idx, i)
                        assert key not in seen
                        seen[key] = x
            assert len(seen) == sum(p.tiles * p.iters_per_tile for p in probs)
            # every split tile: one owner whose peers are exactly the other contributors
            for (pi, tile), xs in _contributors(seen).items():
                owners = [s for x in xs for s in ctas[x]
                          if (s.problem, s.tile_idx) == (pi, tile) and s.role == S.ROLE_OWNER]
                if len(xs) == 1:
                    assert not owners
                else:
                    assert len(owners) == 1 and list(owners[0].peers) == sorted(xs)[1:]


def _contributors(seen):
    out = {}
    for (pi, tile, _), x in seen.items():
        out.setdefault((pi, tile), set()).add(x)
    return out


@pytest.mark.parametrize("g,sk_tiles", [(9, 9), (36, 9), (148, 9), (4, 0), (5, 4)])
def test_oracle_grouped_single_problem_is_the_gemm_schedule(g, sk_tiles):
    prob = S.Problem(384, 384, 4096, 128, 128, 64)
    ctas = S.grouped_schedule([prob], g, sk_tiles)
    single = S.persistent_schedule(prob, g, sk_tiles, prob.tiles_m)
    flat = [(x, 0) + r[1:] for r in single.trace() for x in [r[0]]]
    assert S.grouped_trace([prob], ctas, [prob.tiles_m]) == flat


def test_oracle_grouped_problems_concatenate():
    # two problems scheduled together on g CTAs: Stream-K over the concatenated
    # space equals Stream-K over one problem whose tiles are the union when all
    # tiles have the same iteration count
    a = S.Problem(256, 256, 640, 128, 128, 64)
    b = S.Problem(384, 128, 640, 128, 128, 64)
    ctas = S.grouped_schedule([a, b], 5, a.tiles + b.tiles)
    union = S.stream_k(a.tiles + b.tiles, a.iters_per_tile, 5)
    got = [[(s.tile_idx + (a.tiles if s.problem else 0), s.local_iter, s.local_iter_end, s.role,
             s.peers) for s in segs] for segs in ctas]
    want = [[(s.tile_idx, s.local_iter, s.local_iter_end, s.role, s.peers) for s in segs]
            for segs in union]
    assert got == want


@pytest.mark.parametrize("mode,tile_n,num_sms", [
    ("dp", 0, 152), ("sk", 128, 152), ("hybrid", 256, 152), ("auto", 0, 152), ("auto", 0, 16),
    ("sk", 256, 16), ("hybrid", 128, 148), ("dp", 256, 148)])
def test_host_planner_matches_oracle(mode, tile_n, num_sms):
    for shapes in _groups():
        info, recs = sk.sk_grouped_plan_describe(shapes, mode, tile_n=tile_n, num_sms=num_sms)
        assert info["tile_k"] == (128 if info["tile_n"] == 128 else 64)
        probs = _problems(shapes, info["tile_n"], info["tile_k"])
        assert info["tiles"] == sum(p.tiles for p in probs)
        ctas = S.grouped_schedule(probs, info["grid"], info["sk_tiles"])
        want = S.grouped_trace(probs, ctas, [min(p.tiles_m, 16) for p in probs])
        assert recs == want
        assert info["grid"] <= num_sms
        assert info["max_segments"] >= max(len(c) for c in ctas)
        split = any(r[7] != S.ROLE_WHOLE for r in recs)
        assert (info["workspace_bytes"] > 0) == split
        if mode == "dp":
            assert info["sk_tiles"] == 0 and not split
        if mode == "hybrid":
            assert (info["sk_tiles"], info["tiles"] - info["sk_tiles"]) == \
                S.hybrid_regions(info["tiles"], info["grid"], S.HYBRID_TWO_TILE) or \
                info["sk_tiles"] == info["tiles"]


def test_host_planner_rejects_bad_groups():
    with pytest.raises(sk.StreamKError):
        sk.sk_grouped_plan_describe([(0, 8, 8)])
    with pytest.raises(sk.StreamKError):
        sk.sk_grouped_plan_describe([(8, 8, 8)], tile_n=96)
    with pytest.raises(sk.StreamKError):
        sk.sk_grouped_plan_describe([(8, 8, 8)], mode="hybrid1")


def test_grouped_cluster_trace_hand_worked():
    """Two problems in 256 x 128 pair tiles, BLK_K = 64: problem 0 is 256 x 256
    x 320 (two tiles of 5 iterations), problem 1 is 512 x 128 x 192 (two tiles
    of 3 iterations); 16 iterations in all, Algorithm 5 within one over g = 3
    units: q = 5, r = 1, so unit 0 takes [0, 6), unit 1 [6, 11), unit 2
    [11, 16).  Tiles in the concatenated space: p0 t0 [0, 5), p0 t1 [5, 10),
    p1 t0 [10, 13), p1 t1 [13, 16).  Raster: p0 (tiles_m 1) t0 -> (0, 0),
    t1 -> (0, 1); p1 (tiles_m 2) t0 -> (0, 0), t1 -> (1, 0).
      unit 0: p0 t0 [0, 5) whole; p0 t1 [0, 1) owner, peers 1..1
      unit 1: p0 t1 [1, 5) partial; p1 t0 [0, 1) owner, peers 2..2
      unit 2: p1 t0 [1, 3) partial; p1 t1 [0, 3) whole
    CTA 2x + r runs unit x on 128-row block 2 tm + r; its peers are 2y + r."""
    W, P, O = S.ROLE_WHOLE, S.ROLE_PARTIAL, S.ROLE_OWNER
    probs = [S.Problem(256, 256, 320, 256, 128, 64), S.Problem(512, 128, 192, 256, 128, 64)]
    ctas = S.grouped_schedule(probs, 3, probs[0].tiles + probs[1].tiles)
    units = S.grouped_trace(probs, ctas, [1, 2])
    want = [
        (0, 0, 0, 0, 0, 0, 5, W, -1, -1), (0, 0, 1, 0, 1, 0, 1, O, 2, 2),
        (1, 0, 0, 1, 0, 0, 5, W, -1, -1), (1, 0, 1, 1, 1, 0, 1, O, 3, 3),
        (2, 0, 1, 0, 1, 1, 5, P, -1, -1), (2, 1, 0, 0, 0, 0, 1, O, 4, 4),
        (3, 0, 1, 1, 1, 1, 5, P, -1, -1), (3, 1, 0, 1, 0, 0, 1, O, 5, 5),
        (4, 1, 0, 0, 0, 1, 3, P, -1, -1), (4, 1, 1, 2, 0, 0, 3, W, -1, -1),
        (5, 1, 0, 1, 0, 1, 3, P, -1, -1), (5, 1, 1, 3, 0, 0, 3, W, -1, -1),
    ]
    assert S.grouped_cluster_trace(units, 2) == want
    assert S.grouped_cluster_trace(units, 1) == units


@pytest.mark.parametrize("mode", ["dp", "sk", "hybrid", "auto"])
def test_host_planner_pairs_match_oracle(mode):
    """Grouped plans on CTA pairs: per-unit records equal the oracle's grouped
    schedule over 256-row tiles on num_sms / 2 units."""
    for shapes in _groups():
        info, recs = sk.sk_grouped_plan_describe(shapes, mode, tile_n=256, num_sms=152, cluster_m=2)
        assert info["cluster_m"] == 2 and info["grid"] <= 76
        probs = [S.Problem(m, n, k, 256, 256, 64) for (m, n, k) in shapes]
        assert info["tiles"] == sum(p.tiles for p in probs)
        ctas = S.grouped_schedule(probs, info["grid"], info["sk_tiles"])
        assert recs == S.grouped_trace(probs, ctas, [min(p.tiles_m, 8) for p in probs])
        split = any(r[7] != S.ROLE_WHOLE for r in recs)
        assert (info["workspace_bytes"] > 0) == split
        if split:
            assert info["workspace_bytes"] >= 2 * info["grid"] * 128 * 256 * 4
