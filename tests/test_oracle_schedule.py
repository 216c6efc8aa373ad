"""Pins of the oracle schedule model against the paper's worked examples
(tests/golden/paper_schedule_examples.json, each entry citing its passage),
against the invariants the paper states, and against brute-force checks.
"""
import json
import os

import pytest

from oracle import schedule as S

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                     "paper_schedule_examples.json")))


def covered(ctas):
    """Multiset of (tile, local iteration) pairs executed by a schedule."""
    out = []
    for segs in ctas:
        for s in segs:
            out.extend((s.tile_idx, i) for i in range(s.local_iter, s.local_iter_end))
    return out


def test_dp_ceilings():
    for key in ("dp_ceiling_9_tiles", "dp_ceiling_18_tiles"):
        ex = GOLDEN[key]
        prob = S.Problem(ex["m"], ex["n"], ex["k"], ex["blk_m"], ex["blk_n"], 1)
        assert prob.tiles == ex["tiles"]
        assert len(S.data_parallel(prob)) == ex["tiles"]
        assert S.dp_utilization(prob.tiles, ex["p"]) == pytest.approx(ex["utilization"])


def test_fixed_split_example():
    ex = GOLDEN["fixed_split_s2"]
    prob = S.Problem(ex["m"], ex["n"], ex["k"], ex["blk_m"], ex["blk_n"], 1)
    fs = S.fixed_split(prob, ex["s"])
    ctas = [segs for row in fs for segs in row]
    assert len(ctas) == ex["ctas"]
    for segs in ctas:
        (seg,) = segs
        assert (seg.local_iter_end - seg.local_iter) * prob.blk_k == ex["k_per_cta"]
    assert S.dp_utilization(len(ctas), ex["p"]) == pytest.approx(ex["utilization"])
    assert sorted(covered(ctas)) == sorted((t, i) for t in range(prob.tiles)
                                           for i in range(prob.iters_per_tile))


def test_basic_stream_k_example():
    ex = GOLDEN["basic_stream_k_g4"]
    prob = S.Problem(ex["m"], ex["n"], ex["k"], ex["blk_m"], ex["blk_n"], ex["blk_k"])
    assert prob.iters_per_tile == ex["iters_per_tile"]
    ctas = S.stream_k(prob.tiles, prob.iters_per_tile, ex["g"])
    for segs in ctas:
        n_iters = sum(s.local_iter_end - s.local_iter for s in segs)
        assert n_iters == ex["iters_per_cta"]
        assert n_iters * prob.blk_k == ex["k_per_cta"]
    assert S.stream_k_utilization(prob.total_iters, ex["g"]) == pytest.approx(ex["utilization"])


def test_skew_offsets_example():
    ex = GOLDEN["skew_offsets"]
    prob = S.Problem(ex["m"], ex["n"], ex["k"], ex["blk_m"], ex["blk_n"], ex["blk_k"])
    ctas = S.stream_k(prob.tiles, prob.iters_per_tile, ex["g"])
    offsets = [segs[0].local_iter * prob.blk_k for segs in ctas]
    assert offsets == ex["first_k_offsets"]


def test_fig7_printed_quantities_and_model():
    ex = GOLDEN["fig7_model"]
    for case in ex["cases"]:
        prob = S.Problem(case["m"], case["n"], case["k"], ex["blk_m"], ex["blk_n"], ex["blk_k"])
        assert prob.tiles == case["tiles"]
        assert prob.iters_per_tile == case["iters_per_tile"]
        shares = sorted({S.cta_iter_range(x, prob.total_iters, case["g_best"])[1]
                         - S.cta_iter_range(x, prob.total_iters, case["g_best"])[0]
                         for x in range(case["g_best"])})
        assert shares == case["iters_per_cta"]
        # The constants a..d are not published; (a, b, c, d) = (0, 20, 1, 8)
        # (in units of one MAC-loop iteration) reproduces all three printed
        # optima with ties going to the smallest g.
        assert S.best_grid_size(prob, ex["p"], 0, 20, 1, 8) == case["g_best"]


def test_fig7_model_terms_by_hand():
    # 128x128x16384 with 128x128x32 tiles: one tile, 512 iterations.
    prob = S.Problem(128, 128, 16384, 128, 128, 32)
    assert S.iters_per_cta_model(prob, 8) == 64
    assert S.fixup_peers_model(prob, 8) == 8
    assert S.time_cta_model(prob, 8, 1, 2, 3, 4) == 1 + 2 + 3 * 64 + 4 * 7
    assert S.iters_per_cta_model(prob, 7) == 74        # ceil(512/7)
    assert S.fixup_peers_model(prob, 7) == 7           # ceil(512/74)
    assert S.time_cta_model(prob, 1, 1, 2, 3, 4) == 1 + 3 * 512


def test_fig8_strong_scaling():
    ex = GOLDEN["fig8_strong_scaling"]
    prob = S.Problem(ex["m"], ex["n"], ex["k"], ex["blk_m"], ex["blk_n"], 32)
    assert len(S.data_parallel(prob)) == ex["dp_ctas"]
    ctas = S.stream_k(prob.tiles, prob.iters_per_tile, ex["p"])
    assert [sum(s.local_iter_end - s.local_iter for s in c) for c in ctas] == [3, 3, 3, 3]
    assert S.dp_utilization(1, ex["p"]) == 0.25
    assert S.stream_k_utilization(prob.total_iters, ex["p"]) == 1.0


SHAPES = [(1, 1, 1), (1, 37, 11), (9, 32, 4), (9, 64, 4), (21, 32, 4), (56, 256, 108),
          (3, 1000, 148), (148, 3, 148), (300, 5, 148), (7, 7, 49), (8, 5, 152), (1, 3, 4)]


@pytest.mark.parametrize("t,ipt,g", SHAPES)
def test_stream_k_covers_every_iteration_once(t, ipt, g):
    ctas = S.stream_k(t, ipt, g)
    got = sorted(covered(ctas))
    assert got == [(tt, i) for tt in range(t) for i in range(ipt)]
    shares = [sum(s.local_iter_end - s.local_iter for s in c) for c in ctas]
    assert max(shares) - min(shares) <= 1                      # within one
    assert len(ctas) == g and sum(shares) == t * ipt
    for x, segs in enumerate(ctas):
        for j, s in enumerate(segs):
            started = s.local_iter == 0
            ended = s.local_iter_end == ipt
            if s.role == S.ROLE_PARTIAL:
                assert not started and j == 0                     # only a first segment spills
            elif s.role == S.ROLE_OWNER:
                assert started and not ended and j == len(segs) - 1
                # peers: exactly the later CTAs that touch this tile
                touch = sorted({y for y, o in enumerate(ctas) for q in o
                                if q.tile_idx == s.tile_idx and y != x})
                assert list(s.peers) == touch and all(y > x for y in touch)
            else:
                assert started and ended


@pytest.mark.parametrize("t,ipt,g", [(9, 32, 4), (21, 32, 4), (200, 7, 148), (148, 64, 148),
                                     (1000, 3, 148)])
def test_at_most_two_ctas_per_tile_when_t_ge_g(t, ipt, g):
    ctas = S.stream_k(t, ipt, g)
    per_tile = {}
    for x, segs in enumerate(ctas):
        for s in segs:
            per_tile.setdefault(s.tile_idx, set()).add(x)
    assert max(len(v) for v in per_tile.values()) <= 2


def test_g_equals_t_is_data_parallel():
    for t, ipt in [(9, 32), (64, 32), (148, 5)]:
        ctas = S.stream_k(t, ipt, t)
        assert ctas == S.data_parallel(S.Problem(t * 128, 128, ipt * 64, 128, 128, 64))


@pytest.mark.parametrize("t,ipt,s", [(9, 32, 2), (9, 32, 4), (3, 12, 3), (5, 64, 8)])
def test_g_multiple_of_t_is_fixed_split(t, ipt, s):
    # With s dividing iters_per_tile, CTA x*s + y of Stream-K (g = s*t) runs
    # exactly split y of tile x of Algorithm 4.
    prob = S.Problem(t * 128, 128, ipt * 64, 128, 128, 64)
    sk = S.stream_k(t, ipt, s * t)
    fs = S.fixed_split(prob, s)
    for x in range(t):
        for y in range(s):
            (a,) = sk[x * s + y]
            (b,) = fs[x][y]
            assert (a.tile_idx, a.local_iter, a.local_iter_end) == \
                (b.tile_idx, b.local_iter, b.local_iter_end)
            if y == 0:
                assert a.role == S.ROLE_OWNER and [p - x * s for p in a.peers] == list(b.peers)
            else:
                assert a.role == S.ROLE_PARTIAL == b.role


def test_hybrid_regions_examples():
    # 896x384 on four SMs (Fig. 3): 21 tiles, w = 5 full waves, one tile left.
    assert S.hybrid_regions(21, 4, S.HYBRID_ONE_TILE) == (1, 20)
    assert S.hybrid_regions(21, 4, S.HYBRID_TWO_TILE) == (5, 16)
    # perfect quantization and the no-full-wave case
    assert S.hybrid_regions(16, 4, S.HYBRID_TWO_TILE) == (0, 16)
    assert S.hybrid_regions(3, 4, S.HYBRID_TWO_TILE) == (3, 0)
    assert S.hybrid_regions(3, 4, S.HYBRID_ONE_TILE) == (3, 0)


@pytest.mark.parametrize("t,p,ipt", [(21, 4, 32), (149, 148, 8), (4096, 148, 128),
                                     (300, 148, 3), (296 + 17, 148, 64)])
def test_two_tile_hybrid_one_peer(t, p, ipt):
    """Two-tile SK + DP: every Stream-K CTA gets between one and two tiles of
    iterations and every accumulating CTA has exactly one peer (Section 5.2)."""
    sk_tiles, dp_tiles = S.hybrid_regions(t, p, S.HYBRID_TWO_TILE)
    assert sk_tiles + dp_tiles == t and dp_tiles % p == 0
    sched = S.persistent_schedule(S.Problem(t * 128, 128, ipt * 64, 128, 128, 64), p,
                                  sk_tiles, group_m=8)
    for segs in sched.ctas:
        sk_iters = sum(s.local_iter_end - s.local_iter for s in segs if s.tile_idx < sk_tiles)
        assert ipt <= sk_iters < 2 * ipt
        for s in segs:
            if s.role == S.ROLE_OWNER:
                assert len(s.peers) == 1
    assert sorted(covered(sched.ctas)) == [(tt, i) for tt in range(t) for i in range(ipt)]
    # data-parallel tiles come after the Stream-K tiles in every CTA
    for segs in sched.ctas:
        seen_dp = False
        for s in segs:
            if s.tile_idx >= sk_tiles:
                seen_dp = True
            else:
                assert not seen_dp


def test_tile_coords_raster_is_a_bijection():
    for tm_, tn_, gm in [(5, 7, 2), (64, 32, 16), (3, 3, 8), (1, 9, 1), (10, 1, 4)]:
        seen = {S.tile_coords(i, tm_, tn_, gm) for i in range(tm_ * tn_)}
        assert seen == {(a, b) for a in range(tm_) for b in range(tn_)}
    # group_m >= tiles_m is the plain m-fastest order
    assert [S.tile_coords(i, 3, 2, 3) for i in range(6)] == \
        [(0, 0), (1, 0), (2, 0), (0, 1), (1, 1), (2, 1)]
    # bands of two tile rows: (0,0),(1,0),(0,1),(1,1),... then the last row
    assert [S.tile_coords(i, 3, 2, 2) for i in range(6)] == \
        [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (2, 1)]


def test_cta_of_iter_agrees_with_ranges():
    for total, g in [(576, 148), (14336, 108), (10, 10), (11, 3)]:
        for i in range(total):
            x = S.cta_of_iter(i, total, g)
            b, e = S.cta_iter_range(x, total, g)
            assert b <= i < e


# ---------------------------------------------------------------------------
# cluster_trace: the CTA-pair trace, pinned by traces worked out by hand.
#
# A schedule unit x of a pair launch is CTAs 2x (rank 0) and 2x + 1 (rank 1).
# Both run unit x's segments (same tile, k-range and role); rank r computes
# 128-row block tm * 2 + r of the unit's 256-row tile and takes its partials
# from, and signals them to, the peers' CTAs of the same rank, 2y + r.
# Records: (cta, tile, tm, tn, kb0, kb1, role, peer_first, peer_last).
# ---------------------------------------------------------------------------
W, P, O = S.ROLE_WHOLE, S.ROLE_PARTIAL, S.ROLE_OWNER


def test_cluster_trace_hand_worked_split_schedule():
    # 512 x 256 x 640 in 256 x 128 pair tiles, BLK_K = 64: tiles_m = tiles_n = 2,
    # t = 4, 10 iterations per tile, 40 in all.  Algorithm 5 within one over
    # g = 3 units: q = 13, r = 1, so unit 0 takes [0, 14), unit 1 [14, 27),
    # unit 2 [27, 40).  Raster with one band (group_m = 2): tile 0 -> (0, 0),
    # tile 1 -> (1, 0), tile 2 -> (0, 1), tile 3 -> (1, 1).
    #   unit 0: tile 0 [0, 10) whole; tile 1 [0, 4) owner, peers 1..1
    #   unit 1: tile 1 [4, 10) partial; tile 2 [0, 7) owner, peers 2..2
    #   unit 2: tile 2 [7, 10) partial; tile 3 [0, 10) whole
    prob = S.Problem(512, 256, 640, 256, 128, 64)
    sched = S.persistent_schedule(prob, 3, prob.tiles, group_m=2)
    want = [
        (0, 0, 0, 0, 0, 10, W, -1, -1),
        (0, 1, 2, 0, 0, 4, O, 2, 2),
        (1, 0, 1, 0, 0, 10, W, -1, -1),
        (1, 1, 3, 0, 0, 4, O, 3, 3),
        (2, 1, 2, 0, 4, 10, P, -1, -1),
        (2, 2, 0, 1, 0, 7, O, 4, 4),
        (3, 1, 3, 0, 4, 10, P, -1, -1),
        (3, 2, 1, 1, 0, 7, O, 5, 5),
        (4, 2, 0, 1, 7, 10, P, -1, -1),
        (4, 3, 2, 1, 0, 10, W, -1, -1),
        (5, 2, 1, 1, 7, 10, P, -1, -1),
        (5, 3, 3, 1, 0, 10, W, -1, -1),
    ]
    assert S.cluster_trace(sched, 2) == want


def test_cluster_trace_hand_worked_multi_peer_tile():
    # One 256 x 128 pair tile, k = 640 (10 iterations) over g = 3 units:
    # q = 3, r = 1 -> unit 0 [0, 4) owns the tile with peers 1..2, unit 1
    # [4, 7) and unit 2 [7, 10) spill partials.  Rank r's peers are CTAs
    # 2 + r .. 4 + r.
    prob = S.Problem(256, 128, 640, 256, 128, 64)
    sched = S.persistent_schedule(prob, 3, 1, group_m=1)
    want = [
        (0, 0, 0, 0, 0, 4, O, 2, 4),
        (1, 0, 1, 0, 0, 4, O, 3, 5),
        (2, 0, 0, 0, 4, 7, P, -1, -1),
        (3, 0, 1, 0, 4, 7, P, -1, -1),
        (4, 0, 0, 0, 7, 10, P, -1, -1),
        (5, 0, 1, 0, 7, 10, P, -1, -1),
    ]
    assert S.cluster_trace(sched, 2) == want


def test_cluster_trace_hand_worked_hybrid_with_dp_tiles():
    # 768 x 256 x 384 in pair tiles: tiles_m = 3, tiles_n = 2, t = 6, six
    # iterations per tile; g = 4 units, Stream-K over the first 2 tiles (12
    # iterations, q = 3, r = 0), then data-parallel tiles 2 + x + 4j.  Raster
    # bands of 2 tile rows: tiles 0..3 -> (0,0) (1,0) (0,1) (1,1), then the
    # last row: tile 4 -> (2, 0), tile 5 -> (2, 1).
    #   unit 0: tile 0 [0, 3) owner, peers 1..1; dp tile 2
    #   unit 1: tile 0 [3, 6) partial;           dp tile 3
    #   unit 2: tile 1 [0, 3) owner, peers 3..3; dp tile 4
    #   unit 3: tile 1 [3, 6) partial;           dp tile 5
    prob = S.Problem(768, 256, 384, 256, 128, 64)
    sched = S.persistent_schedule(prob, 4, 2, group_m=2)
    want = [
        (0, 0, 0, 0, 0, 3, O, 2, 2),
        (0, 2, 0, 1, 0, 6, W, -1, -1),
        (1, 0, 1, 0, 0, 3, O, 3, 3),
        (1, 2, 1, 1, 0, 6, W, -1, -1),
        (2, 0, 0, 0, 3, 6, P, -1, -1),
        (2, 3, 2, 1, 0, 6, W, -1, -1),
        (3, 0, 1, 0, 3, 6, P, -1, -1),
        (3, 3, 3, 1, 0, 6, W, -1, -1),
        (4, 1, 2, 0, 0, 3, O, 6, 6),
        (4, 4, 4, 0, 0, 6, W, -1, -1),
        (5, 1, 3, 0, 0, 3, O, 7, 7),
        (5, 4, 5, 0, 0, 6, W, -1, -1),
        (6, 1, 2, 0, 3, 6, P, -1, -1),
        (6, 5, 4, 1, 0, 6, W, -1, -1),
        (7, 1, 3, 0, 3, 6, P, -1, -1),
        (7, 5, 5, 1, 0, 6, W, -1, -1),
    ]
    assert S.cluster_trace(sched, 2) == want
    # cluster_m = 1 is the plain trace of the schedule
    assert S.cluster_trace(sched, 1) == sched.trace()
