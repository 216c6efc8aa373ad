"""Oracle schedule model: the paper's work decompositions, as plain Python.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and
bench.py's cpu_baseline / reference legs may import this module.  It shares no
code with the CUDA path or its host planner; the tests compare the two.

Everything here is integer bookkeeping taken step by step from the paper, in
its notation:

* ``data_parallel``   -- Algorithm 2 (one CTA per output tile).
* ``fixed_split``     -- Algorithm 4 (s CTAs per tile, CTA y = 0 accumulates).
* ``stream_k``        -- Algorithm 5 (an even share of the aggregate MAC-loop
  iterations per CTA, mapped contiguously onto the m -> n -> k linearisation).
* ``hybrid_regions``  -- Section 5.2, "DP + one-tile SK" and "two-tile SK + DP".
* ``best_grid_size``  -- the analytical model of Appendix A.1.
* ``dp_utilization`` / ``stream_k_utilization`` -- the quantization-efficiency
  arithmetic of Section 1 and Section 4.

Readings of passages that are silent, garbled or inconsistent (each one is
listed with its reason in the design notes of the repository):

1. Split rule.  Algorithm 5 sizes CTA ranges as ceil(total_iters / g), but
   Section 1 promises "an even share (within one)" and Fig. 7a prints
   "132/133 iterations per CTA" for 14,336 iterations on 108 CTAs, which only
   the within-one split produces.  CTA x therefore gets
   [x*q + min(x, r), (x+1)*q + min(x+1, r)) with q, r = divmod(T, g).
2. Tile linearisation.  Algorithm 3 divides the tile index by ceil(m/BLK_M)
   for mm and takes the remainder for nn, which swaps the axes of the
   m -> n -> k order named in Section 4.  Here tm = tile % tiles_m and
   tn = tile // tiles_m (m fastest), optionally in bands of ``group_m`` tile
   rows (``tile_coords``); results do not depend on the raster, only the trace.
3. Peer range.  The "cta_end" line of Algorithm 5 is garbled.  The CTAs that
   contribute to the tile owned by CTA x are every y > x whose range meets
   [tile_iter, tile_iter_end), i.e. y in [x+1, cta_of_iter(tile_iter_end-1)].
4. Last CTA.  Algorithm 5 does not clamp iter_end; the within-one split never
   runs past total_iters.  Basic Stream-K needs g <= total_iters.  Inside the
   "DP + one-tile SK" hybrid (Section 5.2) the Stream-K region is balanced over
   every CTA of the grid while each gets "less than one tile's worth", so when
   the partial wave holds fewer iterations than there are CTAs the last CTAs'
   shares are empty (q = 0); they then only run data-parallel tiles.
5. Hybrid edge cases.  With w = floor(t/p) full waves: t mod p == 0 is a
   perfect quantization (pure data-parallel); w == 0 leaves no wave to give up,
   so both hybrids reduce to basic Stream-K over all t tiles; the Stream-K
   region is the first ``sk_tiles`` tile indices, processed before the
   data-parallel tiles, which follow round-robin over the grid.
6. Grid-size model.  ItersPerCta uses the ceiling as printed in Appendix A.1
   even though the schedule itself splits within one; ties go to the smallest g.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

# Roles of a tile segment in a CTA's schedule (the trace format shared with
# the device trace: the format only, no code).
ROLE_WHOLE = 0      # tile_started and tile_ended: StoreTile directly
ROLE_PARTIAL = 1    # not tile_started: StorePartials(partials[x]); Signal(flags[x])
ROLE_OWNER = 2      # tile_started, not tile_ended: Wait + accumulate peers, StoreTile


def ceil_div(a: int, b: int) -> int:
    return -(-a // b)


@dataclass(frozen=True)
class Problem:
    """GEMM shape m x n x k blocked by BLK_M x BLK_N x BLK_K (Section 3)."""
    m: int
    n: int
    k: int
    blk_m: int
    blk_n: int
    blk_k: int

    @property
    def tiles_m(self) -> int:
        return ceil_div(self.m, self.blk_m)

    @property
    def tiles_n(self) -> int:
        return ceil_div(self.n, self.blk_n)

    @property
    def tiles(self) -> int:
        """t, the number of output tiles."""
        return self.tiles_m * self.tiles_n

    @property
    def iters_per_tile(self) -> int:
        """iters_per_tile = ceil(k / BLK_K) (Algorithms 2, 4, 5)."""
        return ceil_div(self.k, self.blk_k)

    @property
    def total_iters(self) -> int:
        """total_iters = tiles * iters_per_tile (Algorithm 5)."""
        return self.tiles * self.iters_per_tile


@dataclass(frozen=True)
class Segment:
    """One MacLoop(tile_idx, local_iter, local_iter_end) call of a CTA and what
    the CTA does with the accumulators afterwards."""
    tile_idx: int
    local_iter: int
    local_iter_end: int
    role: int
    peers: Tuple[int, ...] = ()


# ---------------------------------------------------------------------------
# Algorithm 2: data-parallel.
# ---------------------------------------------------------------------------
def data_parallel(prob: Problem) -> List[List[Segment]]:
    """One CTA per output tile; CTA x runs MacLoop(x, 0, iters_per_tile) and
    stores the tile."""
    ipt = prob.iters_per_tile
    return [[Segment(x, 0, ipt, ROLE_WHOLE)] for x in range(prob.tiles)]


# ---------------------------------------------------------------------------
# Algorithm 4: fixed-split with splitting factor s.
# ---------------------------------------------------------------------------
def fixed_split(prob: Problem, s: int) -> List[List[List[Segment]]]:
    """CTA (x, y) for tile x and split y.  Returns result[x][y] = [Segment].

    iters_per_split = ceil(iters_per_tile / s); split y covers
    [y * iters_per_split, min(iters_per_tile, (y+1) * iters_per_split)).
    Splits y != 0 store partials and signal; split 0 waits for splits
    1 .. s-1 in order, accumulates them and stores the tile.
    """
    if s < 1:
        raise ValueError("splitting factor must be >= 1")
    ipt = prob.iters_per_tile
    ips = ceil_div(ipt, s)
    out = []
    for x in range(prob.tiles):
        row = []
        for y in range(s):
            it = y * ips
            it_end = min(ipt, it + ips)
            it = min(it, it_end)
            if y != 0:
                row.append([Segment(x, it, it_end, ROLE_PARTIAL)])
            else:
                role = ROLE_OWNER if s > 1 else ROLE_WHOLE
                row.append([Segment(x, it, it_end, role, tuple(range(1, s)))])
        out.append(row)
    return out


# ---------------------------------------------------------------------------
# Algorithm 5: basic Stream-K with grid size g.
# ---------------------------------------------------------------------------
def cta_iter_range(x: int, total_iters: int, g: int) -> Tuple[int, int]:
    """Within-one even share of total_iters for CTA x of g (reading 1)."""
    q, r = divmod(total_iters, g)
    begin = x * q + min(x, r)
    end = begin + q + (1 if x < r else 0)
    return begin, end


def cta_of_iter(i: int, total_iters: int, g: int) -> int:
    """The CTA whose range contains global MAC-loop iteration i (by search over
    the ranges, not by inverting the formula)."""
    lo, hi = 0, g - 1
    while lo < hi:
        mid = (lo + hi) // 2
        _, end = cta_iter_range(mid, total_iters, g)
        if i < end:
            hi = mid
        else:
            lo = mid + 1
    b, e = cta_iter_range(lo, total_iters, g)
    assert b <= i < e
    return lo


def stream_k(num_tiles: int, iters_per_tile: int, g: int) -> List[List[Segment]]:
    """Algorithm 5 over tiles 0 .. num_tiles-1.  Returns the segment list of
    each of the g CTAs, in processing order."""
    total_iters = num_tiles * iters_per_tile
    if g < 1 or total_iters < 1:
        raise ValueError("need g >= 1 and at least one iteration")
    ctas = []
    for x in range(g):
        it, it_end = cta_iter_range(x, total_iters, g)
        segs = []
        while it < it_end:
            tile_idx = it // iters_per_tile
            tile_iter = tile_idx * iters_per_tile
            tile_iter_end = tile_iter + iters_per_tile
            local_iter = it - tile_iter
            local_iter_end = min(it_end, tile_iter_end) - tile_iter
            tile_started = it == tile_iter
            tile_ended = it_end >= tile_iter_end
            if not tile_started:
                segs.append(Segment(tile_idx, local_iter, local_iter_end, ROLE_PARTIAL))
            elif not tile_ended:
                last = cta_of_iter(tile_iter_end - 1, total_iters, g)
                segs.append(Segment(tile_idx, local_iter, local_iter_end, ROLE_OWNER,
                                    tuple(range(x + 1, last + 1))))
            else:
                segs.append(Segment(tile_idx, local_iter, local_iter_end, ROLE_WHOLE))
            it = tile_iter_end
        ctas.append(segs)
    return ctas


# ---------------------------------------------------------------------------
# Section 5.2: data-parallel hybridization.
# ---------------------------------------------------------------------------
HYBRID_ONE_TILE = "dp_one_tile_sk"
HYBRID_TWO_TILE = "two_tile_sk_dp"


def hybrid_regions(t: int, p: int, variant: str) -> Tuple[int, int]:
    """(sk_tiles, dp_tiles) for t output tiles on p SMs.

    w = floor(t / p) full waves.  "DP + one-tile SK" balances iterations only
    over the t mod p tiles of the final partial wave.  "Two-tile SK + DP" runs
    one fewer full wave, so Stream-K covers (t mod p) + p tiles.  Edge cases
    follow reading 5.
    """
    w, rem = divmod(t, p)
    if rem == 0:
        return 0, t
    if w == 0:
        return t, 0
    if variant == HYBRID_ONE_TILE:
        return rem, w * p
    if variant == HYBRID_TWO_TILE:
        return rem + p, (w - 1) * p
    raise ValueError(variant)


def tile_coords(tile_idx: int, tiles_m: int, tiles_n: int, group_m: int) -> Tuple[int, int]:
    """Output-tile raster (reading 2): m fastest, in bands of group_m tile rows.
    group_m >= tiles_m gives the plain m -> n order."""
    band_tiles = group_m * tiles_n
    band = tile_idx // band_tiles
    first_m = band * group_m
    rows = min(group_m, tiles_m - first_m)
    local = tile_idx - band * band_tiles
    return first_m + local % rows, local // rows


@dataclass
class Schedule:
    """A complete persistent-grid schedule: g CTAs, a Stream-K region over the
    first sk_tiles tiles, then data-parallel tiles round-robin over the grid."""
    prob: Problem
    g: int
    sk_tiles: int
    group_m: int
    ctas: List[List[Segment]] = field(default_factory=list)

    def trace(self) -> List[Tuple[int, ...]]:
        """Records (cta, tile_idx, tm, tn, local_iter, local_iter_end, role,
        peer_first, peer_last), CTA by CTA in processing order; peer_first =
        peer_last = -1 when the segment has no peers."""
        out = []
        for x, segs in enumerate(self.ctas):
            for s in segs:
                tm, tn = tile_coords(s.tile_idx, self.prob.tiles_m, self.prob.tiles_n,
                                     self.group_m)
                pf = s.peers[0] if s.peers else -1
                pl = s.peers[-1] if s.peers else -1
                out.append((x, s.tile_idx, tm, tn, s.local_iter, s.local_iter_end, s.role,
                            pf, pl))
        return out


def cluster_trace(sched: Schedule, cluster_m: int) -> List[Tuple[int, ...]]:
    """The trace of a schedule whose unit of work is a cluster of cluster_m
    CTAs: unit x's segments are executed by CTAs x*cluster_m + r, each on its
    own 128-row block (tile row tm*cluster_m + r) of the unit's tile, and the
    peers of CTA x*cluster_m + r are the CTAs with the same r.  (The paper's
    schedules are the cluster_m = 1 case.)"""
    if cluster_m == 1:
        return sched.trace()
    by_unit = {}
    for rec in sched.trace():
        by_unit.setdefault(rec[0], []).append(rec)
    out = []
    for x in range(sched.g):
        for r in range(cluster_m):
            for (_, tile, tm, tn, k0, k1, role, pf, pl) in by_unit.get(x, []):
                out.append((x * cluster_m + r, tile, tm * cluster_m + r, tn, k0, k1, role,
                            pf * cluster_m + r if pf >= 0 else -1,
                            pl * cluster_m + r if pl >= 0 else -1))
    return out


def persistent_schedule(prob: Problem, g: int, sk_tiles: int, group_m: int) -> Schedule:
    """Stream-K (Algorithm 5) over tiles [0, sk_tiles) with g CTAs, followed by
    the data-parallel tiles [sk_tiles, t) with tile sk_tiles + x + j*g going to
    CTA x (Algorithm 2 run as full waves of a persistent grid)."""
    t, ipt = prob.tiles, prob.iters_per_tile
    if not (0 <= sk_tiles <= t):
        raise ValueError("sk_tiles out of range")
    ctas: List[List[Segment]] = [[] for _ in range(g)]
    if sk_tiles > 0:
        for x, segs in enumerate(stream_k(sk_tiles, ipt, g)):
            ctas[x].extend(segs)
    for x in range(g):
        tile = sk_tiles + x
        while tile < t:
            ctas[x].append(Segment(tile, 0, ipt, ROLE_WHOLE))
            tile += g
    return Schedule(prob, g, sk_tiles, group_m, ctas)


# ---------------------------------------------------------------------------
# Appendix A.1: analytical grid-size model.
# ---------------------------------------------------------------------------
def iters_per_cta_model(prob: Problem, g: int) -> int:
    """ItersPerCta(g) = ceil(ceil(m/BM) * ceil(n/BN) * ceil(k/BK) / g)."""
    return ceil_div(prob.tiles_m * prob.tiles_n * prob.iters_per_tile, g)


def fixup_peers_model(prob: Problem, g: int) -> int:
    """FixupPeers(g) = ceil(ceil(k/BK) / ItersPerCta(g))."""
    return ceil_div(prob.iters_per_tile, iters_per_cta_model(prob, g))


def time_cta_model(prob: Problem, g: int, a: float, b: float, c: float, d: float) -> float:
    """time_CTA(g) = a + b*[FixupPeers(g) > 1] + c*ItersPerCta(g)
    + d*(FixupPeers(g) - 1)."""
    peers = fixup_peers_model(prob, g)
    return a + b * (1 if peers > 1 else 0) + c * iters_per_cta_model(prob, g) + d * (peers - 1)


def best_grid_size(prob: Problem, p: int, a: float, b: float, c: float, d: float) -> int:
    """The g in [1, p] minimising time_CTA(g); ties go to the smallest g."""
    best_g, best_t = 1, None
    for g in range(1, p + 1):
        tg = time_cta_model(prob, g, a, b, c, d)
        if best_t is None or tg < best_t:
            best_g, best_t = g, tg
    return best_g


# ---------------------------------------------------------------------------
# Section 1 / Section 4: quantization efficiency.
# ---------------------------------------------------------------------------
def dp_utilization(num_ctas: int, p: int) -> float:
    """Utilization ceiling of equal-sized CTA work volumes dispatched in waves
    over p SMs: num_ctas / (ceil(num_ctas / p) * p)."""
    return num_ctas / (ceil_div(num_ctas, p) * p)


def stream_k_utilization(total_iters: int, g: int, p: Optional[int] = None) -> float:
    """Fraction of p SMs' time spent on MAC iterations when g CTAs (one wave,
    g <= p) split total_iters within one: total / (p * max per-CTA share)."""
    p = g if p is None else p
    per_cta = max(cta_iter_range(x, total_iters, g)[1] - cta_iter_range(x, total_iters, g)[0]
                  for x in range(g))
    return total_iters / (p * per_cta)


# ---------------------------------------------------------------------------
# Stream-K across a group of problems (the Conclusion, Section 7, names other
# GEMM-like workloads as future work): the problems' MAC-loop iteration spaces are laid
# end to end, problem after problem and, inside a problem, tile after tile,
# and Algorithm 5 splits that single space evenly over g CTAs.  Tiles of
# different problems may have different iteration counts.
# ---------------------------------------------------------------------------
@dataclass
class GroupSegment:
    """MacLoop over local iterations [local_iter, local_iter_end) of tile
    tile_idx of problem `problem`, with the CTA's role for that tile."""
    problem: int
    tile_idx: int
    local_iter: int
    local_iter_end: int
    role: int
    peers: Tuple[int, ...] = ()


def group_offsets(probs: List[Problem]) -> Tuple[List[int], List[int]]:
    """Prefix sums: first global tile and first global iteration of each
    problem, each list one longer than probs."""
    tile_off, iter_off = [0], [0]
    for p in probs:
        tile_off.append(tile_off[-1] + p.tiles)
        iter_off.append(iter_off[-1] + p.tiles * p.iters_per_tile)
    return tile_off, iter_off


def group_tile(probs: List[Problem], tile_off: List[int], gtile: int) -> Tuple[int, int]:
    """(problem, local tile) of global tile index gtile."""
    for pi in range(len(probs)):
        if tile_off[pi] <= gtile < tile_off[pi + 1]:
            return pi, gtile - tile_off[pi]
    raise ValueError("tile out of range")


def grouped_schedule(probs: List[Problem], g: int, sk_tiles: int) -> List[List[GroupSegment]]:
    """Stream-K (Algorithm 5) over the first sk_tiles global tiles with g CTAs,
    then the remaining global tiles data-parallel, tile sk_tiles + x + j*g to
    CTA x.  Returns each CTA's segments in processing order."""
    tile_off, iter_off = group_offsets(probs)
    t = tile_off[-1]
    if not (0 <= sk_tiles <= t) or g < 1:
        raise ValueError("bad grouped schedule")
    # global iteration of the start of global tile j (tiles laid end to end)
    def tile_iter(j: int) -> int:
        pi, lt = (len(probs), 0) if j == t else group_tile(probs, tile_off, j)
        return iter_off[pi] + lt * (probs[pi].iters_per_tile if pi < len(probs) else 0)
    sk_iters = tile_iter(sk_tiles)
    ctas: List[List[GroupSegment]] = [[] for _ in range(g)]
    if sk_iters > 0:
        for x in range(g):
            it, it_end = cta_iter_range(x, sk_iters, g)
            while it < it_end:
                # the tile holding iteration it
                pi = max(q for q in range(len(probs)) if iter_off[q] <= it)
                ipt = probs[pi].iters_per_tile
                lt = (it - iter_off[pi]) // ipt
                start = iter_off[pi] + lt * ipt
                end = start + ipt
                seg = (pi, lt, it - start, min(it_end, end) - start)
                if it != start:
                    ctas[x].append(GroupSegment(*seg, ROLE_PARTIAL))
                elif it_end < end:
                    last = cta_of_iter(end - 1, sk_iters, g)
                    ctas[x].append(GroupSegment(*seg, ROLE_OWNER, tuple(range(x + 1, last + 1))))
                else:
                    ctas[x].append(GroupSegment(*seg, ROLE_WHOLE))
                it = end
    for x in range(g):
        j = sk_tiles + x
        while j < t:
            pi, lt = group_tile(probs, tile_off, j)
            ctas[x].append(GroupSegment(pi, lt, 0, probs[pi].iters_per_tile, ROLE_WHOLE))
            j += g
    return ctas


def grouped_trace(probs: List[Problem], ctas: List[List[GroupSegment]],
                  group_m: List[int]) -> List[Tuple[int, ...]]:
    """Records (cta, problem, tile_idx, tm, tn, local_iter, local_iter_end,
    role, peer_first, peer_last), CTA by CTA in processing order, with each
    problem's tile raster (reading 2) of band height group_m[problem]."""
    out = []
    for x, segs in enumerate(ctas):
        for s in segs:
            pr = probs[s.problem]
            tm, tn = tile_coords(s.tile_idx, pr.tiles_m, pr.tiles_n, group_m[s.problem])
            pf = s.peers[0] if s.peers else -1
            pl = s.peers[-1] if s.peers else -1
            out.append((x, s.problem, s.tile_idx, tm, tn, s.local_iter, s.local_iter_end, s.role,
                        pf, pl))
    return out


def grouped_cluster_trace(trace: List[Tuple[int, ...]], cluster_m: int) -> List[Tuple[int, ...]]:
    """The trace of a grouped schedule whose unit of work is a cluster of
    cluster_m CTAs, from its per-unit records (as grouped_trace returns them,
    with each problem's tiles cluster_m * 128 rows high): unit x's segments are
    executed by CTAs x*cluster_m + r, each on its own 128-row block (tile row
    tm*cluster_m + r), and the peers of CTA x*cluster_m + r are the CTAs with
    the same r.  Records (cta, problem, tile, tm, tn, kb0, kb1, role,
    peer_first, peer_last), CTA by CTA."""
    if cluster_m == 1:
        return list(trace)
    by_unit = {}
    for rec in trace:
        by_unit.setdefault(rec[0], []).append(rec)
    out = []
    for x in sorted(by_unit):
        for r in range(cluster_m):
            for (_, prob, tile, tm, tn, k0, k1, role, pf, pl) in by_unit[x]:
                out.append((x * cluster_m + r, prob, tile, tm * cluster_m + r, tn, k0, k1, role,
                            pf * cluster_m + r if pf >= 0 else -1,
                            pl * cluster_m + r if pl >= 0 else -1))
    return out

