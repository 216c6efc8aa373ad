// Host planner: tile shape, decomposition (Algorithms 2 and 5, the hybrids of
// Section 5.2) and grid size (Appendix A.1).  Pure integer/host arithmetic, no
// CUDA calls, so it is testable without a GPU through sk_plan_describe and
// sk_grid_model.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "../../include/streamk.h"
#include "planner.h"

namespace sk {

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Appendix A.1 time_CTA(g) with ItersPerCta(g) and FixupPeers(g) as printed.
static double model_time(int64_t tiles, int64_t ipt, int64_t g, const double* c) {
  const int64_t iters_per_cta = cdiv(tiles * ipt, g);
  const int64_t peers = cdiv(ipt, iters_per_cta);
  return c[0] + c[1] * (peers > 1 ? 1.0 : 0.0) + c[2] * static_cast<double>(iters_per_cta) +
         c[3] * static_cast<double>(peers - 1);
}

int grid_model(int64_t tiles, int64_t ipt, int p, const double coef[4]) {
  int best = 1;
  double best_t = 0.0;
  for (int g = 1; g <= p; ++g) {
    const double t = model_time(tiles, ipt, g, coef);
    if (g == 1 || t < best_t) {
      best = g;
      best_t = t;
    }
  }
  return best;
}

// Model constants for this kernel family on GB300, in microseconds, per tile
// configuration (BLK_N, CTAs per cluster along M).  The first four are the
// terms of Appendix A.1: a = fixed per-launch cost, b = a schedule with split
// tiles (spill, signal, wait), c = one MAC-loop iteration of a unit
// (BLK_M x BLK_N x BLK_K), d = reading and adding one more peer's partials.
// The paper's model folds the epilogue into c; two more terms make it
// explicit: e = per tile segment (one accumulator handed to the epilogue),
// and f = the shortest period of consecutive whole tiles of a unit: the next
// tile's MAC loop overlaps this tile's epilogue, so a tile takes
// max(c * iterations, f), and f (the epilogue's own time) paces tiles of few
// iterations.  Fitted by least squares on the log ratio of model to
// measurement (python -m paper_2301_03598_gb300.calibrate) to the times of the
// 2,000-shape log-uniform sweep planned with each configuration and each of
// data-parallel, two-tile hybrid and basic Stream-K forced (15 plans per
// shape), measured on a GB300.
void model_coefficients(int tile_n, int cluster_m, double out[kModelTerms]) {
  static const double k64x1[kModelTerms] = {3.452, 2.219, 0.4159, 0.419, 0.173, 0.996};
  static const double k128x1[kModelTerms] = {3.742, 3.728, 0.5640, 0.569, 0.141, 1.370};
  static const double k256x1[kModelTerms] = {4.398, 8.278, 0.3974, 0.711, 0.137, 1.120};
  static const double k128x2[kModelTerms] = {4.271, 4.468, 0.4521, 0.494, 0.314, 1.681};
  static const double k256x2[kModelTerms] = {4.756, 9.852, 0.3034, 0.461, 0.435, 2.363};
  const double* c = cluster_m == 2 ? (tile_n == 256 ? k256x2 : k128x2)
                                   : (tile_n == 256 ? k256x1 : tile_n == 64 ? k64x1 : k128x1);
  for (int i = 0; i < kModelTerms; ++i) out[i] = c[i];
}

// Modelled time of a resolved schedule: the Appendix A.1 terms evaluated on
// the busiest unit (its Stream-K share plus its data-parallel tiles, each of
// those at least f), plus the per-segment term.
static double predict_us(const sk_schedule_info& s, const double c[kModelTerms]) {
  const int64_t ipt = s.iters_per_tile, g = std::max<int64_t>(1, s.grid);
  if (s.tiles == 0 || ipt == 0) return c[0];
  const int64_t sk_iters = s.sk_tiles * ipt;
  const int64_t q = sk_iters / g;
  const int64_t sk_share = cdiv(sk_iters, g);
  const int64_t dp_per_unit = cdiv(s.dp_tiles, g);
  const double split = s.workspace_bytes > 0 ? 1.0 : 0.0;
  const int64_t peers = s.sk_tiles ? cdiv(ipt, std::max<int64_t>(q, 1)) : 1;
  const int64_t sk_segs = s.sk_tiles ? cdiv(q + 1, ipt) + 1 : 0;
  const double tile_period = std::max(c[2] * static_cast<double>(ipt), c[5]);
  // The tile period holds inside the Stream-K share too: the whole tiles a
  // share can hold (sk_share / ipt of them, e.g. every iteration when
  // ipt = 1) each take max(c * ipt, f), like data-parallel tiles; the split
  // segments at its ends take c per iteration, their epilogues being the
  // spill and the fixup of the b and d terms.
  const int64_t share_whole = sk_share / ipt;
  const double sk_time = c[2] * static_cast<double>(sk_share - share_whole * ipt) +
                         static_cast<double>(share_whole) * tile_period;
  return c[0] + c[1] * split + sk_time +
         static_cast<double>(dp_per_unit) * tile_period +
         c[3] * static_cast<double>(peers - 1) * split +
         c[4] * static_cast<double>(sk_segs + dp_per_unit);
}

static int describe_fixed(int64_t m, int64_t n, int64_t k, int mode, int tile_n, int grid,
                          int raster_group, int cluster_m, int num_sms, sk_schedule_info* out);

// Planning with choices left open: a tile width or cluster size of 0 tries
// each candidate configuration, SK_MODE_AUTO tries data-parallel tiling, the
// two-tile hybrid and, below one full wave of tiles, basic Stream-K at every
// grid size g (at a wave or more the hybrid is the paper's Stream-K form; a
// Stream-K run over many tiles per CTA also loses the raster's L2 reuse), and
// the schedule with the smallest modelled time is kept (ties: the earliest
// candidate, i.e. narrower tiles, single CTAs, data-parallel, smaller g).
// A schedule that splits tiles must beat the best data-parallel one by more
// than the model's error (kSplitMargin, relative): the model's rms error on
// the sweep is 5-8%, and a mistaken split costs more than a mistaken wave.
int describe(int64_t m, int64_t n, int64_t k, int mode, int tile_n, int grid, int raster_group,
             int cluster_m, int num_sms, sk_schedule_info* out, int min_tile_n) {
  if (out == nullptr || num_sms < 1) return SK_ERR_INVALID;
  if (cluster_m != 0 && cluster_m != 1 && cluster_m != 2) return SK_ERR_UNSUPPORTED;
  if (tile_n != 0 && tile_n != 64 && tile_n != 128 && tile_n != 256) return SK_ERR_UNSUPPORTED;
  if (tile_n == 64 && cluster_m == 2) return SK_ERR_UNSUPPORTED;
  if (mode < SK_MODE_AUTO || mode > SK_MODE_HYBRID_ONE_TILE) return SK_ERR_INVALID;
  int tns[3], ntn = 0, cms[2], ncm = 0, modes[3], nmode = 0;
  if (tile_n) {
    tns[ntn++] = tile_n;
  } else {
    if (cluster_m != 2 && min_tile_n <= 64) tns[ntn++] = 64;  // narrow tiles: more tiles for few-tile shapes
    tns[ntn++] = 128;
    if (n > 128) tns[ntn++] = 256;  // a 256-wide tile over <= 128 columns only wastes work
  }
  if (cluster_m) {
    cms[ncm++] = cluster_m;
  } else {
    cms[ncm++] = 1;
    if (m > kTileM && num_sms >= 2) cms[ncm++] = 2;  // a pair needs two 128-row blocks
  }
  if (mode == SK_MODE_AUTO) {
    modes[nmode++] = SK_MODE_DP;
    modes[nmode++] = SK_MODE_HYBRID;
    modes[nmode++] = SK_MODE_SK;
  } else {
    modes[nmode++] = mode;
  }
  int status = SK_ERR_INVALID;
  double best_us = 0.0;
  auto consider = [&](int md, int tn, int cm, int g) {
    sk_schedule_info s{};
    const int st = describe_fixed(m, n, k, md, tn, g, raster_group, cm, num_sms, &s);
    if (st != SK_OK) {
      if (status != SK_OK) status = st;
      return;
    }
    double c[kModelTerms];
    model_coefficients(s.tile_n, s.cluster_m, c);
    double us = predict_us(s, c);
    if (mode == SK_MODE_AUTO && s.workspace_bytes > 0) us *= 1.0 + kSplitMargin;
    if (status != SK_OK || us < best_us) {
      *out = s;
      best_us = us;
      status = SK_OK;
    }
  };
  for (int i = 0; i < ntn; ++i) {
    for (int j = 0; j < ncm; ++j) {
      if (tns[i] == 64 && cms[j] == 2) continue;  // BLK_N = 64 runs on single CTAs
      for (int h = 0; h < nmode; ++h) {
        if (mode == SK_MODE_AUTO && modes[h] == SK_MODE_SK && grid == 0) {
          const int64_t units = num_sms / cms[j];
          const int64_t tiles = cdiv(m, int64_t(kTileM) * cms[j]) * cdiv(n, tns[i]);
          if (tiles >= units) continue;  // a wave or more: the hybrids cover it
          const int64_t iters = tiles * cdiv(k, tile_k_for(tns[i]));
          const int64_t g_max = std::min<int64_t>(units, std::max<int64_t>(iters, 1));
          for (int64_t g = 1; g <= g_max; ++g) consider(SK_MODE_SK, tns[i], cms[j], static_cast<int>(g));
        } else {
          consider(modes[h], tns[i], cms[j], grid);
        }
      }
    }
  }
  return status;
}

static int describe_fixed(int64_t m, int64_t n, int64_t k, int mode, int tile_n, int grid,
                          int raster_group, int cluster_m, int num_sms, sk_schedule_info* out) {
  if (out == nullptr || m < 0 || n < 0 || k < 0 || num_sms < 1 || grid < 0 || raster_group < 0)
    return SK_ERR_INVALID;
  if (cluster_m != 1 && cluster_m != 2) return SK_ERR_UNSUPPORTED;
  if (num_sms > kMaxGrid || grid > num_sms) return SK_ERR_INVALID;
  if (mode < SK_MODE_DP || mode > SK_MODE_HYBRID_ONE_TILE) return SK_ERR_INVALID;
  if (tile_n != 64 && tile_n != 128 && tile_n != 256) return SK_ERR_UNSUPPORTED;
  if (tile_n == 64 && cluster_m != 1) return SK_ERR_UNSUPPORTED;
  // Index arithmetic on the device is 32-bit for tiles and k-blocks.
  if (m > (int64_t(1) << 31) - 1 || n > (int64_t(1) << 31) - 1 || k > (int64_t(1) << 31) - 1)
    return SK_ERR_INVALID;

  sk_schedule_info s{};
  s.tile_k = tile_k_for(tile_n);
  s.tile_n = tile_n;
  s.cluster_m = cluster_m;
  // The schedule's unit is a cluster: cluster_m CTAs computing a
  // (128 * cluster_m) x BLK_N tile; the paper's p is the number of such units.
  s.tile_m = kTileM * s.cluster_m;
  num_sms /= s.cluster_m;
  if (num_sms < 1) return SK_ERR_INVALID;
  if (grid > num_sms) return SK_ERR_INVALID;
  s.tiles_m = static_cast<int32_t>(cdiv(m, s.tile_m));
  s.tiles_n = static_cast<int32_t>(cdiv(n, s.tile_n));
  s.tiles = static_cast<int64_t>(s.tiles_m) * s.tiles_n;
  s.iters_per_tile = static_cast<int32_t>(cdiv(k, s.tile_k));
  if (s.tiles > (int64_t(1) << 31) - 1 || s.tiles * std::max<int64_t>(1, s.iters_per_tile) >
                                               (int64_t(1) << 40))
    return SK_ERR_INVALID;
  // Default raster: bands of 2048 rows (16 tile rows of 128), the best of a
  // measured sweep of band heights on large square shapes.
  s.raster_group = raster_group ? raster_group
                                : std::min<int32_t>(std::max(1, s.tiles_m), 16 / s.cluster_m);

  const int64_t t = s.tiles;
  const int64_t ipt = s.iters_per_tile;
  const int p = num_sms;
  double coef[kModelTerms];
  model_coefficients(s.tile_n, s.cluster_m, coef);

  if (t == 0 || ipt == 0) {
    // Nothing to multiply: no MAC loop, C = beta * C handled by the launcher.
    s.mode = SK_MODE_DP;
    s.grid = static_cast<int32_t>(std::min<int64_t>(std::max<int64_t>(t, 1), p));
    s.sk_tiles = 0;
    s.dp_tiles = t;
  } else {
    const int resolved = mode;
    s.mode = resolved;
    const int64_t w = t / p, rem = t % p;
    switch (resolved) {
      case SK_MODE_DP:
        s.sk_tiles = 0;
        s.grid = static_cast<int32_t>(std::min<int64_t>(t, p));
        break;
      case SK_MODE_SK: {
        s.sk_tiles = t;
        int64_t g = grid ? grid : grid_model(t, ipt, p, coef);
        g = std::min<int64_t>(g, std::min<int64_t>(p, t * ipt));
        s.grid = static_cast<int32_t>(std::max<int64_t>(g, 1));
        break;
      }
      case SK_MODE_HYBRID:
      case SK_MODE_HYBRID_ONE_TILE: {
        if (rem == 0) {  // perfect quantization: full waves only
          s.sk_tiles = 0;
          s.grid = static_cast<int32_t>(std::min<int64_t>(t, p));
        } else if (w == 0) {  // no full wave to trade: basic Stream-K over all tiles
          s.sk_tiles = t;
          int64_t g = grid ? grid : grid_model(t, ipt, p, coef);
          g = std::min<int64_t>(g, std::min<int64_t>(p, t * ipt));
          s.grid = static_cast<int32_t>(std::max<int64_t>(g, 1));
        } else if (resolved == SK_MODE_HYBRID) {
          s.sk_tiles = rem + p;  // one fewer full wave; each CTA gets 1..2 tiles
          s.grid = p;
        } else {
          s.sk_tiles = rem;  // only the partial wave is balanced
          s.grid = p;
        }
        break;
      }
      default:
        return SK_ERR_INVALID;
    }
    s.dp_tiles = t - s.sk_tiles;
  }
  s.sk_iters = s.sk_tiles * ipt;

  // Most segments a CTA can see: its Stream-K share (at most q+1 iterations,
  // so ceil((q+1)/ipt) + 1 segments) plus its round-robin data-parallel tiles.
  int64_t segs = 0;
  if (s.sk_tiles > 0 && ipt > 0) {
    const int64_t q = s.sk_iters / s.grid;
    segs += cdiv(q + 1, ipt) + 1;
  }
  segs += cdiv(s.dp_tiles, s.grid);
  s.max_segments = static_cast<int32_t>(std::max<int64_t>(segs, 1));

  // Workspace: one BLK_M x BLK_N FP32 partial slot and one flag per CTA,
  // only when some tile is split across CTAs.
  bool split = false;
  if (s.sk_tiles > 0 && ipt > 0) {
    const int64_t q = s.sk_iters / s.grid, r = s.sk_iters % s.grid;
    // Every range begins on a tile boundary iff ipt divides each CTA's start.
    for (int64_t x = 1; x < s.grid && !split; ++x) {
      const int64_t begin = x * q + std::min<int64_t>(x, r);
      if (begin % ipt != 0) split = true;
    }
  }
  s.ctas = s.grid * s.cluster_m;
  s.workspace_bytes = split ? workspace_bytes_for(s.ctas, s.tile_n) : 0;
  *out = s;
  return SK_OK;
}

int64_t workspace_bytes_for(int grid, int tile_n) {
  return kFlagBytes + static_cast<int64_t>(grid) * kTileM * tile_n * 4;
}

}  // namespace sk

extern "C" int sk_plan_describe(int64_t m, int64_t n, int64_t k, int mode, int tile_n, int grid,
                                int raster_group, int cluster_m, int num_sms,
                                sk_schedule_info* out) {
  return sk::describe(m, n, k, mode, tile_n, grid, raster_group, cluster_m, num_sms, out);
}

extern "C" int sk_grid_model(int64_t m, int64_t n, int64_t k, int bm, int bn, int bk, int p,
                             const double coef[4], int* g_out) {
  if (m < 1 || n < 1 || k < 1 || bm < 1 || bn < 1 || bk < 1 || p < 1 || coef == nullptr ||
      g_out == nullptr)
    return SK_ERR_INVALID;
  const int64_t tiles = sk::cdiv(m, bm) * sk::cdiv(n, bn);
  const int64_t ipt = sk::cdiv(k, bk);
  *g_out = sk::grid_model(tiles, ipt, p, coef);
  return SK_OK;
}

extern "C" int sk_model_coefficients(int tile_n, int cluster_m, double coef[6]) {
  if (coef == nullptr) return SK_ERR_INVALID;
  if ((tile_n != 64 && tile_n != 128 && tile_n != 256) || (cluster_m != 1 && cluster_m != 2) ||
      (tile_n == 64 && cluster_m == 2))
    return SK_ERR_UNSUPPORTED;
  static_assert(sk::kModelTerms == 6, "sk_model_coefficients returns six terms");
  sk::model_coefficients(tile_n, cluster_m, coef);
  return SK_OK;
}

extern "C" int sk_model_time(const sk_schedule_info* s, const double coef[6], double* us) {
  if (s == nullptr || coef == nullptr || us == nullptr || s->grid < 1 || s->iters_per_tile < 0 ||
      s->tiles < 0 || s->sk_tiles < 0 || s->dp_tiles < 0)
    return SK_ERR_INVALID;
  *us = sk::predict_us(*s, coef);
  return SK_OK;
}

// ------------------------------------------------------------------ grouped
namespace sk {

namespace {

struct GroupShape {
  int64_t tiles_m, tiles_n, tiles, ipt, group_m, kfull64;
};

// The CTA whose share of `total` iterations (within-one split over g) holds i.
int64_t owner_of(int64_t i, int64_t total, int64_t g) {
  const int64_t q = total / g, r = total % g;
  const int64_t big = r * (q + 1);
  return i < big ? i / (q + 1) : r + (i - big) / q;
}

void raster(int64_t tile, const GroupShape& p, int64_t& tm, int64_t& tn) {
  const int64_t band_tiles = p.group_m * p.tiles_n;
  const int64_t band = tile / band_tiles;
  const int64_t first_m = band * p.group_m;
  const int64_t rows = std::min(p.group_m, p.tiles_m - first_m);
  const int64_t local = tile - band * band_tiles;
  tm = first_m + local % rows;
  tn = local / rows;
}

// Lays out the schedule: Stream-K (Algorithm 5) over the first sk_tiles
// global tiles of the concatenated problems, then the remaining tiles
// data-parallel round-robin.  Returns false when a record field overflows.
bool build_group(const std::vector<GroupShape>& ps, int64_t g, int64_t sk_tiles, GroupPlan* out) {
  const size_t P = ps.size();
  std::vector<int64_t> tile_off(P + 1, 0), iter_off(P + 1, 0);
  for (size_t i = 0; i < P; ++i) {
    tile_off[i + 1] = tile_off[i] + ps[i].tiles;
    iter_off[i + 1] = iter_off[i] + ps[i].tiles * ps[i].ipt;
  }
  const int64_t t = tile_off[P];
  // global iteration at which global tile sk_tiles starts
  int64_t sk_iters = 0;
  {
    size_t pi = 0;
    while (pi < P && tile_off[pi + 1] <= sk_tiles) ++pi;
    sk_iters = pi < P ? iter_off[pi] + (sk_tiles - tile_off[pi]) * ps[pi].ipt : iter_off[P];
  }
  out->segs.clear();
  out->start.assign(static_cast<size_t>(g) + 1, 0);
  out->split = false;
  out->sk_tiles = sk_tiles;
  out->sk_iters = sk_iters;
  out->tiles = t;
  int max_segs = 0;
  auto emit = [&](size_t pi, int64_t lt, int64_t kb0, int64_t kb1, int role, int64_t pf,
                  int64_t pl) -> bool {
    const GroupShape& p = ps[pi];
    int64_t tm, tn;
    raster(lt, p, tm, tn);
    if (tm > 32767 || tn > 32767 || kb1 > 32767 || p.kfull64 > 32767 || lt > INT32_MAX)
      return false;
    GroupSeg r{};
    r.problem = static_cast<int32_t>(pi);
    r.tile = static_cast<int32_t>(lt);
    r.tm = static_cast<int16_t>(tm);
    r.tn = static_cast<int16_t>(tn);
    r.kb0 = static_cast<int16_t>(kb0);
    r.kb1 = static_cast<int16_t>(kb1);
    r.role = static_cast<int16_t>(role);
    r.kfull64 = static_cast<int16_t>(p.kfull64);
    r.peer_first = static_cast<int16_t>(pf);
    r.peer_last = static_cast<int16_t>(pl);
    out->segs.push_back(r);
    if (role != kRoleWhole) out->split = true;
    return true;
  };
  for (int64_t x = 0; x < g; ++x) {
    const size_t first = out->segs.size();
    if (sk_iters > 0) {
      const int64_t q = sk_iters / g, r = sk_iters % g;
      int64_t it = x * q + std::min(x, r);
      const int64_t it_end = it + q + (x < r ? 1 : 0);
      size_t pi = 0;
      while (it < it_end) {
        while (iter_off[pi + 1] <= it) ++pi;
        const int64_t ipt = ps[pi].ipt;
        const int64_t lt = (it - iter_off[pi]) / ipt;
        const int64_t start = iter_off[pi] + lt * ipt, end = start + ipt;
        const int64_t kb0 = it - start, kb1 = std::min(it_end, end) - start;
        bool ok;
        if (it != start)
          ok = emit(pi, lt, kb0, kb1, kRolePartial, -1, -1);
        else if (it_end < end)
          ok = emit(pi, lt, kb0, kb1, kRoleOwner, x + 1, owner_of(end - 1, sk_iters, g));
        else
          ok = emit(pi, lt, kb0, kb1, kRoleWhole, -1, -1);
        if (!ok) return false;
        it = end;
      }
    }
    size_t pi = 0;
    for (int64_t j = sk_tiles + x; j < t; j += g) {
      while (tile_off[pi + 1] <= j) ++pi;
      if (!emit(pi, j - tile_off[pi], 0, ps[pi].ipt, kRoleWhole, -1, -1)) return false;
    }
    out->start[static_cast<size_t>(x) + 1] = static_cast<int32_t>(out->segs.size());
    max_segs = std::max(max_segs, static_cast<int>(out->segs.size() - first));
  }
  out->max_segments = std::max(max_segs, 1);
  return true;
}

// The device walk table of a schedule (Stream-K over the first sk_tiles
// global tiles, data-parallel round-robin after them, over g CTAs): one
// entry per problem plus a sentinel with the totals, and per CTA the
// problems holding its first Stream-K iteration and first data-parallel tile.
void build_walk(const std::vector<GroupShape>& ps, int64_t g, int64_t sk_tiles, GroupPlan* out) {
  const size_t P = ps.size();
  out->walk.assign(P + 1, GroupWalk{});
  int64_t t = 0, it = 0;
  for (size_t i = 0; i <= P; ++i) {
    GroupWalk& w = out->walk[i];
    w.tile_off = static_cast<int32_t>(t);
    w.iter_off = static_cast<int32_t>(it);
    if (i == P) break;
    const GroupShape& p = ps[i];
    const int64_t rows_last = p.tiles_m - (cdiv(p.tiles_m, p.group_m) - 1) * p.group_m;
    w.tiles_m = static_cast<int32_t>(p.tiles_m);
    w.tiles_n = static_cast<int32_t>(p.tiles_n);
    w.ipt = static_cast<int32_t>(p.ipt);
    w.group_m = static_cast<int32_t>(p.group_m);
    w.kfull64 = static_cast<int32_t>(p.kfull64);
    w.div_ipt = make_fastdiv(static_cast<uint32_t>(p.ipt));
    w.div_band = make_fastdiv(static_cast<uint32_t>(p.group_m * p.tiles_n));
    w.div_rows = make_fastdiv(static_cast<uint32_t>(p.group_m));
    w.div_rows_last = make_fastdiv(static_cast<uint32_t>(std::max<int64_t>(1, rows_last)));
    t += p.tiles;
    it += p.tiles * p.ipt;
  }
  // global iteration at which global tile sk_tiles starts
  size_t pi = 0;
  while (pi < P && out->walk[pi + 1].tile_off <= sk_tiles) ++pi;
  const int64_t sk_iters =
      pi < P ? out->walk[pi].iter_off + (sk_tiles - out->walk[pi].tile_off) * ps[pi].ipt : it;
  out->gstart.assign(static_cast<size_t>(2 * g), 0);
  const int64_t q = sk_iters / g, r = sk_iters % g;
  size_t a = 0, b = 0;
  for (int64_t x = 0; x < g; ++x) {
    const int64_t first = x * q + std::min(x, r);
    while (a + 1 < P && out->walk[a + 1].iter_off <= first) ++a;
    const int64_t j = sk_tiles + x;
    while (b + 1 < P && out->walk[b + 1].tile_off <= j) ++b;
    out->gstart[static_cast<size_t>(2 * x)] = static_cast<int32_t>(a);
    out->gstart[static_cast<size_t>(2 * x + 1)] = static_cast<int32_t>(b);
  }
  out->tiles = t;
  out->sk_tiles = sk_tiles;
  out->sk_iters = sk_iters;
}

// HBM bandwidth the model assumes for operand traffic, bytes per microsecond
// (the measured copy bandwidth of this GB300, rounded down).
constexpr double kHbmBytesPerUs = 6.5e6;

// Operand bytes a grouped schedule moves from HBM.  Data-parallel waves run p
// neighbouring tiles of a problem's raster at once, which share A row blocks
// and B column blocks in L2: each problem's operands come from HBM about
// once.  A Stream-K region of more tiles than CTAs gives every CTA its own
// contiguous run of tiles, far from its neighbours' and at different k
// offsets, so nothing is shared: every iteration's A and B tiles come from
// HBM.
double group_dram_bytes(const std::vector<GroupShape>& ps, const std::vector<int64_t>& m,
                        const std::vector<int64_t>& n, const std::vector<int64_t>& k,
                        const GroupPlan& gp, int tile_n, int cluster_m) {
  // operand bytes of one unit's MAC-loop iteration
  const double stage =
      static_cast<double>(kTileM * cluster_m + tile_n) * tile_k_for(tile_n) * 2.0;
  double bytes = 0.0;
  int64_t tile0 = 0;
  for (size_t i = 0; i < ps.size(); ++i) {
    const int64_t t0 = tile0, t1 = tile0 + ps[i].tiles;
    tile0 = t1;
    const int64_t sk = std::max<int64_t>(0, std::min(t1, gp.sk_tiles) - t0);
    const double once = 2.0 * static_cast<double>(m[i] * k[i] + n[i] * k[i]);
    const double frac_dp = static_cast<double>(ps[i].tiles - sk) / static_cast<double>(ps[i].tiles);
    if (gp.sk_tiles > gp.grid)
      bytes += static_cast<double>(sk) * static_cast<double>(ps[i].ipt) * stage + once * frac_dp;
    else
      bytes += once;
  }
  return bytes;
}

// Modelled time of a grouped schedule: the busiest CTA's iterations and
// segments under the Appendix A.1 terms plus the per-segment term.
double predict_group(const GroupPlan& gp, const double c[kModelTerms]) {
  double worst = 0.0;
  int64_t peers_max = 1;
  for (size_t x = 0; x + 1 < gp.start.size(); ++x) {
    double t = 0.0;
    for (int32_t i = gp.start[x]; i < gp.start[x + 1]; ++i) {
      const GroupSeg& r = gp.segs[static_cast<size_t>(i)];
      const double mac = c[2] * static_cast<double>(r.kb1 - r.kb0);
      t += (r.role == kRoleWhole ? std::max(mac, c[5]) : mac) + c[4];
      if (r.role == kRoleOwner) peers_max = std::max<int64_t>(peers_max, r.peer_last - r.peer_first + 2);
    }
    worst = std::max(worst, t);
  }
  const double split = gp.split ? 1.0 : 0.0;
  return c[0] + c[1] * split + c[3] * static_cast<double>(peers_max - 1) * split + worst;
}

}  // namespace

void set_group_walk_args(SkArgs& a, const GroupPlan& gp) {
  a.grid = gp.grid;
  a.tiles = static_cast<int32_t>(gp.tiles);
  a.sk_tiles = static_cast<int32_t>(gp.sk_tiles);
  a.sk_q = static_cast<int32_t>(gp.sk_iters / gp.grid);
  a.sk_r = static_cast<int32_t>(gp.sk_iters % gp.grid);
  a.div_q1 = make_fastdiv(static_cast<uint32_t>(a.sk_q + 1));
  a.div_q = make_fastdiv(static_cast<uint32_t>(std::max(1, a.sk_q)));
  a.fast_iters = 1;  // the planner keeps the concatenated space below 2^31
}

int describe_grouped_dp(int count, const int64_t* m, const int64_t* n, const int64_t* k,
                        int tile_n, int num_sms, GroupPlan* out) {
  if (out == nullptr || count < 1 || m == nullptr || n == nullptr || k == nullptr || num_sms < 1 ||
      num_sms > kMaxGrid)
    return SK_ERR_INVALID;
  if (tile_n != 0 && tile_n != 64 && tile_n != 128 && tile_n != 256) return SK_ERR_UNSUPPORTED;
  int64_t max_n = 0;
  for (int i = 0; i < count; ++i) {
    if (m[i] < 1 || n[i] < 1 || k[i] < 1 || m[i] > INT32_MAX || n[i] > INT32_MAX || k[i] > INT32_MAX)
      return SK_ERR_INVALID;
    max_n = std::max(max_n, n[i]);
  }
  const int bn = tile_n ? tile_n : (max_n > 128 ? 256 : 128);
  const int bk = tile_k_for(bn);
  std::vector<GroupShape> ps(static_cast<size_t>(count));
  int64_t t = 0, total_iters = 0;
  for (int j = 0; j < count; ++j) {
    GroupShape& p = ps[static_cast<size_t>(j)];
    p.tiles_m = cdiv(m[j], kTileM);
    p.tiles_n = cdiv(n[j], bn);
    p.tiles = p.tiles_m * p.tiles_n;
    p.ipt = cdiv(k[j], bk);
    p.group_m = std::min<int64_t>(p.tiles_m, 16);
    p.kfull64 = bk == 128 && k[j] / 64 >= 2 ? k[j] / 64 : 0;
    t += p.tiles;
    total_iters += p.tiles * p.ipt;
  }
  if (t > INT32_MAX || total_iters > INT32_MAX) return SK_ERR_INVALID;
  const int64_t g = std::min<int64_t>(num_sms, t);
  out->segs.clear();
  out->start.clear();
  build_walk(ps, g, 0, out);
  out->mode = SK_MODE_DP;
  out->tile_n = bn;
  out->tile_k = bk;
  out->grid = static_cast<int32_t>(g);
  out->split = false;
  out->workspace_bytes = 0;
  out->max_segments = static_cast<int>(cdiv(t, g));
  return SK_OK;
}

int describe_grouped(int count, const int64_t* m, const int64_t* n, const int64_t* k, int mode,
                     int tile_n, int grid, int num_sms, GroupPlan* out, int cluster_m) {
  if (out == nullptr || count < 1 || m == nullptr || n == nullptr || k == nullptr || num_sms < 1 ||
      num_sms > kMaxGrid || grid < 0 || grid > num_sms)
    return SK_ERR_INVALID;
  if (tile_n != 0 && tile_n != 64 && tile_n != 128 && tile_n != 256) return SK_ERR_UNSUPPORTED;
  if (cluster_m != 0 && cluster_m != 1 && cluster_m != 2) return SK_ERR_UNSUPPORTED;
  if (tile_n == 64 && cluster_m == 2) return SK_ERR_UNSUPPORTED;
  if (mode != SK_MODE_AUTO && mode != SK_MODE_DP && mode != SK_MODE_SK && mode != SK_MODE_HYBRID)
    return SK_ERR_UNSUPPORTED;
  int64_t max_n = 0;
  for (int i = 0; i < count; ++i) {
    if (m[i] < 1 || n[i] < 1 || k[i] < 1 || m[i] > INT32_MAX || n[i] > INT32_MAX || k[i] > INT32_MAX)
      return SK_ERR_INVALID;
    max_n = std::max(max_n, n[i]);
  }
  int64_t max_m = 0;
  for (int i = 0; i < count; ++i) max_m = std::max(max_m, m[i]);
  int tns[2], ntn = 0, cms[2], ncm = 0;
  if (tile_n) {
    tns[ntn++] = tile_n;
  } else {
    tns[ntn++] = 128;
    if (max_n > 128) tns[ntn++] = 256;
  }
  if (cluster_m) {
    cms[ncm++] = cluster_m;
  } else {
    cms[ncm++] = 1;
    if (max_m > kTileM && num_sms >= 2) cms[ncm++] = 2;  // a pair needs two 128-row blocks
  }
  int status = SK_ERR_INVALID;
  double best_us = 0.0;
  for (int i = 0; i < ntn; ++i) {
  for (int ci = 0; ci < ncm; ++ci) {
    const int bn = tns[i];
    const int cm = cms[ci];
    if (bn == 64 && cm == 2) continue;  // BLK_N = 64 runs on single CTAs
    const int bk = tile_k_for(bn);
    // The schedule's unit is a cluster of cm CTAs computing a (128 * cm) x bn
    // tile; p counts units.
    std::vector<GroupShape> ps(static_cast<size_t>(count));
    int64_t t = 0, total_iters = 0;
    for (int j = 0; j < count; ++j) {
      GroupShape& p = ps[static_cast<size_t>(j)];
      p.tiles_m = cdiv(m[j], int64_t(kTileM) * cm);
      p.tiles_n = cdiv(n[j], bn);
      p.tiles = p.tiles_m * p.tiles_n;
      p.ipt = cdiv(k[j], bk);
      p.group_m = std::min<int64_t>(p.tiles_m, 16 / cm);
      p.kfull64 = bk == 128 && k[j] / 64 >= 2 ? k[j] / 64 : 0;
      t += p.tiles;
      total_iters += p.tiles * p.ipt;
    }
    if (t > INT32_MAX || total_iters > INT32_MAX) return SK_ERR_INVALID;
    double c[kModelTerms];
    model_coefficients(bn, cm, c);
    const int64_t p = num_sms / cm;
    if (grid > p) continue;
    // candidate (mode, sk_tiles, grid)
    struct Cand { int mode; int64_t sk_tiles, g; };
    std::vector<Cand> cands;
    const int64_t g_all = grid ? grid : std::min<int64_t>(p, total_iters);
    const int64_t g_dp = grid ? grid : std::min<int64_t>(p, t);
    if (mode == SK_MODE_AUTO || mode == SK_MODE_DP) cands.push_back({SK_MODE_DP, 0, g_dp});
    if (mode == SK_MODE_AUTO || mode == SK_MODE_SK) cands.push_back({SK_MODE_SK, t, g_all});
    if (mode == SK_MODE_AUTO || mode == SK_MODE_HYBRID) {
      const int64_t w = t / p, rem = t % p;
      const int64_t skt = rem == 0 ? 0 : (w == 0 ? t : rem + p);
      cands.push_back({SK_MODE_HYBRID, skt, skt == t ? g_all : (grid ? grid : p)});
    }
    const std::vector<int64_t> mv(m, m + count), nv(n, n + count), kv(k, k + count);
    for (const Cand& cd : cands) {
      GroupPlan gp;
      if (!build_group(ps, std::max<int64_t>(cd.g, 1), cd.sk_tiles, &gp)) return SK_ERR_INVALID;
      build_walk(ps, std::max<int64_t>(cd.g, 1), cd.sk_tiles, &gp);
      gp.grid = static_cast<int32_t>(std::max<int64_t>(cd.g, 1));
      const double us =
          std::max(predict_group(gp, c),
                   c[0] + group_dram_bytes(ps, mv, nv, kv, gp, bn, cm) / kHbmBytesPerUs);
      if (status != SK_OK || us < best_us) {
        gp.mode = cd.mode;
        gp.tile_n = bn;
        gp.tile_k = bk;
        gp.cluster_m = cm;
        gp.grid = static_cast<int32_t>(std::max<int64_t>(cd.g, 1));
        gp.workspace_bytes = gp.split ? workspace_bytes_for(gp.grid * cm, bn) : 0;
        *out = std::move(gp);
        best_us = us;
        status = SK_OK;
      }
    }
  }
  }
  return status;
}

}  // namespace sk

// Host-only planning of a grouped launch (no device needed): the summary and
// the segment records of sk_grouped_plan's schedule for num_sms SMs.
extern "C" int sk_grouped_plan_describe(int count, const int64_t* m, const int64_t* n,
                                        const int64_t* k, int mode, int tile_n, int grid,
                                        int num_sms, int cluster_m, int64_t* summary,
                                        int32_t* records, int64_t capacity, int64_t* nrec) {
  sk::GroupPlan gp;
  const int st = sk::describe_grouped(count, m, n, k, mode, tile_n, grid, num_sms, &gp, cluster_m);
  if (st != SK_OK) return st;
  if (summary != nullptr) {
    const int64_t sm[9] = {gp.mode, gp.tile_n, gp.tile_k, gp.grid, gp.tiles, gp.sk_tiles,
                           gp.workspace_bytes, gp.max_segments, gp.cluster_m};
    for (int i = 0; i < 9; ++i) summary[i] = sm[i];
  }
  if (nrec != nullptr) *nrec = static_cast<int64_t>(gp.segs.size());
  if (records == nullptr) return SK_OK;
  if (capacity < static_cast<int64_t>(gp.segs.size()) * 10) return SK_ERR_INVALID;
  int64_t o = 0;
  for (size_t x = 0; x + 1 < gp.start.size(); ++x) {
    for (int32_t i = gp.start[x]; i < gp.start[x + 1]; ++i) {
      const sk::GroupSeg& r = gp.segs[static_cast<size_t>(i)];
      const int32_t f[10] = {static_cast<int32_t>(x), r.problem, r.tile, r.tm, r.tn,
                             r.kb0, r.kb1, r.role, r.peer_first, r.peer_last};
      for (int j = 0; j < 10; ++j) records[o++] = f[j];
    }
  }
  return SK_OK;
}
