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

// Model constants of Appendix A.1 for this kernel family on GB300, in
// microseconds, fitted by relative least squares to measured times of basic
// Stream-K over grid sizes g in [t, p] for 70 shapes drawn like the
// log-uniform shape sweep (t < p), each tile width: a = fixed per-launch
// cost, b = a CTA spilling partial sums, c = one MAC-loop iteration
// (BLK_M x BLK_N x 64), d = reading and adding one peer's partials.
void model_coefficients(int tile_n, double out[4]) {
  if (tile_n == 256) {
    out[0] = 5.45;
    out[1] = 4.10;
    out[2] = 0.295;
    out[3] = 1.719;
  } else {
    out[0] = 5.51;
    out[1] = 1.68;
    out[2] = 0.261;
    out[3] = 0.943;
  }
}

// BLK_N = 256 is the ideal blocking factor for throughput: an M=128 MMA with
// N=128 takes as long as one with N=256.  When the 128-wide tiling fits in one
// wave, the extra parallelism of the narrower tile (and its half-size partial
// sums) measured faster, so it is used there and for outputs of at most 128
// columns.
static int auto_tile_n(int64_t m, int64_t n, int64_t /*k*/, int num_sms) {
  if (n <= 128) return 128;
  const int64_t t128 = cdiv(m, kTileM) * cdiv(n, 128);
  return t128 <= num_sms ? 128 : 256;
}

// CTA pairs along M (clusters of 2 sharing the B tile by multicast) halve
// the L2 -> SM traffic of B; they pay off once the problem fills the GPU with
// 128 x 256 tiles, and need at least two 128-row blocks.
static int auto_cluster_m(int64_t m, int64_t n, int tile_n, int num_sms) {
  const int64_t tm = cdiv(m, kTileM);
  if (tile_n != 256 || tm < 2 || num_sms < 2) return 1;
  return tm * cdiv(n, 256) >= num_sms ? 2 : 1;
}

int describe(int64_t m, int64_t n, int64_t k, int mode, int tile_n, int grid, int raster_group,
             int cluster_m, int num_sms, sk_schedule_info* out) {
  if (out == nullptr || m < 0 || n < 0 || k < 0 || num_sms < 1 || grid < 0 || raster_group < 0)
    return SK_ERR_INVALID;
  if (cluster_m != 0 && cluster_m != 1 && cluster_m != 2) return SK_ERR_UNSUPPORTED;
  if (num_sms > kMaxGrid || grid > num_sms) return SK_ERR_INVALID;
  if (mode < SK_MODE_AUTO || mode > SK_MODE_HYBRID_ONE_TILE) return SK_ERR_INVALID;
  if (tile_n != 0 && tile_n != 128 && tile_n != 256) return SK_ERR_UNSUPPORTED;
  // Index arithmetic on the device is 32-bit for tiles and k-blocks.
  if (m > (int64_t(1) << 31) - 1 || n > (int64_t(1) << 31) - 1 || k > (int64_t(1) << 31) - 1)
    return SK_ERR_INVALID;

  sk_schedule_info s{};
  s.tile_k = kTileK;
  s.tile_n = tile_n ? tile_n : auto_tile_n(m, n, k, num_sms);
  s.cluster_m = cluster_m ? cluster_m : auto_cluster_m(m, n, s.tile_n, num_sms);
  // The schedule's unit is a cluster: cluster_m CTAs computing a
  // (128 * cluster_m) x BLK_N tile; the paper's p is the number of such units.
  s.tile_m = kTileM * s.cluster_m;
  const int num_sms_all = num_sms;
  num_sms /= s.cluster_m;
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
  double coef[4];
  model_coefficients(s.tile_n, coef);

  if (t == 0 || ipt == 0) {
    // Nothing to multiply: no MAC loop, C = beta * C handled by the launcher.
    s.mode = SK_MODE_DP;
    s.grid = static_cast<int32_t>(std::min<int64_t>(std::max<int64_t>(t, 1), p));
    s.sk_tiles = 0;
    s.dp_tiles = t;
  } else {
    int resolved = mode;
    if (mode == SK_MODE_AUTO) {
      if (t % p == 0)
        resolved = SK_MODE_DP;
      else if (t >= p)
        resolved = SK_MODE_HYBRID;
      else
        resolved = SK_MODE_SK;
    }
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
        if (mode == SK_MODE_AUTO && w >= 1 && rem != 0) {
          // The two-tile hybrid pays one spill and one fixup per split tile;
          // with few iterations per tile that can cost more than the partial
          // wave it removes.  Compare both with the model's terms: the spill
          // and fixup overlap the (w - 1) data-parallel tiles that follow the
          // Stream-K region, and whatever those do not cover is exposed.
          const double split_us = std::max(
              0.0, coef[1] + coef[3] - coef[2] * static_cast<double>((w - 1) * ipt));
          const double dp_us = coef[0] + coef[2] * static_cast<double>(ipt * ((t + p - 1) / p));
          const double sk_us =
              coef[0] + split_us + coef[2] * static_cast<double>((t * ipt + p - 1) / p);
          if (dp_us <= sk_us) {
            s.mode = SK_MODE_DP;
            s.sk_tiles = 0;
            s.grid = static_cast<int32_t>(std::min<int64_t>(t, p));
            break;
          }
        }
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
  if (split && cluster_m == 0 && s.cluster_m == 2) {
    // Automatic planning keeps CTA pairs to schedules without split tiles:
    // those launch without the cooperative attribute, which the profiler could
    // not replay together with clusters.  Split schedules use single CTAs.
    return describe(m, n, k, mode, tile_n, grid, raster_group, 1, num_sms_all, out);
  }
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
