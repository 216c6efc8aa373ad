// Host planner interface (see planner.cpp).
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/streamk.h"
#include "sk_args.h"

namespace sk {

constexpr int kTileM = 128;
// BLK_K, the depth of one MAC-loop iteration: two 64-wide k-blocks for
// BLK_N = 64 and 128 (one pipeline stage holds both, see the kernel's Cfg),
// one for 256.
constexpr int tile_k_for(int tile_n) { return tile_n <= 128 ? 128 : 64; }
// Pipeline stages the kernel's 192 KiB shared-memory ring holds for a tile
// configuration (the kernel's Cfg<BN, CM>::kStages): a stage is one MAC-loop
// iteration of A (128 rows) and this CTA's BN / CM rows of B, 128 bytes each
// per 64-deep k-block.
constexpr int max_stages(int tile_n, int cluster_m) {
  return (192 * 1024) / (tile_k_for(tile_n) / 64 * (kTileM + tile_n / cluster_m) * 128);
}
// Workspace layout: kFlagBytes of flags at offset 0 (kFlagsPerCta uint32 per
// CTA, one per 32-row x 128-byte unit of its partial tile, at most kMaxGrid
// CTAs), then one BLK_M x BLK_N FP32 partial slot per CTA.
constexpr int kMaxGrid = 1024;
constexpr int kFlagsPerCta = 32;
constexpr int64_t kFlagBytes = static_cast<int64_t>(kMaxGrid) * kFlagsPerCta * 4;

// tile_n 0 ranks the widths 64, 128 and 256 that are at least min_tile_n
// (E4M3 plans: 128 and 256).
int describe(int64_t m, int64_t n, int64_t k, int mode, int tile_n, int grid, int raster_group,
             int cluster_m, int num_sms, sk_schedule_info* out, int min_tile_n = 64);
int grid_model(int64_t tiles, int64_t ipt, int p, const double coef[4]);
// Terms of the planner's time model per tile configuration: Appendix A.1's
// a, b, c, d, then e (per tile segment) and f (shortest whole-tile period).
constexpr int kModelTerms = 6;
// AUTO keeps a split schedule only if its modelled time, raised by this
// fraction, still beats every data-parallel candidate.
constexpr double kSplitMargin = 0.10;
void model_coefficients(int tile_n, int cluster_m, double out[kModelTerms]);
int64_t workspace_bytes_for(int grid, int tile_n);

// A grouped launch's schedule over the problems' concatenated iteration space
// (single CTAs, one tile width for all problems): per-CTA segment records
// (CTA x owns segs[start[x] .. start[x+1])) for the model and the schedule
// query, and the walk table the device derives the same segments from.
struct GroupPlan {
  // grid counts units of cluster_m CTAs; records and the walk are per unit
  int mode = 0, tile_n = 0, tile_k = 0, grid = 0, max_segments = 1, cluster_m = 1;
  int64_t tiles = 0, sk_tiles = 0, sk_iters = 0, workspace_bytes = 0;
  bool split = false;
  std::vector<GroupSeg> segs;
  std::vector<int32_t> start;
  // what the device walks: count + 1 table entries, 2 * grid start problems
  std::vector<GroupWalk> walk;
  std::vector<int32_t> gstart;
};
// cluster_m 0 tries single CTAs and CTA pairs (units of two CTAs computing
// 256-row tiles); grid counts units.
int describe_grouped(int count, const int64_t* m, const int64_t* n, const int64_t* k, int mode,
                     int tile_n, int grid, int num_sms, GroupPlan* out, int cluster_m = 1);
// The launch-wide walk fields of SkArgs for a grouped schedule: grid, tile
// count, Stream-K region and its within-one split, and their divisors.
void set_group_walk_args(SkArgs& a, const GroupPlan& gp);
// Data-parallel waves over the group (one CTA per tile, at most num_sms CTAs)
// without the segment records: the walk table only, in O(count + grid).
// tile_n 0 picks 256 when some n > 128.
int describe_grouped_dp(int count, const int64_t* m, const int64_t* n, const int64_t* k,
                        int tile_n, int num_sms, GroupPlan* out);

}  // namespace sk
