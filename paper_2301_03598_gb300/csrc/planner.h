// Host planner interface (see planner.cpp).
#pragma once
#include <cstdint>

#include "../../include/streamk.h"

namespace sk {

constexpr int kTileM = 128;
// BLK_K, the depth of one MAC-loop iteration: two 64-wide k-blocks for
// BLK_N = 128 (one pipeline stage each, see the kernel's Cfg), one for 256.
constexpr int tile_k_for(int tile_n) { return tile_n == 128 ? 128 : 64; }
// Workspace layout: kFlagBytes of flags at offset 0 (kFlagsPerCta uint32 per
// CTA, one per 32-row x 128-byte unit of its partial tile, at most kMaxGrid
// CTAs), then one BLK_M x BLK_N FP32 partial slot per CTA.
constexpr int kMaxGrid = 1024;
constexpr int kFlagsPerCta = 32;
constexpr int64_t kFlagBytes = static_cast<int64_t>(kMaxGrid) * kFlagsPerCta * 4;

int describe(int64_t m, int64_t n, int64_t k, int mode, int tile_n, int grid, int raster_group,
             int cluster_m, int num_sms, sk_schedule_info* out);
int grid_model(int64_t tiles, int64_t ipt, int p, const double coef[4]);
void model_coefficients(int tile_n, int cluster_m, double out[5]);
int64_t workspace_bytes_for(int grid, int tile_n);

}  // namespace sk
