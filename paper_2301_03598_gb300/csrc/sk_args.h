// Kernel-argument block of the persistent Stream-K GEMM kernel, filled by the
// host planner and passed by value at launch.
#pragma once
#include <cstdint>

#include <cuda.h>

namespace sk {

constexpr int kBlkM = 128;  // BLK_M: one tcgen05 M=128 MMA covers the tile height
constexpr int kBlkK = 64;   // one k-block: 64 16-bit elements = one 128-byte swizzle row

// Segment roles (the trace format; see include/streamk.h).
constexpr int kRoleWhole = 0;    // tile_started && tile_ended: store the tile
constexpr int kRolePartial = 1;  // !tile_started: spill FP32 partials, then Signal
constexpr int kRoleOwner = 2;    // tile_started && !tile_ended: Wait peers, fix up, store

// Fixup flags per CTA: one per (TMEM lane quarter, output unit) of its
// partial tile, so the owner can consume a unit as soon as it is written.
constexpr int kFlagsPerCtaDev = 32;

constexpr int kTraceFields = 9;  // cta, tile, tm, tn, kb0, kb1, role, peer_first, peer_last
// Trace layout per CTA: a header of kTraceHeaderInts int32 (record count,
// reserved, u64 global-timer ns at kernel start) then records of
// kTraceRecordInts int32: the kTraceFields schedule fields, one reserved, and
// three u64 global-timer stamps (accumulator ready, fixup waits done, tile
// stored or partials signalled).
constexpr int kTraceHeaderInts = 4;
constexpr int kTraceRecordInts = 16;

// Device status codes written to the error word.
constexpr int kDevOk = 0;
constexpr int kDevTimeoutPipeline = 1;  // an mbarrier wait ran out
constexpr int kDevTimeoutFlag = 2;      // a fixup wait on a peer's flag ran out
constexpr int kDevAborted = 3;          // gave up because another CTA reported an error

// Division by a launch-invariant divisor d >= 1 for dividends n < 2^31 with
// one widening multiply (the round-up method of Granlund and Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994): with
// l = ceil(log2 d) and m = ceil(2^(31+l) / d), m < 2^32 and
// floor(n / d) = (n * m) >> (31 + l), because m*d - 2^(31+l) < d <= 2^l.
struct FastDiv {
  uint32_t m;
  uint32_t shift;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  const uint64_t m = ((uint64_t(1) << (31 + l)) + d - 1) / d;
  return FastDiv{static_cast<uint32_t>(m), 31 + l};
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fast_div(uint32_t n, FastDiv f) {
  return static_cast<uint32_t>((static_cast<uint64_t>(n) * f.m) >> f.shift);
}
#endif

// Grouped GEMM: one launch runs several problems as one Stream-K iteration
// space.  The host planner evaluates candidate schedules as per-CTA lists of
// segment records (also what the schedule query returns); the kernel derives
// the same segments from the walk table below.
struct alignas(16) GroupSeg {
  int32_t problem;
  int32_t tile;        // the problem's tile index (its raster order)
  int16_t tm, tn;      // tile row (128 rows) and column (BLK_N columns) in the problem
  int16_t kb0, kb1;    // MAC-loop iterations [kb0, kb1) of the tile
  int16_t role;        // kRoleWhole / kRolePartial / kRoleOwner
  int16_t kfull64;     // the problem's k-blocks of 64 entirely inside k
  int16_t peer_first;  // owner: contributing CTAs, else -1
  int16_t peer_last;
  int32_t pad[2];
};
static_assert(sizeof(GroupSeg) == 32, "segment record size");

// The walk of a grouped launch over problem i (device table of count + 1
// entries, the last a sentinel holding the totals): its first tile and first
// MAC-loop iteration in the concatenated space, its tile grid and raster,
// and the divisors the walk needs.  Each CTA derives its segments from this
// table exactly as the single-GEMM walk does (Stream-K share, then
// data-parallel tiles), advancing a problem cursor as it goes.
struct alignas(16) GroupWalk {
  int32_t tile_off;  // first global tile of the problem
  int32_t iter_off;  // first global iteration
  int32_t tiles_m, tiles_n;
  int32_t ipt;       // iterations per tile
  int32_t group_m;   // raster band height in tiles
  int32_t kfull64;   // k-blocks of 64 entirely inside k
  int32_t pad;
  FastDiv div_ipt, div_band, div_rows, div_rows_last;
};
static_assert(sizeof(GroupWalk) == 64, "walk entry size");

// Per-problem operands of a grouped launch (device memory, 128-byte aligned
// for the tensor maps, which TMA reads in place).
struct alignas(128) GroupProblem {
  CUtensorMap tmA, tmB, tmC, tmA3, tmB3;
  void* C;
  int64_t ldc;
  int32_t m, n;
  int32_t c_tma, c_vec;
  float alpha, beta;
  // E4M3 problems: FP32 scales per 128 x 128 block, [ceil(rows/128)][ld_scale]
  const float* scale_a;
  const float* scale_b;
  int32_t ld_scale;  // ceil(k / 128)
};

struct SkArgs {
  // problem
  int32_t m, n, k;
  int32_t tiles_m, tiles_n, tiles;
  int32_t iters_per_tile;  // ceil(k / BLK_K)
  int32_t group_m;         // raster band height in tiles
  // Stream-K region: tiles [0, sk_tiles), sk_iters = sk_tiles * iters_per_tile
  // split within one over the grid: CTA x owns [x*q + min(x,r), ...)
  int32_t sk_tiles;
  int32_t sk_q, sk_r;
  int32_t grid;  // g, persistent CTAs; data-parallel tiles sk_tiles + x + j*g
  // Divisors of the walk, precomputed: iterations per tile, q + 1 and q (the
  // Stream-K shares), the raster band's tiles and its height (a full band
  // and the last one).  fast_iters: the Stream-K iteration space is below
  // 2^31, so iteration indices use them; tile indices always do.
  FastDiv div_ipt, div_q1, div_q, div_band, div_rows, div_rows_last;
  int32_t fast_iters;
  int32_t kfull64;  // k-blocks of 64 that lie entirely inside k (3-D loads need two of them)
  // MMA instruction descriptor (input format bits, N, M)
  uint32_t idesc;
  // epilogue
  void* C;
  int64_t ldc;  // elements
  int32_t c_vec;  // rows of C start 16-byte aligned: 16-byte vector loads/stores allowed
  int32_t c_tma;  // 1: C through TMA tensor stores (tensor map valid); 2: coalesced
                  // stores from the staging buffer; 0: row-wise stores (C not 16-byte aligned)
  float alpha, beta;
  // fixup workspace: grid slots of BLK_M x BLK_N FP32, plus one flag per slot
  float* partials;
  uint32_t* flags;
  uint32_t epoch;
  // status, tracing, bounded waits
  int32_t* err;         // err[0]: first device status, err[1]: CTA, err[2]: where
  int32_t* err_host;    // nullptr, or mapped pinned host memory: a failing CTA also stores
                        // its status here, so the host sees it without a copy
  int32_t* trace;       // nullptr: off; else grid x (header + trace_cap records)
  int32_t trace_cap;    // records per CTA
  int32_t debug_skip_signal;  // CTA index that withholds its Signal (tests), -1 off
  uint64_t timeout_ns;
  int32_t pdl;  // launched with programmatic stream serialization (host side only)
  // 1: the operands (A, B, scales) are not written by the kernels before this
  // launch in its stream, so the producer and MMA warps start before those
  // kernels complete; only the epilogue warps (C, workspace) wait for them
  int32_t early;
  // pipeline stages the ring cycles through: 0 = all the kernel's ring holds,
  // else 2 .. that count
  int32_t stages;
  // grouped launches: the walk table and, per CTA x, the problems holding
  // its first Stream-K iteration (gstart[2x]) and first data-parallel tile
  // (gstart[2x + 1]); tiles / sk_tiles / sk_q / sk_r / grid describe the
  // concatenated space
  const GroupWalk* gwalk;
  const int32_t* gstart;
  const GroupProblem* gprobs;
  // E4M3 launches: FP32 scale of every 128 x 128 block of A (m x k) and of B
  // (n x k), row-major [ceil(rows / 128)][ld_scale], ld_scale = ceil(k / 128)
  const float* scale_a;
  const float* scale_b;
  int32_t ld_scale;
};

}  // namespace sk
