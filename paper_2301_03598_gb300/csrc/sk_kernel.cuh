// Persistent Stream-K GEMM kernel for sm_103a.
//
// One kernel serves every schedule of the paper: data-parallel (Algorithm 2,
// Stream-K region empty), basic Stream-K (Algorithm 5, data-parallel region
// empty) and the hybrids of Section 5.2 (a Stream-K region over the first
// sk_tiles tiles followed by full data-parallel waves).  The schedule is a pure
// function of (blockIdx.x, SkArgs) that all three warp roles walk in lockstep.
//
// Roles (320 threads, one CTA per SM):
//   warp 0      TMA producer: streams the A and B fragments of every MAC-loop
//               iteration (Algorithm 3's LoadFragment) into an S-stage ring of
//               128-byte-swizzled shared-memory tiles.
//   warp 1      TMEM allocator and MMA issuer: one thread issues four
//               tcgen05.mma per 128-byte k-block into one of two TMEM
//               accumulators (E4M3: one product per k-block, a stage's two
//               k-blocks into one of two buffer pairs).
//   warps 2..9  epilogue: (E4M3: first sums the k-block products times their
//               block scales in FP32) per tile segment, either spill the FP32
//               partial sums to this CTA's workspace slot and Signal (segment
//               does not start the tile), or Wait for the contributing CTAs
//               (all their flags polled at once) and add their partials in
//               increasing CTA order (tile started here, not finished here),
//               then compute alpha*acc + beta*C and store the tile.
//
// A grouped launch walks the problems' concatenated iteration space with the
// same roles, reading each problem's operands, output and scales from device
// tables.
//
// Every wait is bounded by SkArgs::timeout_ns; on expiry the kernel records a
// status in SkArgs::err and all roles unwind, drain their in-flight TMA loads
// and MMAs, free TMEM and return.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ptx.cuh"
#include "sk_args.h"

namespace sk {

constexpr int kEpiWarps = 8;  // two warps per TMEM lane quarter, splitting the columns
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr uint32_t kEpiBarrier = 1;  // named barrier id of the epilogue warps

// Shared-memory stage ring per CTA: 192 KiB of operand stages.  A k-block is
// one 128-byte row per operand row: 64 16-bit elements, or 128 E4M3 elements
// (F8).  A stage holds KD consecutive k-blocks (one MAC-loop iteration):
// KD = 2 for BLK_N = 64 and 128, whose 2-D stages are too small for the SM's
// TMA path (a stage costs about as much as its bytes), KD = 1 for 256.
//
// F8 (E4M3 operands with one FP32 scale per 128 x 128 block of A and of B):
// the host describes the operands to TMA as 16-bit rows of k/2 elements (the
// same bytes), so loads and stages are the 16-bit path's.  Every k-block is
// one scale block: the MMA warp writes the products of a stage's KD k-blocks
// into the KD TMEM buffers of one of kAccBufs = 2 buffer groups (pairs for
// BLK_N = 128, single 256-column buffers for BLK_N = 256) and publishes them
// with one commit; the epilogue warps add each product, times its block's two
// scales, into a running FP32 sum held in registers (BLK_N / 2 per thread),
// and release the group.  The tile segment's sum goes to the first buffer of
// the segment's last group, which is released only after the common epilogue
// has read it.  A stage's second k-block beyond k (an odd count of k-blocks
// with KD = 2) is zero-filled by TMA and carries scale 0.
template <int BN, int CM, bool F8 = false>
struct Cfg {
  static constexpr int KD = BN <= 128 ? 2 : 1;
  static constexpr int kSubA = kBlkM * 128;          // one k-block of this CTA's 128 A rows
  static constexpr int kSubB = (BN / CM) * 128;      // one k-block of its BN/CM B rows
  static constexpr int kABytes = KD * kSubA;
  static constexpr int kBBytes = KD * kSubB;
  static constexpr int kStageBytes = kABytes + kBBytes;
  // 4, 4 (BN 64); 3, 4 (BN 128); 4, 6 (BN 256); F8: 3
  static constexpr int kStages = (192 * 1024) / kStageBytes;
  // two accumulators (F8: two pairs of KD product buffers, one pair per stage)
  static constexpr int kAccBufs = 2;
  static constexpr int kAccCols = F8 ? KD * BN : BN;  // TMEM columns of one of them
  static constexpr int kTmemCols = kAccBufs * kAccCols;
  // Output staging for TMA stores: per epilogue warp one buffer of 32 rows x
  // 128 B, 128-byte swizzled (1 KiB aligned).
  static constexpr int kStagingOffset = kStages * kStageBytes;
  static constexpr int kStagingBytesPerWarp = 32 * 128;
  static constexpr int kStagingBytes = kEpiWarps * kStagingBytesPerWarp;
  static constexpr int kBarOffset = kStagingOffset + kStagingBytes;
  static constexpr int kNumBars = 2 * kStages + 2 * kAccBufs + 1;
  static constexpr int kSmemBytes = kBarOffset + 256 + 1024;  // + barriers, + 1 KiB alignment
  static_assert(kNumBars * 8 + 8 <= 256, "barrier area");
  static_assert(kSmemBytes <= 232448, "shared memory per CTA");
  static_assert(!F8 || BN == 128 || (BN == 256 && CM == 1),
                "F8 tiles are 128 x 128 (256 x 128 on a pair) or 128 x 256");
  static_assert(kTmemCols <= 512, "TMEM columns");
  // Warps: 0 producer, 1 MMA issuer, then the epilogue warps from kEpiWarp0.
  // 10 warps put three on two of the SM's four sub-partitions, which caps a
  // thread at 168 registers (a sub-partition's file holds 512 per lane).  The
  // E4M3 128 x 256 tile's running sum alone is 128 registers per epilogue
  // thread, so that kernel runs 12 warps -- warpgroup 0 (producer, MMA issuer
  // and two idle warps) and two epilogue warpgroups -- launched at 168 and
  // rebalanced with setmaxnreg: warpgroup 0 gives up registers down to
  // kRegsLow, the epilogue raises to kRegsHigh, kRegsLow + 2 kRegsHigh = 3 x 168.
  static constexpr bool kRebalance = F8 && BN == 256;
  static constexpr int kEpiWarp0 = kRebalance ? 4 : 2;
  static constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);
  static constexpr int kRegsLaunch = 168;
  static constexpr int kRegsLow = 56;
  static constexpr int kRegsHigh = 224;
  static_assert(kRegsLow + 2 * kRegsHigh <= 3 * kRegsLaunch, "register rebalance exceeds the launch");
};

// Where a bounded wait gave up (err[2]).
enum : int { kAtProducerEmpty = 1, kAtMmaAccEmpty, kAtMmaFull, kAtEpiAccFull, kAtFlag, kAtDrain };

__device__ __forceinline__ void report(const SkArgs& a, int code, int where) {
  if (atomicCAS(&a.err[0], 0, code) == 0) {
    a.err[1] = static_cast<int32_t>(blockIdx.x);
    a.err[2] = where;
  }
  atomicExch(reinterpret_cast<unsigned*>(&a.err[3]), a.epoch);
  __threadfence();
  if (a.err_host != nullptr) {
    *reinterpret_cast<volatile int32_t*>(a.err_host) = code;
    __threadfence_system();
  }
}

// Bounded mbarrier wait.  Returns false if this CTA is aborting or the time
// limit ran out (then it also records the timeout and raises the CTA's abort).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                         const SkArgs& a, int where) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0) {
      if (*abort_flag) return false;
      if (globaltimer_ns() - t0 > a.timeout_ns) {
        report(a, kDevTimeoutPipeline, where);
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// Bounded Wait(flags[y]) of Algorithms 4/5: acquire-load until the peer has
// published this launch's epoch.
__device__ __forceinline__ bool wait_flag(const uint32_t* flag, volatile int* abort_flag,
                                          const SkArgs& a) {
  if (ld_acquire_gpu(flag) == a.epoch) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t i = 1;; ++i) {
    if (i > 256) __nanosleep(64);  // spin tightly first: the peer is usually about to publish
    if (ld_acquire_gpu(flag) == a.epoch) return true;
    if ((i & 31u) == 0) {
      if (*abort_flag) return false;
      if (static_cast<uint32_t>(ld_volatile_s32(&a.err[3])) == a.epoch) {  // another CTA failed
        report(a, kDevAborted, kAtFlag);
        *abort_flag = 1;
        return false;
      }
      if (globaltimer_ns() - t0 > a.timeout_ns) {
        report(a, kDevTimeoutFlag, kAtFlag);
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// Epilogue-wide OR of a per-thread predicate (bar.red over the 128 epilogue
// threads), so that every epilogue thread takes the same branch.
__device__ __forceinline__ bool epi_any(bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"(pred ? 1u : 0u), "r"(kEpiBarrier), "r"(kEpiThreads)
      : "memory");
  return out != 0;
}

// The CTA's walk over its tile segments: first its within-one share of the
// Stream-K iteration range (Algorithm 5), then its data-parallel tiles.
struct Walker {
  int64_t it, it_end;
  int32_t dp_tile;

  __device__ __forceinline__ void init(const SkArgs& a, int x) {
    const int64_t q = a.sk_q, r = a.sk_r;
    it = static_cast<int64_t>(x) * q + min(static_cast<int64_t>(x), r);
    it_end = it + q + (x < r ? 1 : 0);
    dp_tile = a.sk_tiles + x;
  }

  __device__ __forceinline__ bool next(const SkArgs& a, int& tile, int& kb0, int& kb1) {
    if (it < it_end) {
      const int64_t ipt = a.iters_per_tile;
      tile = a.fast_iters ? static_cast<int>(fast_div(static_cast<uint32_t>(it), a.div_ipt))
                          : static_cast<int>(it / ipt);
      const int64_t tile_iter = static_cast<int64_t>(tile) * ipt;
      const int64_t tile_iter_end = tile_iter + ipt;
      kb0 = static_cast<int>(it - tile_iter);
      kb1 = static_cast<int>(min(it_end, tile_iter_end) - tile_iter);
      it = tile_iter_end;
      return true;
    }
    if (dp_tile < a.tiles) {
      tile = dp_tile;
      kb0 = 0;
      kb1 = a.iters_per_tile;
      dp_tile += a.grid;
      return true;
    }
    return false;
  }
};

// The CTA whose Stream-K range holds global iteration i.
__device__ __forceinline__ int cta_of_iter(const SkArgs& a, int64_t i) {
  if (a.fast_iters) {
    const uint32_t i32 = static_cast<uint32_t>(i);
    const uint32_t big = static_cast<uint32_t>(a.sk_r) * static_cast<uint32_t>(a.sk_q + 1);
    return static_cast<int>(i32 < big ? fast_div(i32, a.div_q1)
                                      : static_cast<uint32_t>(a.sk_r) + fast_div(i32 - big, a.div_q));
  }
  const int64_t q = a.sk_q, r = a.sk_r;
  const int64_t big = r * (q + 1);
  if (i < big) return static_cast<int>(i / (q + 1));
  return static_cast<int>(r + (i - big) / q);
}

// Tile raster: m fastest within bands of group_m tile rows.
__device__ __forceinline__ void tile_coords(const SkArgs& a, int tile, int& tm, int& tn) {
  const int band_tiles = a.group_m * a.tiles_n;
  const int band = static_cast<int>(fast_div(static_cast<uint32_t>(tile), a.div_band));
  const int first_m = band * a.group_m;
  const int rows = min(a.group_m, a.tiles_m - first_m);
  const int local = tile - band * band_tiles;
  tn = static_cast<int>(
      fast_div(static_cast<uint32_t>(local), rows == a.group_m ? a.div_rows : a.div_rows_last));
  tm = first_m + local - tn * rows;
}

// One segment of a CTA's walk, as every role sees it.  Peers are schedule
// units (CTA pairs count once); the epilogue turns them into CTA indices.
struct Seg {
  int problem, tile, tm, tn, kb0, kb1, role, peer_first, peer_last, kfull64;
};

// Tile raster of one problem of a grouped launch (as tile_coords).
__device__ __forceinline__ void group_tile_coords(const GroupWalk& w, int tile, int& tm, int& tn) {
  const int band_tiles = w.group_m * w.tiles_n;
  const int band = static_cast<int>(fast_div(static_cast<uint32_t>(tile), w.div_band));
  const int first_m = band * w.group_m;
  const int rows = min(w.group_m, w.tiles_m - first_m);
  const int local = tile - band * band_tiles;
  tn = static_cast<int>(
      fast_div(static_cast<uint32_t>(local), rows == w.group_m ? w.div_rows : w.div_rows_last));
  tm = first_m + local - tn * rows;
}

// A CTA's segments, derived from its Stream-K share and data-parallel tiles:
// of one GEMM, or (grouped) of the problems' concatenated iteration space,
// where a problem cursor follows the CTA through the walk table.
template <bool GROUPED>
struct SegCursor {
  Walker w;
  int x, pi_sk, pi_dp;

  __device__ __forceinline__ void init(const SkArgs& a, int unit) {
    x = unit;
    w.init(a, unit);
    if constexpr (GROUPED) {
      pi_sk = a.gstart[2 * unit];
      pi_dp = a.gstart[2 * unit + 1];
    }
  }

  __device__ __forceinline__ bool next(const SkArgs& a, Seg& s) {
    if constexpr (GROUPED) {
      const GroupWalk* gw = a.gwalk;
      int lt;
      if (w.it < w.it_end) {
        // Algorithm 5 over the concatenated iterations
        const int32_t it = static_cast<int32_t>(w.it);
        while (gw[pi_sk + 1].iter_off <= it) ++pi_sk;
        const GroupWalk p = gw[pi_sk];
        const int32_t local = it - p.iter_off;
        lt = static_cast<int>(fast_div(static_cast<uint32_t>(local), p.div_ipt));
        const int32_t start = p.iter_off + lt * p.ipt;
        const int32_t end = start + p.ipt;
        s.problem = pi_sk;
        s.kb0 = it - start;
        s.kb1 = static_cast<int>(min(w.it_end, static_cast<int64_t>(end)) - start);
        s.role = s.kb0 != 0 ? kRolePartial : (s.kb1 != p.ipt ? kRoleOwner : kRoleWhole);
        s.peer_first = s.peer_last = -1;
        if (s.role == kRoleOwner) {
          s.peer_first = x + 1;
          s.peer_last = cta_of_iter(a, end - 1);
        }
        s.kfull64 = p.kfull64;
        group_tile_coords(p, lt, s.tm, s.tn);
        w.it = end;
      } else if (w.dp_tile < a.tiles) {
        const int32_t j = w.dp_tile;
        while (gw[pi_dp + 1].tile_off <= j) ++pi_dp;
        const GroupWalk p = gw[pi_dp];
        lt = j - p.tile_off;
        s.problem = pi_dp;
        s.kb0 = 0;
        s.kb1 = p.ipt;
        s.role = kRoleWhole;
        s.peer_first = s.peer_last = -1;
        s.kfull64 = p.kfull64;
        group_tile_coords(p, lt, s.tm, s.tn);
        w.dp_tile += a.grid;
      } else {
        return false;
      }
      s.tile = lt;
      return true;
    } else {
      int tile, kb0, kb1;
      if (!w.next(a, tile, kb0, kb1)) return false;
      const int ipt = a.iters_per_tile;
      s.problem = 0;
      s.tile = tile;
      s.kb0 = kb0;
      s.kb1 = kb1;
      s.role = kb0 != 0 ? kRolePartial : (kb1 != ipt ? kRoleOwner : kRoleWhole);
      s.peer_first = s.peer_last = -1;
      if (s.role == kRoleOwner) {
        s.peer_first = x + 1;
        s.peer_last = cta_of_iter(a, static_cast<int64_t>(tile) * ipt + ipt - 1);
      }
      tile_coords(a, tile, s.tm, s.tn);
      s.kfull64 = a.kfull64;
      return true;
    }
  }
};

template <typename TC>
__device__ __forceinline__ float to_f32(TC v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

template <typename TC>
__device__ __forceinline__ TC from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi, __nv_bfloat16*) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi, __half*) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack2(uint32_t u, __nv_bfloat16*) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
  return __bfloat1622float2(h);
}
__device__ __forceinline__ float2 unpack2(uint32_t u, __half*) {
  __half2 h = *reinterpret_cast<__half2*>(&u);
  return __half22float2(h);
}

// Where and how a segment's output tile goes: the launch's C (single GEMM) or
// the segment's problem's C (grouped).
struct OutView {
  void* C;
  int64_t ldc;
  int32_t m, n;
  int32_t c_vec, c_tma;
  float alpha, beta;
  const CUtensorMap* tmC;
};

// StoreTile for one thread's 32 consecutive columns of one row:
// C[row, col .. col+31] = alpha * v + beta * C[row, col .. col+31].
template <typename TC>
__device__ __forceinline__ void store_row32(const OutView& o, int grow, int gcol, const float (&v)[32]) {
  if (grow >= o.m) return;
  TC* crow = reinterpret_cast<TC*>(o.C) + static_cast<int64_t>(grow) * o.ldc + gcol;
  const float alpha = o.alpha, beta = o.beta;
  if (o.c_vec && gcol + 32 <= o.n) {
    if constexpr (sizeof(TC) == 4) {
      float4* p = reinterpret_cast<float4*>(crow);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float4 o = make_float4(alpha * v[4 * j], alpha * v[4 * j + 1], alpha * v[4 * j + 2],
                               alpha * v[4 * j + 3]);
        if (beta != 0.0f) {
          const float4 c = p[j];
          o.x = fmaf(beta, c.x, o.x);
          o.y = fmaf(beta, c.y, o.y);
          o.z = fmaf(beta, c.z, o.z);
          o.w = fmaf(beta, c.w, o.w);
        }
        p[j] = o;
      }
    } else {
      uint4* p = reinterpret_cast<uint4*>(crow);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) o[e] = alpha * v[8 * j + e];
        if (beta != 0.0f) {
          const uint4 c = p[j];
          const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 f = unpack2(cw[e], static_cast<TC*>(nullptr));
            o[2 * e] = fmaf(beta, f.x, o[2 * e]);
            o[2 * e + 1] = fmaf(beta, f.y, o[2 * e + 1]);
          }
        }
        uint4 w;
        w.x = pack2(o[0], o[1], static_cast<TC*>(nullptr));
        w.y = pack2(o[2], o[3], static_cast<TC*>(nullptr));
        w.z = pack2(o[4], o[5], static_cast<TC*>(nullptr));
        w.w = pack2(o[6], o[7], static_cast<TC*>(nullptr));
        p[j] = w;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (gcol + j < o.n) {
        float o = alpha * v[j];
        if (beta != 0.0f) o = fmaf(beta, to_f32<TC>(crow[j]), o);
        crow[j] = from_f32<TC>(o);
      }
    }
  }
}

// 16 bytes of output (8 16-bit or 4 FP32 values, packed as stored) at
// C[row, col ..]: one vector store when the chunk lies inside the matrix,
// else element by element up to column n.
template <typename TC>
__device__ __forceinline__ void store_chunk16(const OutView& o, int grow, int gcol, uint32_t w0,
                                              uint32_t w1, uint32_t w2, uint32_t w3) {
  constexpr int kPer = 16 / static_cast<int>(sizeof(TC));
  TC* dst = reinterpret_cast<TC*>(o.C) + static_cast<int64_t>(grow) * o.ldc + gcol;
  if (gcol + kPer <= o.n) {
    *reinterpret_cast<uint4*>(dst) = make_uint4(w0, w1, w2, w3);
  } else if (gcol < o.n) {
    const uint32_t w[4] = {w0, w1, w2, w3};
    const TC* vals = reinterpret_cast<const TC*>(w);
#pragma unroll
    for (int e = 0; e < kPer; ++e)
      if (gcol + e < o.n) dst[e] = vals[e];
  }
}

// v[j] += beta * C[row, col + j] for the columns of this chunk inside the matrix.
template <typename TC>
__device__ __forceinline__ void add_beta_c(const OutView& o, int grow, int gcol, float (&v)[32]) {
  if (grow >= o.m) return;
  const TC* crow = reinterpret_cast<const TC*>(o.C) + static_cast<int64_t>(grow) * o.ldc + gcol;
  const float beta = o.beta;
  if (o.c_vec && gcol + 32 <= o.n) {
    if constexpr (sizeof(TC) == 4) {
      const float4* p = reinterpret_cast<const float4*>(crow);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 c = p[j];
        v[4 * j] = fmaf(beta, c.x, v[4 * j]);
        v[4 * j + 1] = fmaf(beta, c.y, v[4 * j + 1]);
        v[4 * j + 2] = fmaf(beta, c.z, v[4 * j + 2]);
        v[4 * j + 3] = fmaf(beta, c.w, v[4 * j + 3]);
      }
    } else {
      const uint4* p = reinterpret_cast<const uint4*>(crow);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint4 c = p[j];
        const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 f = unpack2(cw[e], static_cast<TC*>(nullptr));
          v[8 * j + 2 * e] = fmaf(beta, f.x, v[8 * j + 2 * e]);
          v[8 * j + 2 * e + 1] = fmaf(beta, f.y, v[8 * j + 2 * e + 1]);
        }
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (gcol + j < o.n) v[j] = fmaf(beta, to_f32<TC>(crow[j]), v[j]);
  }
}

// v += P[first] + P[first + CM] + ... + P[last], added one peer at a time in
// that order (Algorithm 5's fixup), for one lane's 32 columns of one (32-column
// chunk, lane quarter) block of the peers' partial slots, blk = chunk * 4 +
// quarter.  Two peers' 4 KiB blocks per warp are in flight.
template <int CM, int BN>
__device__ __forceinline__ void add_peers(const float* partials, int first, int last, int blk,
                                          int lane, float (&v)[32]) {
  for (int y = first; y <= last; y += 2 * CM) {
    const float4* s0 = reinterpret_cast<const float4*>(partials + static_cast<size_t>(y) * (kBlkM * BN)) +
                       blk * 256 + lane;
    const bool two = y + CM <= last;
    const float4* s1 = two ? s0 + CM * (kBlkM * BN) / 4 : s0;
    float4 p0[8], p1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) p0[j] = __ldcg(s0 + j * 32);
    if (two) {
#pragma unroll
      for (int j = 0; j < 8; ++j) p1[j] = __ldcg(s1 + j * 32);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[4 * j] += p0[j].x;
      v[4 * j + 1] += p0[j].y;
      v[4 * j + 2] += p0[j].z;
      v[4 * j + 3] += p0[j].w;
    }
    if (two) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        v[4 * j] += p1[j].x;
        v[4 * j + 1] += p1[j].y;
        v[4 * j + 2] += p1[j].z;
        v[4 * j + 3] += p1[j].w;
      }
    }
  }
}

// CM = CTAs per cluster along M (1 or 2).  With CM = 2 the two CTAs of a
// cluster form a tcgen05 CTA pair computing one 256 x BN tile: the schedule's
// unit is that tile.  Each CTA loads its own 128 rows of A and BN/2 rows of B
// per k-block, the even CTA issues the pair MMAs (M = 256), and each CTA's
// TMEM receives its own 128 rows of the accumulator, which its epilogue
// spills, fixes up and stores exactly as a single CTA does.
template <int BN, int CM, typename TC, bool GROUPED, bool F8>
__global__ void __launch_bounds__(Cfg<BN, CM, F8>::kThreads, 1)
    sk_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmA3,
                   const __grid_constant__ CUtensorMap tmB3, const __grid_constant__ SkArgs a) {
  static_assert(CM == 1 || CM == 2, "cluster size along M");
  using C_ = Cfg<BN, CM, F8>;
  constexpr int NB = C_::kAccBufs;
  constexpr int S = C_::kStages;
  // The ring's stages the MAC loop cycles through (SkArgs::stages, the
  // autotuners' pipeline-depth choice; the full ring by default).
  const int nst = a.stages >= 2 && a.stages < S ? a.stages : S;
  constexpr int KD = C_::KD;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 128-byte swizzle atoms need 1 KiB alignment
  uint8_t* base_ptr = smem_raw + (base - raw);
  const uint32_t bar0 = base + C_::kBarOffset;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + C_::kBarOffset + 8 * C_::kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  auto stage_a = [&](int s) { return base + static_cast<uint32_t>(s * C_::kStageBytes); };
  auto stage_b = [&](int s) { return base + static_cast<uint32_t>(s * C_::kStageBytes + C_::kABytes); };
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * S + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * S + NB + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * S + 2 * NB);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int cta = blockIdx.x;                                 // this CTA (flags, partials, trace)
  const int rank = CM == 2 ? static_cast<int>(cluster_ctarank()) : 0;
  const int x = cta / CM;                                     // schedule unit (CTA pair)
  constexpr bool kPair = CM == 2;
  constexpr uint16_t kPairMask = 0x3;
  // In a pair the even CTA's full and acce barriers gather both CTAs: the
  // shared::cluster addresses of the even CTA's copies.
  const uint32_t full0 = kPair ? mapa_shared(full_bar(0), 0) : full_bar(0);
  const uint32_t acce0 = kPair ? mapa_shared(acce_bar(0), 0) : acce_bar(0);
  const bool issuer = !kPair || rank == 0;  // this CTA issues the MMAs
  // An epilogue warp has read accumulator b: tell the issuer it may reuse it.
  auto release_acc = [&](int b) {
    if constexpr (kPair)
      mbar_arrive_cluster(acce0 + 8u * b);
    else
      mbar_arrive(acce_bar(b));
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1);   // the issuer's producer arrives with both CTAs' bytes
      mbar_init(empty_bar(s), 1);  // released by the issuer's commit
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), CM * kEpiWarps);  // every epilogue warp of the pair
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    if constexpr (!GROUPED) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      if (a.c_tma == 1) tma_prefetch_desc(&tmC);
      if (KD == 2 && a.kfull64 >= 2) {
        tma_prefetch_desc(&tmA3);
        tma_prefetch_desc(&tmB3);
      }
    }
  }
  if (warp == 1) {
    if constexpr (kPair) {
      tmem_alloc_pair(smem_u32(tmem_slot), C_::kTmemCols);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), C_::kTmemCols);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (kPair) cluster_sync();  // both CTAs' barriers exist before either signals them
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // Everything above overlaps the previous kernel in the stream under
  // programmatic dependent launch; nothing is loaded into shared memory or
  // written to global memory before this point.  By default every thread
  // waits for that kernel to complete at the top of its role below.  With
  // a.early the caller has declared the operands independent of the
  // preceding kernels: the producer and MMA warps go ahead, so the MAC loop
  // overlaps the previous kernel's tail, and the next kernel may launch at
  // once; only the epilogue warps, which read and write C and the fixup
  // workspace, wait.  (The wait sits inside each role's branch: one shared
  // conditional wait here made the grouped E4M3 kernel 11% slower.)

  if (warp < C_::kEpiWarp0) {
    // Register rebalance (warpgroup-uniform; the host checked that the launch's
    // registers cover it): warpgroup 0 releases, the epilogue warpgroups take.
    if constexpr (C_::kRebalance) setmaxnreg_dec<C_::kRegsLow>();
    if (warp == 0) {
      if (!a.early) grid_dependency_wait();
      if (lane == 0) {
        // ------------------------------------------------------------ producer
        SegCursor<GROUPED> cur;
        cur.init(a, x);
        Seg sg;
        int last_problem = -1;  // grouped: the problem whose tensor maps were last acquired
        int stage = 0;
        uint32_t phase = 0;
        int64_t issued = 0;
        bool ok = true;
        // ready: the current stage's empty barrier is known to have completed
        // (probed while the previous stage's B load was issued).
        bool ready = false;
        while (ok && cur.next(a, sg)) {
          const int kb0 = sg.kb0, kb1 = sg.kb1;
          const int tm = sg.tm * CM + rank;  // this CTA's 128-row block
          const int tn = sg.tn;
          const CUtensorMap *pA = &tmA, *pB = &tmB, *pA3 = &tmA3, *pB3 = &tmB3;
          if constexpr (GROUPED) {
            const GroupProblem* gp = a.gprobs + sg.problem;
            pA = &gp->tmA;
            pB = &gp->tmB;
            pA3 = &gp->tmA3;
            pB3 = &gp->tmB3;
            if (sg.problem != last_problem) {
              tensormap_acquire(pA);
              tensormap_acquire(pB);
              tensormap_acquire(pA3);
              tensormap_acquire(pB3);
              last_problem = sg.problem;
            }
          }
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!ready && !wait_bar(empty_bar(stage), phase ^ 1u, abort_flag, a, kAtProducerEmpty)) {
              ok = false;
              break;
            }
            int next = stage + 1;
            uint32_t next_phase = phase;
            if (next == nst) {
              next = 0;
              next_phase ^= 1u;
            }
            // k-blocks k0 .. k0+KD-1 of this CTA's A rows and its BN/CM rows of
            // B.  A KD = 2 stage of two full k-blocks is one 3-D box per
            // operand; a stage reaching into the k tail loads its k-blocks as
            // 2-D boxes, whose out-of-range columns TMA fills with zeros.
            const int k0 = kb * KD;
            const bool box3 = KD == 2 && k0 + 2 <= sg.kfull64;
            const int brow = tn * BN + rank * (BN / CM);
            if constexpr (kPair) {
              // completing on the issuer's full barrier, which expects both
              // CTAs' bytes
              const uint32_t fb = full0 + 8u * stage;
              if (rank == 0) mbar_arrive_expect_tx(full_bar(stage), 2 * C_::kStageBytes);
              if (box3) {
                tma_load_3d_pair(stage_a(stage), pA3, fb, 0, tm * kBlkM, k0);
                ready = tma_load_3d_pair_probe(stage_b(stage), pB3, fb, 0, brow, k0, empty_bar(next),
                                               next_phase ^ 1u);
              } else if constexpr (KD == 1) {
                tma_load_2d_pair(stage_a(stage), pA, fb, k0 * kBlkK, tm * kBlkM);
                ready = tma_load_2d_pair_probe(stage_b(stage), pB, fb, k0 * kBlkK, brow,
                                               empty_bar(next), next_phase ^ 1u);
              } else {
#pragma unroll
                for (int j = 0; j < KD; ++j) {
                  tma_load_2d_pair(stage_a(stage) + j * C_::kSubA, pA, fb, (k0 + j) * kBlkK, tm * kBlkM);
                  tma_load_2d_pair(stage_b(stage) + j * C_::kSubB, pB, fb, (k0 + j) * kBlkK, brow);
                }
                ready = false;
              }
            } else {
              const uint32_t fb = full_bar(stage);
              mbar_arrive_expect_tx(fb, C_::kStageBytes);
              if (box3) {
                tma_load_3d(stage_a(stage), pA3, fb, 0, tm * kBlkM, k0);
                ready = tma_load_3d_probe(stage_b(stage), pB3, fb, 0, brow, k0, empty_bar(next),
                                          next_phase ^ 1u);
              } else if constexpr (KD == 1) {
                tma_load_2d(stage_a(stage), pA, fb, k0 * kBlkK, tm * kBlkM);
                ready = tma_load_2d_probe(stage_b(stage), pB, fb, k0 * kBlkK, brow, empty_bar(next),
                                          next_phase ^ 1u);
              } else {
#pragma unroll
                for (int j = 0; j < KD; ++j) {
                  tma_load_2d(stage_a(stage) + j * C_::kSubA, pA, fb, (k0 + j) * kBlkK, tm * kBlkM);
                  tma_load_2d(stage_b(stage) + j * C_::kSubB, pB, fb, (k0 + j) * kBlkK, brow);
                }
                ready = false;
              }
            }
            ++issued;
            stage = next;
            phase = next_phase;
          }
        }
        if (ok) {
          // Tail: wait until the MMA warp has released every stage, so no
          // tcgen05.commit arrival is still in flight when the CTA exits.
          for (int i = 0; i < nst; ++i) {
            if (!wait_bar(empty_bar(stage), phase ^ 1u, abort_flag, a, kAtProducerEmpty)) break;
            if (++stage == nst) {
              stage = 0;
              phase ^= 1u;
            }
          }
        } else {
          // Unwind: let the loads already issued land before shared memory
          // goes away.  They complete within microseconds; the waits share one
          // bound.  A pair's odd CTA cannot observe its loads (they complete on
          // the even CTA's barriers), so it waits out a fixed interval.
          constexpr uint64_t kUnwindNs = 1000000;
          const uint64_t t0 = globaltimer_ns();
          if (issuer) {
            const int64_t first = issued > nst ? issued - nst : 0;
            for (int64_t j = first; j < issued; ++j) {
              const int s = static_cast<int>(j % nst);
              const uint32_t par = static_cast<uint32_t>((j / nst) & 1);
              while (!mbar_try_wait(full_bar(s), par) && globaltimer_ns() - t0 < kUnwindNs) {
              }
            }
          } else {
            while (globaltimer_ns() - t0 < kUnwindNs / 20) {
            }
          }
        }
      }
    } else if (warp == 1) {
      if (!a.early)
        grid_dependency_wait();
      else if (lane == 0)
        grid_launch_dependents();
      if (lane == 0 && !issuer) grid_launch_dependents();  // a pair's odd CTA issues nothing
      if (lane == 0 && issuer) {
        // ------------------------------------------------------------ MMA issuer
        SegCursor<GROUPED> cur;
        cur.init(a, x);
        Seg sg;
        int stage = 0, acc = 0;
        uint32_t phase = 0, acc_phase = 0;
        bool ok = true;
        // ready: the current stage's full barrier is known to have completed
        // (probed while the previous k-block's last MMA was issued).
        bool ready = false;
        if constexpr (F8) {
          // One product per k-block (one scale block); a stage's KD k-blocks
          // go to the KD buffers of one pair, published with one commit; the
          // epilogue warps scale and sum them.
          // ready_acc: the current pair is known to be free (probed with the
          // previous stage's last MMA, like `ready` for the stage)
          bool ready_acc = false;
          while (ok && cur.next(a, sg)) {
            for (int kb = sg.kb0; kb < sg.kb1; ++kb) {
              if (!ready && !wait_bar(full_bar(stage), phase, abort_flag, a, kAtMmaFull)) {
                ok = false;
                break;
              }
              if (!ready_acc && !wait_bar(acce_bar(acc), acc_phase ^ 1u, abort_flag, a, kAtMmaAccEmpty)) {
                ok = false;
                break;
              }
              tc_fence_after();
              int next = stage + 1;
              uint32_t next_phase = phase;
              if (next == nst) {
                next = 0;
                next_phase ^= 1u;
              }
              const int nacc = acc ^ 1;
              const uint32_t nacc_phase = acc == 1 ? acc_phase ^ 1u : acc_phase;
#pragma unroll
              for (int j = 0; j < KD; ++j) {
                const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * C_::kAccCols + j * BN);
                const uint64_t adesc = smem_desc_sw128(stage_a(stage) + j * C_::kSubA);
                const uint64_t bdesc = smem_desc_sw128(stage_b(stage) + j * C_::kSubB);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                  // 32 E4M3 elements (32 B) along K per MMA
                  if (j == KD - 1 && kk == 3) {
                    // the stage's last MMA: probe the next stage and the next pair
                    uint32_t r;
                    if constexpr (kPair)
                      r = mma_f8_pair_probe2(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, a.idesc, 1u,
                                             full_bar(next), next_phase, acce_bar(nacc), nacc_phase ^ 1u);
                    else
                      r = mma_f8_probe2(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, a.idesc, 1u,
                                        full_bar(next), next_phase, acce_bar(nacc), nacc_phase ^ 1u);
                    ready = (r & 1u) != 0;
                    ready_acc = (r & 2u) != 0;
                  } else if constexpr (kPair) {
                    mma_f8_pair(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, a.idesc, kk > 0 ? 1u : 0u);
                  } else {
                    mma_f8(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, a.idesc, kk > 0 ? 1u : 0u);
                  }
                }
              }
              // publishes the pair's products, then frees the stage (in both
              // CTAs of a pair) once these MMAs finish
              if constexpr (kPair) {
                mma_commit_pair_multicast(accf_bar(acc), kPairMask);
                mma_commit_pair_multicast(empty_bar(stage), kPairMask);
              } else {
                mma_commit(accf_bar(acc));
                mma_commit(empty_bar(stage));
              }
              stage = next;
              phase = next_phase;
              acc = nacc;
              acc_phase = nacc_phase;
            }
          }
        }
        while (!F8 && ok && cur.next(a, sg)) {
          const int kb0 = sg.kb0, kb1 = sg.kb1;
          if (!wait_bar(acce_bar(acc), acc_phase ^ 1u, abort_flag, a, kAtMmaAccEmpty)) break;
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * BN);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!ready && !wait_bar(full_bar(stage), phase, abort_flag, a, kAtMmaFull)) {
              ok = false;
              break;
            }
            tc_fence_after();
            int next = stage + 1;
            uint32_t next_phase = phase;
            if (next == nst) {
              next = 0;
              next_phase ^= 1u;
            }
#pragma unroll
            for (int j = 0; j < KD; ++j) {
              const uint64_t adesc = smem_desc_sw128(stage_a(stage) + j * C_::kSubA);
              const uint64_t bdesc = smem_desc_sw128(stage_b(stage) + j * C_::kSubB);
#pragma unroll
              for (int kk = 0; kk < kBlkK / 16; ++kk) {
                // advance 16 elements (32 B) along K inside the swizzle atom
                const uint32_t acc_flag = (kb > kb0 || j > 0 || kk > 0) ? 1u : 0u;
                if (j == KD - 1 && kk == kBlkK / 16 - 1) {
                  // the stage's last MMA, fused with a probe of the next stage
                  if constexpr (kPair)
                    ready = mma_f16_pair_probe(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, a.idesc,
                                               acc_flag, full_bar(next), next_phase);
                  else
                    ready = mma_f16_probe(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, a.idesc, acc_flag,
                                          full_bar(next), next_phase);
                } else if constexpr (kPair) {
                  mma_f16_pair(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, a.idesc, acc_flag);
                } else {
                  mma_f16(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, a.idesc, acc_flag);
                }
              }
            }
            // frees the stage (in both CTAs of a pair) once these MMAs finish
            if constexpr (kPair)
              mma_commit_pair_multicast(empty_bar(stage), kPairMask);
            else
              mma_commit(empty_bar(stage));
            stage = next;
            phase = next_phase;
          }
          if (!ok) break;
          // accumulator complete (in both CTAs' TMEM for a pair)
          if constexpr (kPair)
            mma_commit_pair_multicast(accf_bar(acc), kPairMask);
          else
            mma_commit(accf_bar(acc));
          acc ^= 1;
          if (acc == 0) acc_phase ^= 1u;
        }
        // All MMAs are issued: the next kernel in the stream may start launching
        // (it runs its prologue and then waits for this grid to complete).
        grid_launch_dependents();
        // Drain: every MMA issued above completes before TMEM is released.
        if constexpr (kPair)
          mma_commit_pair_multicast(drain_bar, 0x1);
        else
          mma_commit(drain_bar);
        const uint64_t t0 = globaltimer_ns();
        while (!mbar_try_wait(drain_bar, 0) && globaltimer_ns() - t0 < a.timeout_ns) {
        }
      }
    }
  } else {
    if constexpr (C_::kRebalance) setmaxnreg_inc<C_::kRegsHigh>();
    grid_dependency_wait();
    // -------------------------------------------------------------- epilogue
    const int quarter = warp & 3;                     // TMEM lanes this warp may access
    const int col_half = (warp - C_::kEpiWarp0) >> 2;  // which interleaved column units
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    SegCursor<GROUPED> cur;
    cur.init(a, x);
    Seg sg;
    int acc = 0, nrec = 0;
    uint32_t acc_phase = 0;
    // the single GEMM's output; a grouped segment switches to its problem's
    OutView out{a.C, a.ldc, a.m, a.n, a.c_vec, a.c_tma, a.alpha, a.beta, &tmC};
    // F8: the block scales (row-major, ld_scale k-blocks per 128-row block)
    const float* scale_a = a.scale_a;
    const float* scale_b = a.scale_b;
    int32_t ld_scale = a.ld_scale;
    constexpr int kCpu = (sizeof(TC) == 4) ? 1 : 2;  // 32-column chunks per output unit
    // BLK_N = 64 with a 16-bit output has one unit (two 32-column chunks) per
    // lane quarter: the quarter's two warps take one chunk each for the TMEM
    // read, the spill and the fixup, and meet in the first warp's staging
    // buffer for the store (named barrier 2 + quarter, 64 threads).
    constexpr bool kSplit = !F8 && BN == 64 && kCpu == 2;
    float* const my_slot = a.partials + static_cast<size_t>(cta) * (kBlkM * BN);
    const uint32_t staging = base + static_cast<uint32_t>(C_::kStagingOffset +
                                                         (warp - C_::kEpiWarp0) * C_::kStagingBytesPerWarp);
    const bool tracer = a.trace != nullptr && warp == C_::kEpiWarp0 && lane == 0;
    int32_t* const tb =
        a.trace + static_cast<size_t>(cta) * (kTraceHeaderInts + a.trace_cap * kTraceRecordInts);
    if (tracer) {
      const uint64_t t = globaltimer_ns();
      tb[0] = 0;
      tb[1] = 0;
      tb[2] = static_cast<int32_t>(t & 0xffffffffu);
      tb[3] = static_cast<int32_t>(t >> 32);
    }
    while (cur.next(a, sg)) {
      const int tile = sg.tile, kb0 = sg.kb0, kb1 = sg.kb1, role = sg.role;
      // Peers as CTA indices: the same half (rank) of each contributing unit.
      int peer_first = -1, peer_last = -1;
      if (role == kRoleOwner) {
        peer_first = sg.peer_first * CM + rank;
        peer_last = sg.peer_last * CM + rank;
      }
      const int tm = sg.tm * CM + rank, tn = sg.tn;
      if constexpr (GROUPED) {
        const GroupProblem* gp = a.gprobs + sg.problem;
        out = OutView{gp->C, gp->ldc, gp->m, gp->n, gp->c_vec, gp->c_tma, gp->alpha, gp->beta, &gp->tmC};
        if (lane == 0 && out.c_tma == 1) tensormap_acquire(out.tmC);
        if constexpr (F8) {
          scale_a = gp->scale_a;
          scale_b = gp->scale_b;
          ld_scale = gp->ld_scale;
        }
      }

      bool fail = false;
      if constexpr (F8) {
        // The segment's sum over its k-blocks, in k order, of
        // scale_a[tm][kb] * scale_b[tn][kb] * (product of k-block kb), for
        // this warp's output units (the columns it stores below).
        constexpr int kMine = BN / (32 * kCpu) / 2;
        uint32_t sum[kMine][32 * kCpu];  // FP32 bit patterns
#pragma unroll
        for (int i = 0; i < kMine; ++i)
#pragma unroll
          for (int j = 0; j < 32 * kCpu; ++j) sum[i][j] = 0u;
        // A tile is kHalves blocks of 128 B rows wide, each with its own row
        // of B scales (BLK_N = 256: two; the second exists only inside n).
        constexpr int kHalves = BN / 128;
        const float* sa = scale_a + static_cast<size_t>(tm) * ld_scale;
        const float* sb = scale_b + static_cast<size_t>(tn * kHalves) * ld_scale;
        const int nblk_b = (out.n + 127) / 128;
        // The segment's k-blocks: KD per MAC-loop iteration.  Those inside k
        // (ld_scale of them per row of scales) carry scales; a stage's second
        // k-block beyond k is all zeros and gets scale 0.
        const int kq0 = kb0 * KD, kq1 = kb1 * KD;
        const int kreal = min(kq1, ld_scale);
        // lane l holds the scale product of k-block first + l (per half);
        // the next 32 are loaded one window ahead
        auto window = [&](int first, int h) {
          const int kq = first + lane;
          return kq < kreal && (kHalves == 1 || tn * kHalves + h < nblk_b)
                     ? __ldg(sa + kq) * __ldg(sb + static_cast<size_t>(h) * ld_scale + kq)
                     : 0.0f;
        };
        float s_cur[kHalves], s_nxt[kHalves];
#pragma unroll
        for (int h = 0; h < kHalves; ++h) {
          s_cur[h] = window(kq0, h);
          s_nxt[h] = kq0 + 32 < kq1 ? window(kq0 + 32, h) : 0.0f;
        }
        for (int it = kb0; it < kb1; ++it) {
          if (!wait_bar(accf_bar(acc), acc_phase, abort_flag, a, kAtEpiAccFull)) {
            fail = true;
            break;
          }
          tc_fence_after();
#pragma unroll 1
          for (int j = 0; j < KD; ++j) {
            const int kq = it * KD + j;
            const int i = kq - kq0;
            if (i > 0 && (i & 31) == 0) {
#pragma unroll
              for (int h = 0; h < kHalves; ++h) {
                s_cur[h] = s_nxt[h];
                if (kq + 32 < kq1) s_nxt[h] = window(kq + 32, h);
              }
            }
            float sc[kHalves];
#pragma unroll
            for (int h = 0; h < kHalves; ++h) sc[h] = __shfl_sync(0xffffffffu, s_cur[h], i & 31);
            const uint32_t pbase =
                tmem_base + lane_base + static_cast<uint32_t>(acc * C_::kAccCols + j * BN);
            // 32 columns at a time, so that the product needs 32 registers
            // next to the sum's BN / 2
            constexpr int kChunks = kMine * kCpu;
#pragma unroll
            for (int c = 0; c < kChunks; ++c) {
              const int mi = c / kCpu;
              const int j0 = 32 * (c % kCpu);
              const uint32_t col = static_cast<uint32_t>((col_half + 2 * mi) * 32 * kCpu + j0);
              uint32_t r[32];
              tmem_ld_x32(pbase + col, r);
              tmem_wait_ld();
              if (j == KD - 1 && c == kChunks - 1 && it + 1 < kb1) {
                // the pair is read: the MMA warp may overwrite it (the
                // segment's last pair is kept for its sum, below)
                tc_fence_before();
                __syncwarp();
                if (lane == 0) release_acc(acc);
              }
              // sum += sc * product, two columns per packed FMA; the unit's
              // columns (col_half + 2 mi) * 32 * kCpu onward lie in half
              // mi * kCpu / 2 of the tile for either col_half
              const uint32_t scb = __float_as_uint(sc[kHalves == 1 ? 0 : (mi * kCpu) / 2]);
#pragma unroll
              for (int jj = 0; jj < 32; jj += 2)
                fma2(scb, r[jj], r[jj + 1], sum[mi][j0 + jj], sum[mi][j0 + jj + 1]);
            }
          }
          if (it + 1 < kb1) {
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
          }
        }
        if (!fail) {
          // the sum goes to the first buffer of the segment's last pair (acc)
          const uint32_t sbase = tmem_base + lane_base + static_cast<uint32_t>(acc * C_::kAccCols);
#pragma unroll
          for (int mi = 0; mi < kMine; ++mi) {
            const uint32_t col = static_cast<uint32_t>((col_half + 2 * mi) * 32 * kCpu);
            if constexpr (kCpu == 2)
              tmem_st_x64(sbase + col, sum[mi]);
            else
              tmem_st_x32(sbase + col, sum[mi]);
          }
          // this thread reads back exactly the lanes and columns it wrote
          tmem_wait_st();
        }
      } else {
        fail = !wait_bar(accf_bar(acc), acc_phase, abort_flag, a, kAtEpiAccFull);
      }
      if (epi_any(fail)) break;
      tc_fence_after();
      const uint64_t t_acc = tracer ? globaltimer_ns() : 0;
      uint64_t t_fix = t_acc;

      // the accumulator (F8: the sum, in the first buffer of the segment's last pair)
      const uint32_t tbase = tmem_base + lane_base + static_cast<uint32_t>(acc * C_::kAccCols);
      const int grow = tm * kBlkM + row;
      const int col0 = tn * BN;
      // Column units of 128 output bytes (32 FP32 or 64 16-bit columns); the
      // two warps of a lane quarter take alternate units.  Only units holding
      // columns < n are read, spilled, fixed up and stored.
      const int nchunks = (min(BN, out.n - col0) + 31) / 32;
      const int nunits = (nchunks + kCpu - 1) / kCpu;
      const int my_last_unit = (nunits - 1 - col_half) >= 0 ? nunits - 1 - ((nunits - 1 - col_half) & 1) : -1;
      if constexpr (kSplit) {
        const int c = col_half;  // this warp's 32-column chunk of the unit
        const bool mine = c < nchunks;
        float v[32];
        {
          uint32_t r[32];
          if (mine) {
            tmem_ld_x32(tbase + static_cast<uint32_t>(c * 32), r);
            tmem_wait_ld();
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) release_acc(acc);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
        }
        if (role == kRolePartial) {
          if (mine) {
            float4* dst = reinterpret_cast<float4*>(my_slot) + (c * 4 + quarter) * 256 + lane;
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcg(dst + j * 32, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
            // Signal(flags[cta][quarter][c]); the warp barrier orders every
            // lane's stores before lane 0's release, which is cumulative
            __syncwarp();
            if (lane == 0 && cta != a.debug_skip_signal)
              st_release_gpu(&a.flags[cta * kFlagsPerCtaDev + quarter * 8 + c], a.epoch);
          }
        } else {
          if (role == kRoleOwner && mine) {
            for (int y = peer_first + lane * CM; y <= peer_last && !fail; y += 32 * CM)
              fail = !wait_flag(&a.flags[y * kFlagsPerCtaDev + quarter * 8 + c], abort_flag, a);
            __syncwarp();
            fail = __any_sync(0xffffffffu, fail);
            if (tracer) t_fix = globaltimer_ns();
            // acc + P[x+1] + P[x+2] + ... in increasing CTA order
            if (!fail) add_peers<CM, BN>(a.partials, peer_first, peer_last, c * 4 + quarter, lane, v);
          }
          // Every warp takes the same branch below (owners agree on failure
          // first), so the two warps of a quarter always meet at both barriers.
          if (role == kRoleOwner && epi_any(fail)) break;
          if (!out.c_tma) {
            if (mine) store_row32<TC>(out, grow, col0 + c * 32, v);
          } else {
            const float alpha = out.alpha, beta = out.beta;
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] *= alpha;
            if (beta != 0.0f && mine) add_beta_c<TC>(out, grow, col0 + c * 32, v);
            // the quarter's staging buffer: that of its first warp
            const uint32_t stage0 =
                base + static_cast<uint32_t>(C_::kStagingOffset +
                                             (warp - C_::kEpiWarp0 - 4 * col_half) * C_::kStagingBytesPerWarp);
            const uint32_t srow = stage0 + static_cast<uint32_t>(lane * 128);
            const uint32_t bar_id = 2u + static_cast<uint32_t>(quarter);
            // the previous store from the buffer has finished reading it
            if (col_half == 0 && lane == 0) bulk_wait_group_read<0>();
            named_bar_sync(bar_id, 64);
            if (mine) {
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                const int j = c * 4 + jj;  // 16-byte granule of the 128-byte row
                st_shared_v4(srow + static_cast<uint32_t>(((j ^ (lane & 7)) * 16)),
                             pack2(v[8 * jj], v[8 * jj + 1], static_cast<TC*>(nullptr)),
                             pack2(v[8 * jj + 2], v[8 * jj + 3], static_cast<TC*>(nullptr)),
                             pack2(v[8 * jj + 4], v[8 * jj + 5], static_cast<TC*>(nullptr)),
                             pack2(v[8 * jj + 6], v[8 * jj + 7], static_cast<TC*>(nullptr)));
              }
            }
            fence_proxy_async_smem();
            named_bar_sync(bar_id, 64);
            if (col_half == 0) {
              if (out.c_tma == 1) {
                if (lane == 0) {
                  tma_store_2d(out.tmC, stage0, col0, tm * kBlkM + quarter * 32);
                  bulk_commit_group();
                }
              } else {
                // the same 32 rows x 128 B through coalesced global stores
                const int chunk = lane & 7;
                const int gcol = col0 + chunk * (16 / static_cast<int>(sizeof(TC)));
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  const int r = i * 4 + (lane >> 3);
                  const int grow_r = tm * kBlkM + quarter * 32 + r;
                  uint32_t w0, w1, w2, w3;
                  ld_shared_v4(stage0 + static_cast<uint32_t>(r * 128 + ((chunk ^ (r & 7)) * 16)), w0,
                               w1, w2, w3);
                  if (grow_r < out.m) store_chunk16<TC>(out, grow_r, gcol, w0, w1, w2, w3);
                }
                __syncwarp();
              }
            }
          }
        }
      } else {
      if (my_last_unit < 0) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) release_acc(acc);
      }
#pragma unroll 1
      for (int u = col_half; u < nunits; u += 2) {
        // One TMEM load per unit (32 or 64 FP32 columns), then one wait.
        float v[kCpu][32];
        {
          uint32_t r[32 * kCpu];
          if constexpr (kCpu == 2)
            tmem_ld_x64(tbase + static_cast<uint32_t>(u * 64), r);
          else
            tmem_ld_x32(tbase + static_cast<uint32_t>(u * 32), r);
          tmem_wait_ld();
          if (u == my_last_unit) {
            // all of this warp's TMEM reads are done: hand the buffer (F8:
            // the segment's last pair) back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) release_acc(acc);
          }
#pragma unroll
          for (int cc = 0; cc < kCpu; ++cc)
#pragma unroll
            for (int j = 0; j < 32; ++j) v[cc][j] = __uint_as_float(r[cc * 32 + j]);
        }
        const int cvalid = min(kCpu, nchunks - u * kCpu);  // 32-column chunks inside n
        // Workspace slot layout: [chunk][quarter][j][lane] float4, so the 32
        // rows x 32 columns of a (chunk, quarter) are one contiguous 4 KiB block.
        if (role == kRolePartial) {
#pragma unroll
          for (int cc = 0; cc < kCpu; ++cc) {
            if (cc >= cvalid) break;
            float4* dst =
                reinterpret_cast<float4*>(my_slot) + ((u * kCpu + cc) * 4 + quarter) * 256 + lane;
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcg(dst + j * 32, make_float4(v[cc][4 * j], v[cc][4 * j + 1], v[cc][4 * j + 2],
                                               v[cc][4 * j + 3]));
          }
          // Signal(flags[cta][quarter][u]): this warp's part of the partial is
          // written.  The warp barrier orders every lane's stores before lane
          // 0's release, which is cumulative over them.
          __syncwarp();
          if (lane == 0 && cta != a.debug_skip_signal)
            st_release_gpu(&a.flags[cta * kFlagsPerCtaDev + quarter * 8 + u], a.epoch);
          continue;
        }
        if (role == kRoleOwner) {
          // Wait(flags[y][quarter][u]) for every peer y: the unit this warp
          // adds next, so the fixup overlaps the peers' remaining spills.
          // The lanes poll the peers' flags at once (lane l takes peers l,
          // l + 32, ...), one acquire round trip instead of one per peer; the
          // warp barrier then orders every lane's acquire before all lanes'
          // reads of the partials, as the peer's barrier orders its lanes'
          // stores before its release.
          for (int y = peer_first + lane * CM; y <= peer_last && !fail; y += 32 * CM)
            fail = !wait_flag(&a.flags[y * kFlagsPerCtaDev + quarter * 8 + u], abort_flag, a);
          __syncwarp();
          if (__any_sync(0xffffffffu, fail)) {
            fail = true;
            break;
          }
          if (tracer && u == col_half) t_fix = globaltimer_ns();
          // acc + P[x+1] + P[x+2] + ... in increasing CTA order
#pragma unroll
          for (int cc = 0; cc < kCpu; ++cc) {
            if (cc >= cvalid) break;
            add_peers<CM, BN>(a.partials, peer_first, peer_last, (u * kCpu + cc) * 4 + quarter, lane,
                              v[cc]);
          }
        }
        if (!out.c_tma) {
#pragma unroll
          for (int cc = 0; cc < kCpu; ++cc)
            if (cc < cvalid) store_row32<TC>(out, grow, col0 + (u * kCpu + cc) * 32, v[cc]);
          continue;
        }
        // StoreTile through a swizzled staging row and one TMA tensor store of
        // 32 rows x 128 B.
        const float alpha = out.alpha, beta = out.beta;
#pragma unroll
        for (int cc = 0; cc < kCpu; ++cc) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[cc][j] *= alpha;
          if (beta != 0.0f && cc < cvalid) add_beta_c<TC>(out, grow, col0 + (u * kCpu + cc) * 32, v[cc]);
        }
        const uint32_t srow = staging + static_cast<uint32_t>(lane * 128);
        // the previous store from this buffer has finished reading it
        if (lane == 0) bulk_wait_group_read<0>();
        __syncwarp();
        if constexpr (sizeof(TC) == 4) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            st_shared_v4(srow + static_cast<uint32_t>(((j ^ (lane & 7)) * 16)),
                         __float_as_uint(v[0][4 * j]), __float_as_uint(v[0][4 * j + 1]),
                         __float_as_uint(v[0][4 * j + 2]), __float_as_uint(v[0][4 * j + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int cc = j >> 2, jj = j & 3;
            st_shared_v4(srow + static_cast<uint32_t>(((j ^ (lane & 7)) * 16)),
                         pack2(v[cc][8 * jj], v[cc][8 * jj + 1], static_cast<TC*>(nullptr)),
                         pack2(v[cc][8 * jj + 2], v[cc][8 * jj + 3], static_cast<TC*>(nullptr)),
                         pack2(v[cc][8 * jj + 4], v[cc][8 * jj + 5], static_cast<TC*>(nullptr)),
                         pack2(v[cc][8 * jj + 6], v[cc][8 * jj + 7], static_cast<TC*>(nullptr)));
          }
        }
        if (out.c_tma == 1) {
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(out.tmC, staging, col0 + u * (32 * kCpu), tm * kBlkM + quarter * 32);
            bulk_commit_group();
          }
        } else {
          // The same 32 rows x 128 B through coalesced global stores: each
          // instruction writes four whole 128-byte row segments.
          __syncwarp();
          const int chunk = lane & 7;
          const int gcol = col0 + u * (32 * kCpu) + chunk * (16 / static_cast<int>(sizeof(TC)));
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int r = i * 4 + (lane >> 3);
            const int grow_r = tm * kBlkM + quarter * 32 + r;
            uint32_t w0, w1, w2, w3;
            ld_shared_v4(staging + static_cast<uint32_t>(r * 128 + ((chunk ^ (r & 7)) * 16)), w0, w1, w2, w3);
            if (grow_r < out.m) store_chunk16<TC>(out, grow_r, gcol, w0, w1, w2, w3);
          }
          __syncwarp();  // the staging buffer is read before the next unit overwrites it
        }
      }
      // Only owners wait inside the segment; their failure decision must be
      // the same in every epilogue warp.
      if (role == kRoleOwner && epi_any(fail)) break;
      }
      if (role == kRoleOwner && lane == 0) {
        // Every flag has exactly one consumer, this warp: clear the ones it
        // consumed so the next launch (even a graph replay carrying the same
        // epoch) starts clean.  (kSplit: one flag per chunk, this warp's.)
        if constexpr (kSplit) {
          if (col_half < nchunks)
            for (int y = peer_first; y <= peer_last; y += CM)
              a.flags[y * kFlagsPerCtaDev + quarter * 8 + col_half] = 0u;
        } else {
          for (int u = col_half; u < nunits; u += 2)
            for (int y = peer_first; y <= peer_last; y += CM)
              a.flags[y * kFlagsPerCtaDev + quarter * 8 + u] = 0u;
        }
      }
      if (tracer) {
        const uint64_t t_done = globaltimer_ns();
        if (nrec < a.trace_cap) {
          int32_t* rec = tb + kTraceHeaderInts + nrec * kTraceRecordInts;
          rec[0] = cta;
          rec[1] = tile;
          rec[2] = tm;
          rec[3] = tn;
          rec[4] = kb0;
          rec[5] = kb1;
          rec[6] = role;
          rec[7] = peer_first;
          rec[8] = peer_last;
          rec[9] = sg.problem;
          const uint64_t ts[3] = {t_acc, t_fix, t_done};
          for (int i = 0; i < 3; ++i) {
            rec[10 + 2 * i] = static_cast<int32_t>(ts[i] & 0xffffffffu);
            rec[11 + 2 * i] = static_cast<int32_t>(ts[i] >> 32);
          }
        }
        ++nrec;
        tb[0] = nrec;
      }
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
    // The staging buffers are read before the CTA's shared memory goes away;
    // the global writes themselves complete with the grid.
    if (lane == 0) bulk_wait_group_read<0>();
    __syncwarp();
  }

  __syncwarp();  // reconverge the producer / MMA warps (one lane worked)
  tc_fence_before();
  __syncthreads();
  // Neither CTA of a pair leaves while the other may still signal its
  // barriers; the issuer's drain above covers every pair MMA writing the odd
  // CTA's TMEM.
  if constexpr (kPair) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (kPair)
      tmem_dealloc_pair(tmem_base, C_::kTmemCols);
    else
      tmem_dealloc(tmem_base, C_::kTmemCols);
  }
}

}  // namespace sk
