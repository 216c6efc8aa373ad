/*
 * streamk.h -- C ABI of the GB300 (sm_103a) Stream-K GEMM library.
 *
 * The library computes the GEMM of the paper's problem statement (Stream-K,
 * Osama, Merrill, Cecka, Garland, Owens; Section 2 "Background"):
 *
 *     C = alpha * A * B + beta * C,   A: m x k,  B: k x n,  C: m x n,
 *
 * with FP16 or BF16 inputs, FP32 accumulation (including the cross-CTA fixup)
 * and an FP32, BF16 or FP16 result.  The work decomposition is the paper's:
 * the aggregate MAC-loop iterations (output tiles x k-blocks) are split evenly,
 * within one, over a persistent grid of CTAs (Algorithm 5); CTAs that finish a
 * tile they did not start spill FP32 partial sums to a workspace and signal a
 * flag; the CTA that ran the tile's k = 0 iteration waits for their flags,
 * adds their partials in increasing CTA order and stores the tile.  The two
 * hybrids of Section 5.2 ("DP + one-tile SK" and "two-tile SK + DP") and the
 * data-parallel decomposition (Algorithm 2) are the same kernel with a
 * different schedule.  The grid size of basic Stream-K is chosen by the
 * analytical model of Appendix A.1.
 *
 * Conventions for every entry point:
 *   - Every function returns an sk_status; nothing is thrown across the ABI.
 *   - "device pointer" means memory the CUDA device of the plan can address
 *     (cudaMalloc, or memory registered/mapped for it).  The caller keeps
 *     ownership of every matrix it passes.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  sk_gemm is asynchronous (stream-ordered) and returns after the
 *     launch; device-side failures are reported by sk_last_error.
 *   - A plan is not thread-safe.  It owns one fixup workspace, so it serves
 *     one launch at a time: a launch on a stream other than the one of the
 *     plan's previous launch, while that launch is still running, returns
 *     SK_ERR_BUSY and enqueues nothing (checked with an event the plan records
 *     after each launch; launches made while their stream is being captured
 *     into a CUDA graph are not tracked).  Launches on one stream are ordered
 *     by the stream and never busy.
 */
#ifndef STREAMK_H
#define STREAMK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SK_OK = 0,
  SK_ERR_INVALID = 1,     /* bad argument: sizes, null or misaligned pointer, bad leading dim */
  SK_ERR_UNSUPPORTED = 2, /* dtype / layout / mode combination this build does not implement */
  SK_ERR_CUDA = 3,        /* a CUDA runtime call failed (no device, launch failure, ...) */
  SK_ERR_TIMEOUT = 4,     /* a bounded wait on the device ran out (fixup flag or pipeline) */
  SK_ERR_NOMEM = 5,       /* device allocation failed */
  SK_ERR_DEVICE = 6,      /* the current device is not sm_103 (GB300) */
  SK_ERR_BUSY = 7         /* the plan's previous launch is still running on another stream */
} sk_status;

/* SK_E4M3: 8-bit floating point (OCP FP8 E4M3: 1 sign, 4 exponent bits with
 * bias 7, 3 mantissa bits, no infinities, 0x7F / 0xFF NaN, largest finite
 * 448), used as A and B with one FP32 scale per 128 x 128 block of each
 * operand (sk_gemm_scaled). */
typedef enum { SK_F16 = 0, SK_BF16 = 1, SK_F32 = 2, SK_E4M3 = 3 } sk_dtype;

/* Storage order of a matrix.  For A (m x k): ROW_MAJOR = k contiguous;
 * for B (k x n): COL_MAJOR = k contiguous; for C (m x n): ROW_MAJOR = n
 * contiguous.  Supported: A row-major with B column-major (both K-contiguous),
 * C row-major or column-major. */
typedef enum { SK_ROW_MAJOR = 0, SK_COL_MAJOR = 1 } sk_layout;

/* Work decomposition (Sections 3-5 of the paper). */
typedef enum {
  SK_MODE_AUTO = 0,            /* two-tile hybrid when t >= p, DP on a perfect wave count,
                                  basic Stream-K with the modelled grid below one wave */
  SK_MODE_DP = 1,              /* Algorithm 2: one CTA per tile (persistent waves) */
  SK_MODE_SK = 2,              /* Algorithm 5: basic Stream-K over all tiles */
  SK_MODE_HYBRID = 3,          /* Section 5.2: "two-tile Stream-K + data-parallel" */
  SK_MODE_HYBRID_ONE_TILE = 4  /* Section 5.2: "data-parallel + one-tile Stream-K" */
} sk_mode;

/* Plan attributes (sk_plan_set / sk_plan_get).  Settable ones re-plan. */
typedef enum {
  SK_ATTR_TILE_N = 1,        /* set/get: BLK_N, 64, 128 or 256; set 0 for automatic.  64
                                (128 x 64 tiles, single CTAs only) gives shapes with few
                                tiles more of them, so fewer CTAs share each tile */
  SK_ATTR_GRID = 2,          /* set: grid size g (in cluster units) for SK_MODE_SK (0 = model);
                                get: the g in use */
  SK_ATTR_RASTER_GROUP = 3,  /* set/get: tile-raster band height in tiles (0 = automatic) */
  SK_ATTR_TIMEOUT_NS = 4,    /* set/get: limit of every device-side wait, nanoseconds */
  SK_ATTR_LDA = 5,           /* set/get: leading dimension of A in elements (default dense) */
  SK_ATTR_LDB = 6,           /* set/get: leading dimension of B in elements */
  SK_ATTR_LDC = 7,           /* set/get: leading dimension of C in elements */
  SK_ATTR_DEBUG_SKIP_SIGNAL = 8, /* set: a CTA index that withholds its fixup Signal, so the
                                    owner's bounded Wait must expire (failure-detection
                                    tests); -1 = off */
  SK_ATTR_CLUSTER_M = 10,    /* set/get: CTAs per cluster along M, 1 or 2 (0 = automatic);
                                with 2, a tcgen05 CTA pair computes each 256-row tile with
                                two-SM MMAs, each CTA holding half of the B tile */
  SK_ATTR_STORE = 11,        /* set/get: how the epilogue writes C when C's rows are 16-byte
                                aligned: 0 = automatic, 1 = TMA tensor stores, 2 = coalesced
                                global stores from the same staging buffer.  Unaligned C is
                                always written row by row. */
  SK_ATTR_PDL = 9,           /* set/get: 1 (default) = launch with programmatic dependent
                                launch, so the kernel's set-up overlaps the previous kernel
                                in the stream; it touches global memory only after that
                                kernel has completed.  0 = plain stream serialisation. */
  SK_ATTR_INDEPENDENT_INPUTS = 12, /* set/get: 0 (default) or 1.  1 declares that no kernel
                                earlier in the launch's stream writes A, B (or the scales)
                                while it may still run, e.g. a stream of independent GEMMs.
                                With SK_ATTR_PDL 1 the launch then loads A and B and runs its
                                MAC loop while the previous kernel of the stream finishes; its
                                reads and writes of C and of the fixup workspace still wait for
                                that kernel to complete, so C and the workspace keep stream
                                order.  A wrong declaration (a preceding kernel still writing
                                A or B) gives wrong results.  No effect with SK_ATTR_PDL 0. */
  SK_ATTR_STAGES = 13,       /* set/get: pipeline stages of the shared-memory operand ring
                                the MAC loop cycles through: 0 (set) = all the ring holds
                                (get returns the count in use), else 2 .. that count;
                                single and grouped plans; the autotuners choose it */
  SK_ATTR_MODE = 20,         /* get: resolved sk_mode */
  SK_ATTR_TILE_M = 21,       /* get: BLK_M (128) */
  SK_ATTR_TILE_K = 22,       /* get: BLK_K, the depth of one MAC-loop iteration (128 for
                                BLK_N = 64 and 128, 64 for BLK_N = 256) */
  SK_ATTR_TILES_M = 23,      /* get: ceil(m / BLK_M) */
  SK_ATTR_TILES_N = 24,      /* get: ceil(n / BLK_N) */
  SK_ATTR_TILES = 25,        /* get: t */
  SK_ATTR_ITERS_PER_TILE = 26, /* get: ceil(k / BLK_K) */
  SK_ATTR_SK_TILES = 27,     /* get: tiles in the Stream-K region */
  SK_ATTR_DP_TILES = 28,     /* get: tiles in the data-parallel region */
  SK_ATTR_WORKSPACE_BYTES = 29, /* get: device workspace this plan needs (partials + flags) */
  SK_ATTR_NUM_SMS = 30,      /* get: SM count p of the plan's device */
  SK_ATTR_TRACE_INTS = 31,   /* get: int32 entries sk_gemm_traced needs */
  SK_ATTR_TRACE_CAP = 32,    /* get: trace records per CTA */
  SK_ATTR_CTAS = 33,         /* get: CTAs launched (grid * cluster_m) */
  SK_ATTR_SEGMENTS = 34      /* get (grouped plans): segments of the schedule */
} sk_attr;

typedef struct sk_plan_s* sk_plan_t;
typedef struct sk_grouped_s* sk_grouped_t;
typedef struct sk_server_s* sk_server_t;

/* Host-only description of a schedule (sk_plan_describe).  The schedule's
 * unit is a cluster of cluster_m CTAs computing a tile_m x tile_n tile
 * (tile_m = 128 * cluster_m); tiles, grid and the regions count such units,
 * the paper's p being the SM count divided by cluster_m. */
typedef struct {
  int32_t mode;            /* resolved sk_mode */
  int32_t tile_m, tile_n, tile_k;
  int32_t tiles_m, tiles_n;
  int64_t tiles;           /* t */
  int32_t iters_per_tile;  /* ceil(k / BLK_K) */
  int32_t grid;            /* g, CTAs of the persistent launch */
  int64_t sk_tiles;        /* Stream-K region: tiles [0, sk_tiles) */
  int64_t dp_tiles;        /* data-parallel region: tiles [sk_tiles, t) */
  int64_t sk_iters;        /* sk_tiles * iters_per_tile */
  int32_t raster_group;    /* tile raster band height */
  int32_t max_segments;    /* most tile segments any CTA processes */
  int64_t workspace_bytes; /* flags + one 128 x BLK_N FP32 partial slot per CTA, 0 when no split */
  int32_t cluster_m;       /* CTAs per unit along M: 1, or 2 (a pair shares the B tile) */
  int32_t ctas;            /* CTAs launched: grid * cluster_m */
} sk_schedule_info;

/*
 * Create a plan for one GEMM shape on the current CUDA device.
 *   m, n, k   >= 0 (m*n == 0: sk_gemm is a no-op; k == 0: C = beta*C).
 *   a_type == b_type in {SK_F16, SK_BF16, SK_E4M3}; c_type in {SK_F32, SK_BF16,
 *   SK_F16}; compute_type must be SK_F32 (FP32 accumulation, Section 6).
 *   E4M3 plans run 128 x 128 or 128 x 256 tiles on single CTAs, the width
 *   chosen by the planner's model unless SK_ATTR_TILE_N fixes it (128 or 256;
 *   64 is SK_ERR_UNSUPPORTED); SK_ATTR_CLUSTER_M 0 and 1 mean single CTAs, 2
 *   selects CTA pairs of 256 x 128 tiles (width 128 only: 256 with pairs is
 *   SK_ERR_UNSUPPORTED).  They are launched with sk_gemm_scaled.
 *   a_layout SK_ROW_MAJOR, b_layout SK_COL_MAJOR, c_layout either.
 *   mode: an sk_mode.
 * Allocates the plan's device workspace (fixup partials and flags, Algorithm 5
 * "partials" and "flags") and a status word; the plan owns them until
 * sk_plan_destroy.  On error *out is set to NULL.
 */
int sk_plan(sk_plan_t* out, int64_t m, int64_t n, int64_t k, sk_dtype a_type, sk_dtype b_type,
            sk_dtype c_type, sk_dtype compute_type, sk_layout a_layout, sk_layout b_layout,
            sk_layout c_layout, int mode);

/*
 * C = alpha * A * B + beta * C on `stream` (paper, Section 2).
 *   A, B: device pointers, 16-byte aligned, in the plan's layouts and leading
 *   dimensions (each leading dimension times the element size a multiple of
 *   16 bytes).  C: device pointer, 16-byte aligned; read only if beta != 0.
 *   C may not alias A or B.
 * The launch is persistent (g <= SM count CTAs).  When the schedule splits
 * tiles (SK_ATTR_WORKSPACE_BYTES > 0) its CTAs wait on one another, which
 * needs all of them resident at once: single-CTA plans ask for it with the
 * cooperative attribute, CTA-pair plans rely on SMs freeing up, which holds
 * within one stream.  Across streams it does not: two split launches running
 * at the same time can each hold SMs the other's waiting CTAs need (measured,
 * with cooperative launches as well), and a programmatic-dependent launch
 * takes SMs before its stream's previous kernel has finished.  A wait then
 * runs out and the launch reports SK_ERR_TIMEOUT.  Callers running plans on
 * several streams should order split launches so that one runs at a time
 * (the serving loop chains them through an event) and set SK_ATTR_PDL 0 and
 * SK_ATTR_CLUSTER_M 1 on those plans.  Results are bitwise reproducible
 * run to run for a given plan: the fixup adds the contributing CTAs' partials
 * in increasing CTA order.  Returns SK_ERR_INVALID for bad pointers,
 * SK_ERR_BUSY when the plan's previous launch still runs on another stream,
 * SK_ERR_CUDA if the launch fails.
 */
int sk_gemm(sk_plan_t plan, const void* A, const void* B, void* C, float alpha, float beta,
            void* stream);

/*
 * Block-scaled E4M3 GEMM on an SK_E4M3 plan:
 *   C = alpha * sum_kb Sa[i/128][kb] * Sb[j/128][kb] * (A_kb * B_kb)[i][j] + beta * C
 * where kb runs over the k-blocks of 128 (the last one ragged), A_kb is
 * columns [128 kb, 128 kb + 128) of A (E4M3 bytes, row-major m x k) and B_kb
 * rows of B (E4M3, column-major k x n, i.e. an n x k row-major array).
 * Every product of a k-block is accumulated in FP32 by the tensor cores, then
 * scaled and summed in FP32 in k order; Stream-K partials and the fixup stay
 * FP32 (the paper's Section 4 schedule is unchanged: one MAC-loop iteration
 * is two k-blocks of 128, BLK_K = 256).
 *   scale_a: device FP32 array [ceil(m/128)][ceil(k/128)], row-major;
 *   scale_b: device FP32 array [ceil(n/128)][ceil(k/128)], row-major; both
 *   read-only, 4-byte aligned, not copied (they must stay valid until the
 *   launch completes).  A, B, C as for sk_gemm (k a multiple of 16 so that
 *   the dense rows are 16-byte multiples).
 * Returns SK_ERR_INVALID for a null scale pointer or a plan whose inputs are
 * not E4M3; sk_gemm on an E4M3 plan also returns SK_ERR_INVALID.
 */
int sk_gemm_scaled(sk_plan_t plan, const void* A, const void* B, const float* scale_a,
                   const float* scale_b, void* C, float alpha, float beta, void* stream);

/*
 * sk_gemm that also records the schedule each CTA executed, with device
 * timestamps.  For CTA x the trace holds, at trace[x * (4 + cap * 16)], a
 * header of 4 int32 (record count, reserved, then the global timer in ns at
 * the CTA's start as a little-endian u64) followed by records of 16 int32:
 * (cta, tile_idx, tm, tn, local_iter, local_iter_end, role, peer_first,
 * peer_last, reserved) and three u64 global-timer stamps in ns (accumulator
 * ready, fixup waits done, tile stored or partials signalled).  role 0 = whole
 * tile stored, 1 = partials spilled and signalled, 2 = owner that waited for
 * peers peer_first .. peer_last (-1 when none).  cap = SK_ATTR_TRACE_CAP;
 * `trace` is a device buffer of SK_ATTR_TRACE_INTS int32 owned by the caller.
 */
int sk_gemm_traced(sk_plan_t plan, const void* A, const void* B, void* C, float alpha,
                   float beta, int32_t* trace, int64_t trace_ints, void* stream);

/*
 * Wait for the plan's last launch (synchronises its stream), then report and
 * clear the device status: returns SK_OK or SK_ERR_TIMEOUT (also SK_ERR_CUDA
 * if the stream reports a CUDA error).  *device_status (may be NULL) receives
 * the raw device code: 0 ok, 1 pipeline wait expired, 2 fixup-flag wait
 * expired, 3 aborted after another CTA failed.
 */
int sk_last_error(sk_plan_t plan, int* device_status);

/* Release the plan and the device memory it owns.  NULL is accepted. */
int sk_plan_destroy(sk_plan_t plan);

/* Set / get an sk_attr.  Setting a schedule attribute re-plans; the
 * workspace is reallocated when it must grow. */
int sk_plan_set(sk_plan_t plan, int attr, int64_t value);
int sk_plan_get(sk_plan_t plan, int attr, int64_t* value);

/*
 * Use caller-owned device memory as the plan's workspace (for example one
 * buffer shared by many plans that run one after another on one stream).
 * `bytes` must be at least SK_ATTR_WORKSPACE_BYTES and `ws` 256-byte aligned.
 * The flag area is zeroed here (synchronously).  The plan frees its own
 * workspace and never frees `ws`.
 */
int sk_plan_attach_workspace(sk_plan_t plan, void* ws, size_t bytes);

/*
 * Host-only planning, no GPU needed: the schedule sk_plan would choose for
 * this shape on a device with `num_sms` SMs.  tile_n / grid / raster_group /
 * cluster_m as the attributes above (0 = automatic).
 */
int sk_plan_describe(int64_t m, int64_t n, int64_t k, int mode, int tile_n, int grid,
                     int raster_group, int cluster_m, int num_sms, sk_schedule_info* out);

/*
 * The grid-size model of Appendix A.1, host only: the g in [1, p] minimising
 *   time_CTA(g) = a + b*[FixupPeers(g) > 1] + c*ItersPerCta(g) + d*(FixupPeers(g) - 1),
 *   ItersPerCta(g) = ceil(ceil(m/bm) * ceil(n/bn) * ceil(k/bk) / g),
 *   FixupPeers(g) = ceil(ceil(k/bk) / ItersPerCta(g)),
 * ties to the smallest g.  coef = {a, b, c, d}.
 */
int sk_grid_model(int64_t m, int64_t n, int64_t k, int bm, int bn, int bk, int p,
                  const double coef[4], int* g_out);

/*
 * The planner's time model, host only (the model SK_MODE_AUTO ranks its
 * candidates by; Appendix A.1 extended by two terms), for recalibration.
 * coef = {a, b, c, d, e, f} in microseconds: Appendix A.1's fixed cost a,
 * split cost b, per-iteration cost c and per-peer fixup cost d, then e per
 * tile segment and f, the shortest period of consecutive whole tiles.
 *
 * sk_model_coefficients: the built-in terms of one tile configuration
 * (tile_n 64, 128 or 256; cluster_m 1 or 2, 64 with 1 only), else
 * SK_ERR_UNSUPPORTED.
 *
 * sk_model_time: the modelled time of the schedule `s` (as sk_plan_describe
 * returns it) under the terms `coef`: a + b*[split] + c * (iterations of the
 * busiest unit's Stream-K share outside whole tiles) + max(c*ipt, f) * (its
 * whole tiles, data-parallel ones included) + d * (peers - 1)*[split] +
 * e * (its tile segments).  SK_ERR_INVALID for null pointers or a schedule
 * with no units.
 */
int sk_model_coefficients(int tile_n, int cluster_m, double coef[6]);
int sk_model_time(const sk_schedule_info* s, const double coef[6], double* us);

/*
 * Allocation-free GEMM: C = alpha * A * B + beta * C like sk_gemm, for callers
 * that cannot allocate device memory -- for example plugins and custom
 * operators that only receive buffers from a host framework which owns the
 * device memory pool (an allocation behind its back can fail against the
 * pool's reservation), latency-critical serving loops in which a cudaMalloc
 * would synchronise the device and stall every stream, and processes held to
 * a fixed device-memory quota.  The paper has no counterpart; it is an
 * interface of this library only.
 *
 * No plan, no cudaMalloc/cudaFree and no allocating library call: the
 * schedule is planned on the host stack for this call, with BLK_N = 128, and
 * the fixup scratch (128 KiB of flags, status words and up to 12 MiB - 132 KiB
 * of FP32 partial tiles) is one fixed 12 MiB device array inside the library,
 * which every GPU that loads the library keeps until the process exits.  The
 * scratch holds the partial tiles of 189 CTAs; a launch never has more CTAs
 * than the device has SMs (152 on GB300), so every shape fits on sm_103.  The
 * size check stays as a guard and would return SK_ERR_INVALID.  All argument
 * checks run before anything is enqueued: a call that returns an error has
 * put nothing on the stream.
 *
 *   A: m x k row-major, lda >= k; B: k x n column-major (an n x k row-major
 *   array), ldb >= k; both device pointers 16-byte aligned with lda*2 and
 *   ldb*2 multiples of 16.  C: m x n row-major, ldc >= n, 16-byte aligned.
 *   ab_type: SK_F16 or SK_BF16; c_type: SK_F32, SK_BF16 or SK_F16.
 *   mode: an sk_mode.
 *   device_status: NULL, or a 4-byte-aligned device int32 that receives, in
 *   stream order after the kernel, the device status of this call (codes as
 *   in sk_last_error: 0 ok, 1/2 a bounded wait expired, 3 aborted).
 *
 * The first call on a device sets that device up (it looks up the scratch
 * array's device address and the kernel attributes); make that first call
 * before any stream capture on the device.  Every call on a device shares the
 * one scratch array and leaves its contents behind; each call clears the
 * parts that must start at zero.  Calls whose kernels overlap on the GPU
 * (other streams, other threads) race on the scratch: serialise them.
 */
int sk_gemm_noalloc(int64_t m, int64_t n, int64_t k, sk_dtype ab_type, sk_dtype c_type,
                    const void* A, int64_t lda, const void* B, int64_t ldb, void* C,
                    int64_t ldc, float alpha, float beta, int mode, int32_t* device_status,
                    void* stream);

/* Human-readable name of an sk_status. */
const char* sk_status_string(int status);

/* ---------------------------------------------------------------- grouped GEMM
 * Stream-K across a group of independent problems in one persistent launch
 * (the paper's Conclusion, Section 7, names other GEMM-like workloads that
 * suffer the same quantization as future work).  The problems' MAC-loop
 * iterations are laid end to end, problem after problem and tile after tile
 * in each problem's raster, and that single iteration space is scheduled like
 * one GEMM's: Algorithm 5's within-one split over g CTAs, the two-tile hybrid
 * of Section 5.2 over the concatenated tile list, or data-parallel waves.
 * Problem i is C_i = alpha_i * A_i * B_i + beta_i * C_i with A_i row-major
 * m_i x k_i, B_i column-major k_i x n_i (an n_i x k_i row-major array), C_i
 * row-major m_i x n_i, all dense, one input type and one output type for the
 * group, FP32 accumulation.  All problems use one tile configuration: one
 * tile width (BLK_N) and single CTAs or, for 16-bit groups with BLK_N 128
 * or 256, CTA pairs computing 256-row tiles (SK_ATTR_CLUSTER_M).  With
 * pairs the schedule's unit is the pair: SK_ATTR_GRID and the records of
 * sk_grouped_schedule count units (CTA 2x + r, r = 0, 1, runs unit x's
 * segments on 128-row block 2 tm + r of each tile).
 *
 * sk_grouped_plan: count >= 1 problems, m/n/k host arrays of count entries
 *   (each >= 1, k a multiple of 8 so that dense 16-bit rows are 16-byte
 *   multiples as TMA requires; 16 for E4M3); mode SK_MODE_AUTO (the model picks
 *   data-parallel, the two-tile hybrid or basic Stream-K, and the tile width),
 *   SK_MODE_DP, SK_MODE_SK or SK_MODE_HYBRID; the model also picks the
 *   cluster size (E4M3 groups: single CTAs).  The plan owns its device walk
 *   table (64 bytes per problem and 8 per CTA, from which each CTA derives its
 *   segments), problem table, workspace and status words.
 *   Returns SK_ERR_INVALID / SK_ERR_UNSUPPORTED for bad arguments,
 *   SK_ERR_DEVICE off sm_103a, SK_ERR_CUDA / SK_ERR_NOMEM on allocation.
 * sk_grouped_gemm: A, B, C are host arrays of count device pointers (16-byte
 *   aligned); alpha / beta host arrays of count values or NULL (1 and 0).
 *   Asynchronous on `stream`; tensor maps are re-encoded, and the problem
 *   table re-uploaded, only for problems whose pointers or scalars changed
 *   since the previous launch (the upload is stream-ordered).  A launch on
 *   another stream while the plan's previous launch still runs returns
 *   SK_ERR_BUSY, as for sk_gemm.
 * sk_grouped_gemm_traced: as sk_grouped_gemm, recording the schedule as
 *   sk_gemm_traced does (field 9 of each record holds the problem index);
 *   trace_ints >= SK_ATTR_TRACE_INTS.
 * sk_grouped_last_error: as sk_last_error.
 * sk_grouped_set: SK_ATTR_TILE_N, SK_ATTR_GRID, SK_ATTR_MODE,
 *   SK_ATTR_CLUSTER_M (replan), SK_ATTR_TIMEOUT_NS, SK_ATTR_PDL, SK_ATTR_STORE,
 *   SK_ATTR_STAGES.
 * sk_grouped_get: SK_ATTR_MODE, TILE_M, TILE_N, TILE_K, GRID, CTAS, TILES,
 *   SK_TILES, DP_TILES, WORKSPACE_BYTES, NUM_SMS, TRACE_CAP, TRACE_INTS,
 *   TIMEOUT_NS, PDL, STORE, SEGMENTS, STAGES, CLUSTER_M.
 * sk_grouped_schedule: the host copy of the schedule, 10 int32 per segment
 *   (cta, problem, tile, tm, tn, kb0, kb1, role, peer_first, peer_last), CTA
 *   by CTA in processing order; *count receives the number of segments; with
 *   records == NULL only the count is returned; capacity in int32.
 */
int sk_grouped_plan(sk_grouped_t* out, int count, const int64_t* m, const int64_t* n,
                    const int64_t* k, sk_dtype ab_type, sk_dtype c_type, int mode);
int sk_grouped_gemm(sk_grouped_t plan, const void* const* A, const void* const* B,
                    void* const* C, const float* alpha, const float* beta, void* stream);
/* sk_grouped_gemm for an SK_E4M3 group (ab_type SK_E4M3: 128 x 128 x 128
 * tiles by default, 128 x 256 x 128 after SK_ATTR_TILE_N 256, single CTAs;
 * k_i a multiple of 16): SA / SB are host arrays of count device
 * pointers to each problem's block scales, laid out as for sk_gemm_scaled
 * ([ceil(m_i/128)][ceil(k_i/128)] and [ceil(n_i/128)][ceil(k_i/128)] FP32,
 * row-major).  sk_grouped_gemm on an E4M3 group, or this call on a 16-bit
 * group, returns SK_ERR_INVALID. */
int sk_grouped_gemm_scaled(sk_grouped_t plan, const void* const* A, const void* const* B,
                           const float* const* SA, const float* const* SB, void* const* C,
                           const float* alpha, const float* beta, void* stream);
int sk_grouped_gemm_traced(sk_grouped_t plan, const void* const* A, const void* const* B,
                           void* const* C, const float* alpha, const float* beta, int32_t* trace,
                           int64_t trace_ints, void* stream);
int sk_grouped_last_error(sk_grouped_t plan, int* device_status);
int sk_grouped_set(sk_grouped_t plan, int attr, int64_t value);
int sk_grouped_get(sk_grouped_t plan, int attr, int64_t* value);
int sk_grouped_schedule(sk_grouped_t plan, int32_t* records, int64_t capacity, int64_t* count);
int sk_grouped_destroy(sk_grouped_t plan);
/* Host-only planning of a grouped launch for num_sms SMs (no device needed):
 * summary receives 9 int64 (mode, tile_n, tile_k, grid, tiles, sk_tiles,
 * workspace_bytes, max_segments, cluster_m) when non-NULL; records and *nrec
 * as in sk_grouped_schedule.  tile_n 0 / grid 0 / cluster_m 0 = automatic. */
int sk_grouped_plan_describe(int count, const int64_t* m, const int64_t* n, const int64_t* k,
                             int mode, int tile_n, int grid, int num_sms, int cluster_m,
                             int64_t* summary, int32_t* records, int64_t capacity, int64_t* nrec);

/* ---------------------------------------------------------------- autotuning
 * Measured choice among the configurations the planner would otherwise pick
 * by its model: every tile width (64, 128, 256 when n > 128) x cluster size
 * (1, 2 when m > 128 and the tile is at least 128 wide; E4M3: 1) x
 * schedule (data-parallel, two-tile hybrid, basic Stream-K with the model's
 * grid size) x pipeline depth (the full ring, 3 and 2 stages) is planned,
 * launched once untimed and `reps` times timed with CUDA events on `stream`,
 * and the fastest is kept as the plan's fixed configuration (later
 * sk_plan_get shows it).  C is overwritten with A*B (alpha 1, beta 0) by the timing launches;
 * *best_us (when non-NULL) receives the kept configuration's mean time per
 * launch.  Synchronous.  Candidates that cannot be planned (an attached
 * workspace too small for them) are skipped.  Returns SK_ERR_CUDA when no
 * candidate ran. */
int sk_plan_autotune(sk_plan_t plan, const void* A, const void* B, void* C, int reps, void* stream,
                     double* best_us);
int sk_grouped_autotune(sk_grouped_t plan, const void* const* A, const void* const* B,
                        void* const* C, int reps, void* stream, double* best_us);
/* The same for E4M3 plans (tile widths 128, on single CTAs or pairs, and 256
 * on single CTAs; E4M3 groups: 128 and 256 on single CTAs), with the block
 * scales of sk_gemm_scaled / sk_grouped_gemm_scaled. */
int sk_plan_autotune_scaled(sk_plan_t plan, const void* A, const void* B, const float* scale_a,
                            const float* scale_b, void* C, int reps, void* stream, double* best_us);
int sk_grouped_autotune_scaled(sk_grouped_t plan, const void* const* A, const void* const* B,
                               const float* const* SA, const float* const* SB, void* const* C,
                               int reps, void* stream, double* best_us);

/* ---------------------------------------------------------------- serving loop
 * Continuous batching over the grouped launch.  Requests (independent GEMMs,
 * layouts and rules as for grouped problems, device pointers owned by the
 * caller and left untouched until the request completes) are queued on
 * submission.  A worker thread admits queued requests, oldest first, into a
 * free launch slot: at most max_batch requests per batch, all of one input
 * type (the server's 16-bit type, or E4M3 for sk_server_submit_scaled), and
 * while the operand bytes (size(A) + size(B) + mn * sizeof(C)) of all
 * admitted, unfinished requests stay within hbm_budget_bytes (a lone request
 * is always admitted).  Requests are batched only under backlog: while there
 * are at least as many free slots as queued requests, each runs alone.  A
 * lone request is one single-GEMM launch from a plan cached per shape and
 * input type (at most 256 plans), on one stream shared by all lone requests,
 * in arrival order.  A request with at least one wave of 128 x 128 tiles (the
 * SM count) always runs alone that way: it fills the GPU by itself, and its
 * own plan keeps its configuration (CTA pairs, 256-wide tiles).  Requests
 * below a wave are packed: a batch is one grouped launch on its slot's own
 * stream, data-parallel waves over all its problems' tiles; the device derives
 * each CTA's tiles from a per-problem walk table, so planning a batch costs
 * O(batch + SMs) on the host.  Launches of
 * different slots overlap on the device, except that a launch whose schedule
 * splits tiles runs alone (it waits for all work in flight and later
 * launches wait for it).  A failing launch reports through a mapped pinned
 * word, so completion needs no copy back.  Problem and walk tables and fixup
 * workspaces live on the device, preallocated per slot.
 *
 * sk_server_create: slots 1..8 concurrent batches, max_batch 1..4096.
 * sk_server_submit: queue one request; *ticket identifies it.  k must be a
 *   multiple of 8; pointers 16-byte aligned.
 * sk_server_submit_scaled: queue one E4M3 request with block scales as for
 *   sk_gemm_scaled (k a multiple of 16, scales 4-byte aligned).
 * sk_server_poll: *state 0 queued, 1 running, 2 done (then *latency_us is
 *   submission-to-completion and the ticket is retired; the return value is
 *   the request's status).
 * sk_server_wait: block until the request is done; returns its status.
 * sk_server_stats: 6 int64: submitted, completed, batches launched, largest
 *   batch, problems launched, queued now.
 * sk_server_destroy: drain the queue, wait for every batch, free. */
int sk_server_create(sk_server_t* out, sk_dtype ab_type, sk_dtype c_type, int max_batch, int slots,
                     int64_t hbm_budget_bytes);
int sk_server_submit(sk_server_t server, int64_t m, int64_t n, int64_t k, const void* A,
                     const void* B, void* C, float alpha, float beta, uint64_t* ticket);
int sk_server_submit_scaled(sk_server_t server, int64_t m, int64_t n, int64_t k, const void* A,
                            const void* B, const float* scale_a, const float* scale_b, void* C,
                            float alpha, float beta, uint64_t* ticket);
int sk_server_poll(sk_server_t server, uint64_t ticket, int* state, double* latency_us);
int sk_server_wait(sk_server_t server, uint64_t ticket, double* latency_us);
int sk_server_stats(sk_server_t server, int64_t* stats);
int sk_server_destroy(sk_server_t server);

#ifdef __cplusplus
}
#endif

#endif /* STREAMK_H */
