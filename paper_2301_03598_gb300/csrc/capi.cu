// C ABI of the Stream-K GEMM library (declared in include/streamk.h): plan
// objects, device workspace ownership, TMA descriptors, launches and status.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/streamk.h"
#include "launch.h"
#include "planner.h"
#include "host_util.h"
#include "sk_args.h"

using namespace sk::host;

namespace {


// C = beta * C for k == 0 (no MAC-loop iterations).
template <typename TC>
__global__ void scale_kernel(TC* C, int64_t m, int64_t n, int64_t ldc, float beta) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    TC* p = C + i * ldc + j;
    float v = 0.0f;
    if (beta != 0.0f) {
      if constexpr (sizeof(TC) == 4)
        v = beta * static_cast<float>(*p);
      else if constexpr (std::is_same<TC, __nv_bfloat16>::value)
        v = beta * __bfloat162float(*p);
      else
        v = beta * __half2float(*p);
    }
    if constexpr (sizeof(TC) == 4)
      *p = v;
    else if constexpr (std::is_same<TC, __nv_bfloat16>::value)
      *p = __float2bfloat16_rn(v);
    else
      *p = __float2half_rn(v);
  }
}

}  // namespace

struct sk_plan_s {
  // problem as the caller stated it
  int64_t m, n, k;
  int a_type, b_type, c_type;
  int a_layout, b_layout, c_layout;
  int mode_req;
  int tile_n_req = 0, grid_req = 0, group_req = 0, cluster_req = 0;
  int64_t lda, ldb, ldc;
  // problem as the kernel runs it (C column-major runs C^T = B^T A^T)
  bool swap = false;
  // device
  int device = 0;
  int num_sms = 0;
  size_t smem_bytes = 0;
  sk_schedule_info info{};
  // device memory
  char* ws = nullptr;  // partials then flags
  size_t ws_bytes = 0;
  bool ws_owned = true;
  int32_t* err = nullptr;  // 4 words, see SkArgs::err
  // knobs
  uint64_t timeout_ns = kDefaultTimeoutNs;
  int debug_skip_signal = -1;
  bool pdl = true;
  bool early = false;  // SK_ATTR_INDEPENDENT_INPUTS
  int stages_req = 0;  // SK_ATTR_STAGES (0: all the ring holds)
  int store_req = 0;  // SK_ATTR_STORE
  // TMA descriptor cache
  const void* cached_a = nullptr;
  const void* cached_b = nullptr;
  const void* cached_c = nullptr;
  CUtensorMap tm_a{}, tm_b{}, tm_c{};
  CUtensorMap tm_a3{}, tm_b3{};  // 3-D views (two k-blocks per box) for BLK_K = 128 plans
  bool c_tma = false;
  cudaStream_t last_stream = nullptr;
  bool launched = false;
  InFlight inflight;  // the last launch, for SK_ERR_BUSY
};

namespace {

// Run the planner for the plan's (possibly swapped) shape and make sure the
// workspace is large enough.
int replan(sk_plan_s* p) {
  const int64_t m = p->swap ? p->n : p->m;
  const int64_t n = p->swap ? p->m : p->n;
  sk_schedule_info s;
  // An E4M3 row of k elements is, byte for byte, a 16-bit row of k/2: the
  // schedule and the TMA boxes are the 16-bit path's for k/2.
  // E4M3's automatic width ranks 128 and 256 on single CTAs (256-wide E4M3
  // tiles have no CTA-pair kernel, so pairs take 128).
  const bool f8 = p->a_type == SK_E4M3;
  const int tile_n = f8 && p->tile_n_req == 0 && p->cluster_req == 2 ? 128 : p->tile_n_req;
  int st = sk::describe(m, n, f8 ? p->k / 2 : p->k, p->mode_req, tile_n, p->grid_req, p->group_req,
                        f8 && p->cluster_req == 0 ? 1 : p->cluster_req, p->num_sms, &s,
                        f8 ? 128 : 64);
  if (st != SK_OK) return st;
  if (s.workspace_bytes > 0 && static_cast<size_t>(s.workspace_bytes) > p->ws_bytes) {
    if (!p->ws_owned) return SK_ERR_INVALID;  // attached buffer too small for the new schedule
    if (p->ws) cudaFree(p->ws);
    p->ws = nullptr;
    p->ws_bytes = 0;
    void* w = nullptr;
    cudaError_t e = cudaMalloc(&w, static_cast<size_t>(s.workspace_bytes));
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemset(w, 0, static_cast<size_t>(s.workspace_bytes));
    if (e != cudaSuccess) {
      cudaFree(w);
      return cuda_status(e);
    }
    p->ws = static_cast<char*>(w);
    p->ws_bytes = static_cast<size_t>(s.workspace_bytes);
  }
  if (f8) s.tile_k *= 2;  // in E4M3 elements
  p->info = s;
  p->cached_a = p->cached_b = p->cached_c = nullptr;
  return SK_OK;
}

// The walk's precomputed divisors (see FastDiv in sk_args.h).
void set_divisors(sk::SkArgs& a, const sk_schedule_info& s) {
  const int32_t group = std::max(1, s.raster_group);
  const int32_t nbands = (s.tiles_m + group - 1) / group;
  const int32_t rows_last = std::max(1, s.tiles_m - (nbands - 1) * group);
  a.div_ipt = sk::make_fastdiv(static_cast<uint32_t>(std::max(1, s.iters_per_tile)));
  a.div_q1 = sk::make_fastdiv(static_cast<uint32_t>(a.sk_q + 1));
  a.div_q = sk::make_fastdiv(static_cast<uint32_t>(std::max(1, a.sk_q)));
  a.div_band = sk::make_fastdiv(static_cast<uint32_t>(std::max<int64_t>(1, int64_t(group) * s.tiles_n)));
  a.div_rows = sk::make_fastdiv(static_cast<uint32_t>(group));
  a.div_rows_last = sk::make_fastdiv(static_cast<uint32_t>(rows_last));
  a.fast_iters = s.sk_iters < (int64_t(1) << 31) ? 1 : 0;
}

int gemm_impl(sk_plan_t p, const void* A, const void* B, const float* scale_a,
              const float* scale_b, void* C, float alpha, float beta, int32_t* trace,
              int64_t trace_ints, void* stream_v, int32_t* err_host = nullptr) {
  if (p == nullptr) return SK_ERR_INVALID;
  // E4M3 plans take their block scales; 16-bit plans take none
  const bool f8 = p->a_type == SK_E4M3;
  if (f8 != (scale_a != nullptr) || f8 != (scale_b != nullptr)) return SK_ERR_INVALID;
  if (f8 && ((reinterpret_cast<uintptr_t>(scale_a) & 3u) || (reinterpret_cast<uintptr_t>(scale_b) & 3u)))
    return SK_ERR_INVALID;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  if (p->m == 0 || p->n == 0) return SK_OK;
  if (C == nullptr || (reinterpret_cast<uintptr_t>(C) & 15u)) return SK_ERR_INVALID;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != p->device) return SK_ERR_INVALID;
  // The plan's workspace serves one launch at a time: refuse a launch on a
  // second stream while the last one still runs.
  if (const int bs = busy_check(p->inflight, stream); bs != SK_OK) return bs;
  const sk_schedule_info& s = p->info;
  p->last_stream = stream;
  p->launched = true;

  if (p->k == 0) {
    const int64_t m = p->swap ? p->n : p->m, n = p->swap ? p->m : p->n;
    const int64_t total = m * n;
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<int64_t>((total + threads - 1) / threads, 4096));
    if (p->c_type == SK_F32)
      scale_kernel<float><<<blocks, threads, 0, stream>>>(static_cast<float*>(C), m, n, p->ldc, beta);
    else if (p->c_type == SK_BF16)
      scale_kernel<__nv_bfloat16><<<blocks, threads, 0, stream>>>(static_cast<__nv_bfloat16*>(C), m,
                                                                   n, p->ldc, beta);
    else
      scale_kernel<__half><<<blocks, threads, 0, stream>>>(static_cast<__half*>(C), m, n, p->ldc, beta);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    return busy_record(p->inflight, stream);
  }

  if (A == nullptr || B == nullptr || (reinterpret_cast<uintptr_t>(A) & 15u) ||
      (reinterpret_cast<uintptr_t>(B) & 15u))
    return SK_ERR_INVALID;
  if (trace != nullptr) {
    const int64_t need = static_cast<int64_t>(s.ctas) *
                         (sk::kTraceHeaderInts + static_cast<int64_t>(s.max_segments) *
                                                     sk::kTraceRecordInts);
    if (trace_ints < need) return SK_ERR_INVALID;
  }

  // Kernel operands: "A" is m x k K-contiguous, "B" is n x k K-contiguous.
  const void* ka = p->swap ? B : A;
  const void* kb = p->swap ? A : B;
  const int64_t km = p->swap ? p->n : p->m;
  const int64_t kn = p->swap ? p->m : p->n;
  const int64_t klda = p->swap ? p->ldb : p->lda;
  const int64_t kldb = p->swap ? p->lda : p->ldb;
  // E4M3 operands go to TMA as 16-bit rows of k/2 elements (the same bytes)
  const int tma_type = f8 ? SK_BF16 : p->a_type;
  const int64_t tk = f8 ? p->k / 2 : p->k;
  const int64_t tlda = f8 ? klda / 2 : klda, tldb = f8 ? kldb / 2 : kldb;
  const bool use3d = s.tile_n <= 128 && tk / sk::kBlkK >= 2;
  if (ka != p->cached_a) {
    int st = encode_operand(&p->tm_a, ka, tma_type, km, tk, tlda, sk::kBlkM);
    if (st == SK_OK && use3d)
      st = encode_operand_3d(&p->tm_a3, ka, tma_type, km, tk, tlda, sk::kBlkM);
    if (st != SK_OK) return st;
    p->cached_a = ka;
  }
  if (kb != p->cached_b) {
    int st = encode_operand(&p->tm_b, kb, tma_type, kn, tk, tldb, s.tile_n / s.cluster_m);
    if (st == SK_OK && use3d)
      st = encode_operand_3d(&p->tm_b3, kb, tma_type, kn, tk, tldb, s.tile_n / s.cluster_m);
    if (st != SK_OK) return st;
    p->cached_b = kb;
  }

  if (C != p->cached_c) {
    p->c_tma = encode_output(&p->tm_c, C, p->c_type, km, kn, p->ldc);
    p->cached_c = C;
  }

  sk::SkArgs a{};
  a.m = static_cast<int32_t>(km);
  a.n = static_cast<int32_t>(kn);
  a.k = static_cast<int32_t>(p->k);
  a.tiles_m = s.tiles_m;
  a.tiles_n = s.tiles_n;
  a.tiles = static_cast<int32_t>(s.tiles);
  a.iters_per_tile = s.iters_per_tile;
  a.group_m = s.raster_group;
  a.sk_tiles = static_cast<int32_t>(s.sk_tiles);
  a.grid = s.grid;
  a.sk_q = static_cast<int32_t>(s.sk_iters / s.grid);
  a.sk_r = static_cast<int32_t>(s.sk_iters % s.grid);
  set_divisors(a, s);
  a.kfull64 = use3d ? static_cast<int32_t>(tk / sk::kBlkK) : 0;
  a.idesc = make_idesc(p->a_type, s.tile_n, s.cluster_m);
  a.C = C;
  a.ldc = p->ldc;
  a.c_vec = (p->ldc * static_cast<int64_t>(dtype_size(p->c_type))) % 16 == 0 ? 1 : 0;
  a.c_tma = p->c_tma ? store_path(p->store_req) : 0;
  a.alpha = alpha;
  a.beta = beta;
  const bool split = s.workspace_bytes > 0;
  a.flags = split ? reinterpret_cast<uint32_t*>(p->ws) : nullptr;
  a.partials = split ? reinterpret_cast<float*>(p->ws + sk::kFlagBytes) : nullptr;
  a.epoch = next_epoch();
  a.err = p->err;
  a.err_host = err_host;
  a.trace = trace;
  a.trace_cap = s.max_segments;
  a.debug_skip_signal = p->debug_skip_signal;
  a.timeout_ns = p->timeout_ns;
  a.pdl = p->pdl ? 1 : 0;
  a.early = p->pdl && p->early ? 1 : 0;
  a.stages = p->stages_req;
  if (f8) {
    a.scale_a = p->swap ? scale_b : scale_a;
    a.scale_b = p->swap ? scale_a : scale_b;
    a.ld_scale = static_cast<int32_t>((p->k + 127) / 128);
  }

  // Split schedules need every CTA resident at once.  Single CTAs ask the
  // launch to guarantee it (cooperative attribute).  Clustered launches go
  // without it: their grid is at most one CTA per SM and nothing of this
  // stream can hold an SM while they wait (a preceding kernel finishes on its
  // own, a following one starts only after every CTA here has started), so
  // all CTAs become resident; the bounded waits turn anything else into an
  // error status.
  const bool cooperative = split && s.cluster_m == 1;
  const CUtensorMap& ta3 = use3d ? p->tm_a3 : p->tm_a;
  const CUtensorMap& tb3 = use3d ? p->tm_b3 : p->tm_b;
  cudaError_t e;
  if (f8)
    e = sk::launch_f8(p->c_type, s.tile_n, s.cluster_m, p->tm_a, p->tm_b, p->tm_c, ta3, tb3, a, cooperative,
                      stream);
  else if (s.tile_n == 64)
    e = sk::launch_bn64(p->c_type, s.cluster_m, p->tm_a, p->tm_b, p->tm_c, ta3, tb3, a, cooperative,
                        stream);
  else if (s.tile_n == 256)
    e = sk::launch_bn256(p->c_type, s.cluster_m, p->tm_a, p->tm_b, p->tm_c, ta3, tb3, a, cooperative,
                         stream);
  else
    e = sk::launch_bn128(p->c_type, s.cluster_m, p->tm_a, p->tm_b, p->tm_c, ta3, tb3, a, cooperative,
                         stream);
  if (e != cudaSuccess) return cuda_status(e);
  return busy_record(p->inflight, stream);
}

}  // namespace

namespace sk {
int gemm_reporting(sk_plan_t p, const void* A, const void* B, const float* scale_a,
                   const float* scale_b, void* C, float alpha, float beta, void* stream,
                   int32_t* err_host) {
  return gemm_impl(p, A, B, scale_a, scale_b, C, alpha, beta, nullptr, 0, stream, err_host);
}
}  // namespace sk

extern "C" {

const char* sk_status_string(int status) {
  switch (status) {
    case SK_OK: return "SK_OK";
    case SK_ERR_INVALID: return "SK_ERR_INVALID";
    case SK_ERR_UNSUPPORTED: return "SK_ERR_UNSUPPORTED";
    case SK_ERR_CUDA: return "SK_ERR_CUDA";
    case SK_ERR_TIMEOUT: return "SK_ERR_TIMEOUT";
    case SK_ERR_NOMEM: return "SK_ERR_NOMEM";
    case SK_ERR_DEVICE: return "SK_ERR_DEVICE";
    case SK_ERR_BUSY: return "SK_ERR_BUSY";
    default: return "SK_ERR_UNKNOWN";
  }
}

int sk_plan(sk_plan_t* out, int64_t m, int64_t n, int64_t k, sk_dtype a_type, sk_dtype b_type,
            sk_dtype c_type, sk_dtype compute_type, sk_layout a_layout, sk_layout b_layout,
            sk_layout c_layout, int mode) {
  if (out == nullptr) return SK_ERR_INVALID;
  *out = nullptr;
  if (m < 0 || n < 0 || k < 0) return SK_ERR_INVALID;
  if (mode < SK_MODE_AUTO || mode > SK_MODE_HYBRID_ONE_TILE) return SK_ERR_INVALID;
  if (!((a_type == SK_F16 || a_type == SK_BF16 || a_type == SK_E4M3) && b_type == a_type))
    return SK_ERR_UNSUPPORTED;
  if (a_type == SK_E4M3 && k % 16 != 0) return SK_ERR_INVALID;  // 16-byte rows
  if (!(c_type == SK_F32 || c_type == SK_BF16 || c_type == SK_F16)) return SK_ERR_UNSUPPORTED;
  if (compute_type != SK_F32) return SK_ERR_UNSUPPORTED;
  if (a_layout != SK_ROW_MAJOR || b_layout != SK_COL_MAJOR) return SK_ERR_UNSUPPORTED;
  if (c_layout != SK_ROW_MAJOR && c_layout != SK_COL_MAJOR) return SK_ERR_INVALID;

  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SK_ERR_CUDA;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SK_ERR_CUDA;
  if (major != 10 || minor != 3) return SK_ERR_DEVICE;

  sk_plan_s* p = new (std::nothrow) sk_plan_s();
  if (p == nullptr) return SK_ERR_NOMEM;
  p->m = m;
  p->n = n;
  p->k = k;
  p->a_type = a_type;
  p->b_type = b_type;
  p->c_type = c_type;
  p->a_layout = a_layout;
  p->b_layout = b_layout;
  p->c_layout = c_layout;
  p->mode_req = mode;
  p->lda = k;
  p->ldb = k;
  p->ldc = c_layout == SK_ROW_MAJOR ? n : m;
  p->swap = c_layout == SK_COL_MAJOR;
  p->device = dev;
  p->num_sms = sms;
  if (a_type == SK_E4M3) {
    // Single CTAs: a pair's per-k-block buffer hand-off crosses SMs and was
    // measured 2.4x slower (SK_ATTR_CLUSTER_M 2 still selects it); the model
    // picks 128- or 256-wide tiles (tile_n_req 0).
    p->tile_n_req = 0;
    p->cluster_req = 1;
  }
  size_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  cudaError_t e = sk::prepare_bn128(&s1);
  if (e == cudaSuccess) e = sk::prepare_bn64(&s0);
  if (e == cudaSuccess) e = sk::prepare_bn256(&s2);
  if (e == cudaSuccess) e = sk::prepare_f8(&s3);
  if (e != cudaSuccess) {
    delete p;
    return cuda_status(e);
  }
  void* errw = nullptr;
  e = cudaMalloc(&errw, 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(errw, 0, 4 * sizeof(int32_t));
  if (e != cudaSuccess) {
    if (errw) cudaFree(errw);
    delete p;
    return cuda_status(e);
  }
  p->err = static_cast<int32_t*>(errw);
  int st = replan(p);
  if (st != SK_OK) {
    sk_plan_destroy(p);
    return st;
  }
  *out = p;
  return SK_OK;
}

int sk_plan_destroy(sk_plan_t p) {
  if (p == nullptr) return SK_OK;
  busy_release(p->inflight);
  if (p->ws && p->ws_owned) cudaFree(p->ws);
  if (p->err) cudaFree(p->err);
  delete p;
  return SK_OK;
}

int sk_gemm(sk_plan_t p, const void* A, const void* B, void* C, float alpha, float beta,
            void* stream) {
  return gemm_impl(p, A, B, nullptr, nullptr, C, alpha, beta, nullptr, 0, stream);
}

int sk_gemm_scaled(sk_plan_t p, const void* A, const void* B, const float* scale_a,
                   const float* scale_b, void* C, float alpha, float beta, void* stream) {
  if (scale_a == nullptr || scale_b == nullptr) return SK_ERR_INVALID;
  return gemm_impl(p, A, B, scale_a, scale_b, C, alpha, beta, nullptr, 0, stream);
}

int sk_gemm_traced(sk_plan_t p, const void* A, const void* B, void* C, float alpha, float beta,
                   int32_t* trace, int64_t trace_ints, void* stream) {
  if (trace == nullptr) return SK_ERR_INVALID;
  return gemm_impl(p, A, B, nullptr, nullptr, C, alpha, beta, trace, trace_ints, stream);
}

int sk_last_error(sk_plan_t p, int* device_status) {
  if (p == nullptr) return SK_ERR_INVALID;
  if (device_status) *device_status = 0;
  cudaError_t e = p->launched ? cudaStreamSynchronize(p->last_stream) : cudaSuccess;
  if (e != cudaSuccess) return SK_ERR_CUDA;
  int32_t h[4] = {0, 0, 0, 0};
  e = cudaMemcpy(h, p->err, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return SK_ERR_CUDA;
  if (h[0] != 0 || h[3] != 0) {
    // A failed launch can leave flags raised that no owner consumed: clear
    // them with the status so the next launch starts clean.
    e = cudaMemset(p->err, 0, 4 * sizeof(int32_t));
    if (e == cudaSuccess && p->ws != nullptr)
      e = cudaMemset(p->ws, 0, static_cast<size_t>(sk::kFlagBytes));
    if (e != cudaSuccess) return SK_ERR_CUDA;
  }
  if (device_status) *device_status = h[0];
  return h[0] == 0 ? SK_OK : SK_ERR_TIMEOUT;
}

int sk_plan_set(sk_plan_t p, int attr, int64_t v) {
  if (p == nullptr) return SK_ERR_INVALID;
  const int64_t min_ld_a = p->k, min_ld_b = p->k;
  const int64_t min_ld_c = p->c_layout == SK_ROW_MAJOR ? p->n : p->m;
  switch (attr) {
    case SK_ATTR_TILE_N: {
      if (v != 0 && v != 64 && v != 128 && v != 256) return SK_ERR_UNSUPPORTED;
      // E4M3: 0 (the model's choice of 128 and 256), 128 (single CTAs or
      // pairs) or 256 (single CTAs)
      if (p->a_type == SK_E4M3 && v != 0 && v != 128 && !(v == 256 && p->cluster_req != 2))
        return SK_ERR_UNSUPPORTED;
      const int old = p->tile_n_req;
      p->tile_n_req = static_cast<int>(v);
      int st = replan(p);
      if (st != SK_OK) {
        p->tile_n_req = old;
        replan(p);
      }
      return st;
    }
    case SK_ATTR_GRID: {
      if (v < 0 || v > p->num_sms) return SK_ERR_INVALID;
      const int old = p->grid_req;
      p->grid_req = static_cast<int>(v);
      int st = replan(p);
      if (st != SK_OK) {
        p->grid_req = old;
        replan(p);
      }
      return st;
    }
    case SK_ATTR_RASTER_GROUP: {
      if (v < 0 || v > (1 << 20)) return SK_ERR_INVALID;
      p->group_req = static_cast<int>(v);
      return replan(p);
    }
    case SK_ATTR_TIMEOUT_NS:
      if (v <= 0) return SK_ERR_INVALID;
      p->timeout_ns = static_cast<uint64_t>(v);
      return SK_OK;
    case SK_ATTR_LDA:
      if (v < min_ld_a || (v * static_cast<int64_t>(dtype_size(p->a_type))) % 16) return SK_ERR_INVALID;
      p->lda = v;
      p->cached_a = p->cached_b = nullptr;
      return SK_OK;
    case SK_ATTR_LDB:
      if (v < min_ld_b || (v * static_cast<int64_t>(dtype_size(p->b_type))) % 16) return SK_ERR_INVALID;
      p->ldb = v;
      p->cached_a = p->cached_b = nullptr;
      return SK_OK;
    case SK_ATTR_LDC:
      if (v < min_ld_c) return SK_ERR_INVALID;
      p->ldc = v;
      p->cached_c = nullptr;
      return SK_OK;
    case SK_ATTR_DEBUG_SKIP_SIGNAL:
      if (v < -1 || v >= p->num_sms) return SK_ERR_INVALID;
      p->debug_skip_signal = static_cast<int>(v);
      return SK_OK;
    case SK_ATTR_PDL:
      if (v != 0 && v != 1) return SK_ERR_INVALID;
      p->pdl = v != 0;
      return SK_OK;
    case SK_ATTR_STORE:
      if (v < 0 || v > 2) return SK_ERR_INVALID;
      p->store_req = static_cast<int>(v);
      return SK_OK;
    case SK_ATTR_INDEPENDENT_INPUTS:
      if (v != 0 && v != 1) return SK_ERR_INVALID;
      p->early = v != 0;
      return SK_OK;
    case SK_ATTR_STAGES:
      if (v != 0 && (v < 2 || v > sk::max_stages(p->info.tile_n, p->info.cluster_m)))
        return SK_ERR_INVALID;
      p->stages_req = static_cast<int>(v);
      return SK_OK;
    case SK_ATTR_CLUSTER_M: {
      if (v != 0 && v != 1 && v != 2) return SK_ERR_UNSUPPORTED;
      if (p->a_type == SK_E4M3 && v == 2 && p->tile_n_req == 256) return SK_ERR_UNSUPPORTED;
      const int old = p->cluster_req;
      p->cluster_req = static_cast<int>(v);
      int st = replan(p);
      if (st != SK_OK) {
        p->cluster_req = old;
        replan(p);
      }
      return st;
    }
    default:
      return SK_ERR_INVALID;
  }
}

int sk_plan_get(sk_plan_t p, int attr, int64_t* v) {
  if (p == nullptr || v == nullptr) return SK_ERR_INVALID;
  const sk_schedule_info& s = p->info;
  switch (attr) {
    case SK_ATTR_TILE_N: *v = s.tile_n; return SK_OK;
    case SK_ATTR_GRID: *v = s.grid; return SK_OK;
    case SK_ATTR_RASTER_GROUP: *v = s.raster_group; return SK_OK;
    case SK_ATTR_TIMEOUT_NS: *v = static_cast<int64_t>(p->timeout_ns); return SK_OK;
    case SK_ATTR_LDA: *v = p->lda; return SK_OK;
    case SK_ATTR_LDB: *v = p->ldb; return SK_OK;
    case SK_ATTR_LDC: *v = p->ldc; return SK_OK;
    case SK_ATTR_DEBUG_SKIP_SIGNAL: *v = p->debug_skip_signal; return SK_OK;
    case SK_ATTR_PDL: *v = p->pdl ? 1 : 0; return SK_OK;
    case SK_ATTR_STORE: *v = p->store_req; return SK_OK;
    case SK_ATTR_INDEPENDENT_INPUTS: *v = p->early ? 1 : 0; return SK_OK;
    case SK_ATTR_STAGES: {
      const int mx = sk::max_stages(s.tile_n, s.cluster_m);
      *v = p->stages_req >= 2 && p->stages_req < mx ? p->stages_req : mx;
      return SK_OK;
    }
    case SK_ATTR_CLUSTER_M: *v = s.cluster_m; return SK_OK;
    case SK_ATTR_CTAS: *v = s.ctas; return SK_OK;
    case SK_ATTR_MODE: *v = s.mode; return SK_OK;
    case SK_ATTR_TILE_M: *v = s.tile_m; return SK_OK;
    case SK_ATTR_TILE_K: *v = s.tile_k; return SK_OK;
    case SK_ATTR_TILES_M: *v = s.tiles_m; return SK_OK;
    case SK_ATTR_TILES_N: *v = s.tiles_n; return SK_OK;
    case SK_ATTR_TILES: *v = s.tiles; return SK_OK;
    case SK_ATTR_ITERS_PER_TILE: *v = s.iters_per_tile; return SK_OK;
    case SK_ATTR_SK_TILES: *v = s.sk_tiles; return SK_OK;
    case SK_ATTR_DP_TILES: *v = s.dp_tiles; return SK_OK;
    case SK_ATTR_WORKSPACE_BYTES: *v = s.workspace_bytes; return SK_OK;
    case SK_ATTR_NUM_SMS: *v = p->num_sms; return SK_OK;
    case SK_ATTR_TRACE_CAP: *v = s.max_segments; return SK_OK;
    case SK_ATTR_TRACE_INTS:
      *v = static_cast<int64_t>(s.ctas) *
           (sk::kTraceHeaderInts + static_cast<int64_t>(s.max_segments) * sk::kTraceRecordInts);
      return SK_OK;
    default:
      return SK_ERR_INVALID;
  }
}

int sk_plan_attach_workspace(sk_plan_t p, void* ws, size_t bytes) {
  if (p == nullptr || ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255u)) return SK_ERR_INVALID;
  if (bytes < static_cast<size_t>(p->info.workspace_bytes)) return SK_ERR_INVALID;
  if (p->ws && p->ws_owned) cudaFree(p->ws);
  p->ws = static_cast<char*>(ws);
  p->ws_bytes = bytes;
  p->ws_owned = false;
  if (bytes >= static_cast<size_t>(sk::kFlagBytes)) {
    cudaError_t e = cudaMemset(p->ws, 0, static_cast<size_t>(sk::kFlagBytes));
    if (e != cudaSuccess) return cuda_status(e);
  }
  return SK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point (sk_gemm_noalloc, declared in streamk.h).
//
// The fixup scratch (flags, status words, FP32 partial tiles) lives in one
// file-scope __device__ array that every device loading this library holds
// until the process exits.  Host code never names the array's address
// directly: its host-side symbol is only a stand-in, so the device address is
// fetched once per device with cudaGetSymbolAddress (with that device current)
// and passed to the kernel.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(12) << 20;  // 12 MiB per device
constexpr size_t kNoAllocStatusOffset = static_cast<size_t>(sk::kFlagBytes);  // 4 words
constexpr size_t kNoAllocPartialsOffset = kNoAllocStatusOffset + 4096;
constexpr int kNoAllocMaxDevices = 64;
// Partial tiles (128 x 128 FP32, 64 KiB each) the scratch holds after the
// flags and status words: 189.  A launch has at most one CTA per SM.
constexpr size_t kNoAllocMaxCtas =
    (kNoAllocScratchBytes - kNoAllocPartialsOffset) / (size_t(sk::kBlkM) * 128 * 4);
static_assert(kNoAllocMaxCtas == 189, "scratch size and the documented CTA limit");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

struct NoAllocDevice {
  std::once_flag once;
  int status = SK_ERR_CUDA;
  char* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int num_sms = 0;
};
NoAllocDevice g_noalloc_devices[kNoAllocMaxDevices];

void noalloc_setup(NoAllocDevice* d, int dev) {
  int major = 0, minor = 0, sms = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    d->status = SK_ERR_CUDA;
    return;
  }
  if (major != 10 || minor != 3) {
    d->status = SK_ERR_DEVICE;
    return;
  }
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || ptr == nullptr) {
    d->status = SK_ERR_CUDA;
    return;
  }
  size_t smem = 0;
  if (sk::prepare_bn128(&smem) != cudaSuccess) {
    d->status = SK_ERR_CUDA;
    return;
  }
  d->scratch = static_cast<char*>(ptr);
  d->num_sms = sms;
  d->status = SK_OK;
}

}  // namespace

extern "C" int sk_gemm_noalloc(int64_t m, int64_t n, int64_t k, sk_dtype ab_type, sk_dtype c_type,
                               const void* A, int64_t lda, const void* B, int64_t ldb, void* C,
                               int64_t ldc, float alpha, float beta, int mode,
                               int32_t* device_status, void* stream_v) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  if (m < 0 || n < 0 || k < 0) return SK_ERR_INVALID;
  if (ab_type != SK_F16 && ab_type != SK_BF16) return SK_ERR_UNSUPPORTED;
  if (c_type != SK_F32 && c_type != SK_BF16 && c_type != SK_F16) return SK_ERR_UNSUPPORTED;
  if (mode < SK_MODE_AUTO || mode > SK_MODE_HYBRID_ONE_TILE) return SK_ERR_INVALID;
  if (lda < k || ldb < k || ldc < n) return SK_ERR_INVALID;
  if (k > 0 && ((lda * 2) % 16 != 0 || (ldb * 2) % 16 != 0)) return SK_ERR_INVALID;
  if (device_status != nullptr && (reinterpret_cast<uintptr_t>(device_status) & 3u))
    return SK_ERR_INVALID;

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SK_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SK_ERR_UNSUPPORTED;
  NoAllocDevice* d = &g_noalloc_devices[dev];
  std::call_once(d->once, noalloc_setup, d, dev);
  if (d->status != SK_OK) return d->status;

  if (m == 0 || n == 0) return SK_OK;
  if (C == nullptr || (reinterpret_cast<uintptr_t>(C) & 15u)) return SK_ERR_INVALID;
  char* const scratch = d->scratch;
  int32_t* const err = reinterpret_cast<int32_t*>(scratch + kNoAllocStatusOffset);

  // Every host-side check and the tensor-map encoding come first, so that a
  // call that returns an error has enqueued nothing on the stream.
  sk_schedule_info s{};
  CUtensorMap tma, tmb, tmc, tma3, tmb3;
  bool split = false, use3d = false, c_tma = false;
  if (k > 0) {
    if (A == nullptr || B == nullptr || (reinterpret_cast<uintptr_t>(A) & 15u) ||
        (reinterpret_cast<uintptr_t>(B) & 15u))
      return SK_ERR_INVALID;
    int st = sk::describe(m, n, k, mode, 128, 0, 0, 1, d->num_sms, &s);
    if (st != SK_OK) return st;
    split = s.workspace_bytes > 0;
    const size_t partial_bytes = static_cast<size_t>(s.ctas) * sk::kBlkM * 128 * 4;
    // Never taken on sm_103: the grid is at most one CTA per SM, far below
    // the kNoAllocMaxCtas partial tiles the scratch holds.
    if (split && kNoAllocPartialsOffset + partial_bytes > kNoAllocScratchBytes)
      return SK_ERR_INVALID;
    if ((st = encode_operand(&tma, A, ab_type, m, k, lda, sk::kBlkM)) != SK_OK) return st;
    if ((st = encode_operand(&tmb, B, ab_type, n, k, ldb, 128)) != SK_OK) return st;
    use3d = s.tile_k == 2 * sk::kBlkK && k / sk::kBlkK >= 2;
    tma3 = tma;
    tmb3 = tmb;
    if (use3d) {
      if ((st = encode_operand_3d(&tma3, A, ab_type, m, k, lda, sk::kBlkM)) != SK_OK) return st;
      if ((st = encode_operand_3d(&tmb3, B, ab_type, n, k, ldb, 128)) != SK_OK) return st;
    }
    c_tma = encode_output(&tmc, C, c_type, m, n, ldc);
  }

  // The status words must start at zero for every call (flags too, below).
  cudaError_t e = cudaMemsetAsync(err, 0, 4 * sizeof(int32_t), stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (k == 0) {  // C = beta * C
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<int64_t>((m * n + threads - 1) / threads, 4096));
    if (c_type == SK_F32)
      scale_kernel<float><<<blocks, threads, 0, stream>>>(static_cast<float*>(C), m, n, ldc, beta);
    else if (c_type == SK_BF16)
      scale_kernel<__nv_bfloat16><<<blocks, threads, 0, stream>>>(static_cast<__nv_bfloat16*>(C), m,
                                                                   n, ldc, beta);
    else
      scale_kernel<__half><<<blocks, threads, 0, stream>>>(static_cast<__half*>(C), m, n, ldc, beta);
    e = cudaGetLastError();
  } else {
    if (split) {
      e = cudaMemsetAsync(scratch, 0, static_cast<size_t>(sk::kFlagBytes), stream);
      if (e != cudaSuccess) return cuda_status(e);
    }
    sk::SkArgs a{};
    a.m = static_cast<int32_t>(m);
    a.n = static_cast<int32_t>(n);
    a.k = static_cast<int32_t>(k);
    a.tiles_m = s.tiles_m;
    a.tiles_n = s.tiles_n;
    a.tiles = static_cast<int32_t>(s.tiles);
    a.iters_per_tile = s.iters_per_tile;
    a.group_m = s.raster_group;
    a.sk_tiles = static_cast<int32_t>(s.sk_tiles);
    a.grid = s.grid;
    a.sk_q = static_cast<int32_t>(s.sk_iters / s.grid);
    a.sk_r = static_cast<int32_t>(s.sk_iters % s.grid);
    set_divisors(a, s);
    a.kfull64 = use3d ? static_cast<int32_t>(k / sk::kBlkK) : 0;
    a.idesc = make_idesc(ab_type, 128, 1);
    a.C = C;
    a.ldc = ldc;
    a.c_vec = (ldc * static_cast<int64_t>(dtype_size(c_type))) % 16 == 0 ? 1 : 0;
    a.c_tma = c_tma ? store_path(0) : 0;
    a.alpha = alpha;
    a.beta = beta;
    a.flags = split ? reinterpret_cast<uint32_t*>(scratch) : nullptr;
    a.partials = split ? reinterpret_cast<float*>(scratch + kNoAllocPartialsOffset) : nullptr;
    a.epoch = next_epoch();
    a.err = err;
    a.trace = nullptr;
    a.trace_cap = 0;
    a.debug_skip_signal = -1;
    a.timeout_ns = kDefaultTimeoutNs;
    a.pdl = 1;
    e = sk::launch_bn128(c_type, 1, tma, tmb, tmc, tma3, tmb3, a, split, stream);
  }
  if (e != cudaSuccess) return cuda_status(e);
  if (device_status != nullptr) {
    e = cudaMemcpyAsync(device_status, err, sizeof(int32_t), cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return SK_OK;
}

// ------------------------------------------------------------------ grouped GEMM
struct sk_grouped_s {
  int count = 0;
  std::vector<int64_t> m, n, k;
  int ab_type = 0, c_type = 0;
  int mode_req = SK_MODE_AUTO, tile_n_req = 0, grid_req = 0;
  int device = 0, num_sms = 0;
  sk::GroupPlan plan;
  // device: the walk table and per-CTA start problems
  sk::GroupWalk* d_walk = nullptr;
  int32_t* d_start = nullptr;
  sk::GroupProblem* d_probs = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int32_t* err = nullptr;
  // host copy of the problem table (pinned) and what it was encoded for
  sk::GroupProblem* h_probs = nullptr;
  cudaEvent_t copied = nullptr;
  bool copy_pending = false;
  bool table_valid = false;
  std::vector<const void*> enc_a, enc_b;
  std::vector<const float*> enc_sa, enc_sb;
  std::vector<void*> enc_c;
  std::vector<float> enc_alpha, enc_beta;
  // knobs
  uint64_t timeout_ns = kDefaultTimeoutNs;
  bool pdl = true;
  int store_req = 0;
  int stages_req = 0;  // SK_ATTR_STAGES (0: all the ring holds)
  int cluster_req = 0;  // SK_ATTR_CLUSTER_M (0: planned)
  cudaStream_t last_stream = nullptr;
  bool launched = false;
  InFlight inflight;  // the last launch, for SK_ERR_BUSY
};

namespace {

void grouped_free_schedule(sk_grouped_s* g) {
  if (g->d_walk) cudaFree(g->d_walk);
  if (g->d_start) cudaFree(g->d_start);
  g->d_walk = nullptr;
  g->d_start = nullptr;
}

// Plan the group and upload its walk table; grow the workspace if the
// schedule splits tiles.  Any cached problem table is re-encoded next launch
// (the tile width sets the tensor-map boxes).
int grouped_replan(sk_grouped_s* g) {
  sk::GroupPlan gp;
  // E4M3 problems are planned as 16-bit problems of k/2 (the same bytes per row)
  const bool f8 = g->ab_type == SK_E4M3;
  std::vector<int64_t> kk(g->k);
  if (f8)
    for (int64_t& v : kk) v /= 2;
  int st = sk::describe_grouped(g->count, g->m.data(), g->n.data(), kk.data(), g->mode_req,
                                g->tile_n_req, g->grid_req, g->num_sms, &gp, g->cluster_req);
  if (st != SK_OK) return st;
  if (f8) gp.tile_k *= 2;  // in E4M3 elements
  if (g->launched) {
    cudaError_t e = cudaStreamSynchronize(g->last_stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (gp.workspace_bytes > 0 && static_cast<size_t>(gp.workspace_bytes) > g->ws_bytes) {
    if (g->ws) cudaFree(g->ws);
    g->ws = nullptr;
    g->ws_bytes = 0;
    void* w = nullptr;
    cudaError_t e = cudaMalloc(&w, static_cast<size_t>(gp.workspace_bytes));
    if (e == cudaSuccess) e = cudaMemset(w, 0, static_cast<size_t>(gp.workspace_bytes));
    if (e != cudaSuccess) {
      if (w) cudaFree(w);
      return cuda_status(e);
    }
    g->ws = static_cast<char*>(w);
    g->ws_bytes = static_cast<size_t>(gp.workspace_bytes);
  }
  grouped_free_schedule(g);
  void *walk = nullptr, *start = nullptr;
  cudaError_t e = cudaMalloc(&walk, gp.walk.size() * sizeof(sk::GroupWalk));
  if (e == cudaSuccess) e = cudaMalloc(&start, gp.gstart.size() * sizeof(int32_t));
  if (e == cudaSuccess)
    e = cudaMemcpy(walk, gp.walk.data(), gp.walk.size() * sizeof(sk::GroupWalk), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(start, gp.gstart.data(), gp.gstart.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (walk) cudaFree(walk);
    if (start) cudaFree(start);
    return cuda_status(e);
  }
  g->d_walk = static_cast<sk::GroupWalk*>(walk);
  g->d_start = static_cast<int32_t*>(start);
  g->plan = std::move(gp);
  g->table_valid = false;
  return SK_OK;
}

int grouped_impl(sk_grouped_s* g, const void* const* A, const void* const* B,
                 const float* const* SA, const float* const* SB, void* const* C,
                 const float* alpha, const float* beta, int32_t* trace, int64_t trace_ints,
                 void* stream_v) {
  if (g == nullptr || A == nullptr || B == nullptr || C == nullptr) return SK_ERR_INVALID;
  // E4M3 groups take every problem's block scales; 16-bit groups take none
  const bool f8 = g->ab_type == SK_E4M3;
  if (f8 != (SA != nullptr) || f8 != (SB != nullptr)) return SK_ERR_INVALID;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  if (const int bs = busy_check(g->inflight, stream); bs != SK_OK) return bs;
  const sk::GroupPlan& gp = g->plan;
  if (trace != nullptr) {
    const int64_t need = static_cast<int64_t>(gp.grid) * gp.cluster_m *
                         (sk::kTraceHeaderInts + static_cast<int64_t>(gp.max_segments) * sk::kTraceRecordInts);
    if (trace_ints < need) return SK_ERR_INVALID;
  }
  // Encode the problems whose operands changed since the table was built
  // (all of them after a replan), after the previous upload of the pinned
  // table has been read.
  std::vector<char> changed(static_cast<size_t>(g->count), 0);
  bool dirty = false;
  for (int i = 0; i < g->count; ++i) {
    const float al = alpha ? alpha[i] : 1.0f, be = beta ? beta[i] : 0.0f;
    if (A[i] == nullptr || B[i] == nullptr || C[i] == nullptr ||
        (reinterpret_cast<uintptr_t>(A[i]) & 15u) || (reinterpret_cast<uintptr_t>(B[i]) & 15u) ||
        (reinterpret_cast<uintptr_t>(C[i]) & 15u))
      return SK_ERR_INVALID;
    const float* sa = f8 ? SA[i] : nullptr;
    const float* sb = f8 ? SB[i] : nullptr;
    if (f8 && (sa == nullptr || sb == nullptr || (reinterpret_cast<uintptr_t>(sa) & 3u) ||
               (reinterpret_cast<uintptr_t>(sb) & 3u)))
      return SK_ERR_INVALID;
    changed[static_cast<size_t>(i)] =
        !g->table_valid || A[i] != g->enc_a[i] || B[i] != g->enc_b[i] || C[i] != g->enc_c[i] ||
        al != g->enc_alpha[i] || be != g->enc_beta[i] || sa != g->enc_sa[i] || sb != g->enc_sb[i];
    dirty = dirty || changed[static_cast<size_t>(i)];
  }
  if (dirty && g->copy_pending) {
    cudaError_t e = cudaEventSynchronize(g->copied);
    if (e != cudaSuccess) return cuda_status(e);
    g->copy_pending = false;
  }
  for (int i = 0; i < g->count; ++i) {
    if (!changed[static_cast<size_t>(i)]) continue;
    const float al = alpha ? alpha[i] : 1.0f, be = beta ? beta[i] : 0.0f;
    sk::GroupProblem& pr = g->h_probs[i];
    const int64_t m = g->m[i], n = g->n[i], k = g->k[i];
    // E4M3 rows go to TMA as 16-bit rows of k/2 elements
    const int tt = f8 ? SK_BF16 : g->ab_type;
    const int64_t tk = f8 ? k / 2 : k;
    int st = encode_operand(&pr.tmA, A[i], tt, m, tk, tk, sk::kBlkM);
    // a CTA of a pair loads half of the B tile
    if (st == SK_OK) st = encode_operand(&pr.tmB, B[i], tt, n, tk, tk, gp.tile_n / gp.cluster_m);
    const bool use3d = gp.tile_n <= 128 && tk / sk::kBlkK >= 2;
    if (st == SK_OK && use3d) st = encode_operand_3d(&pr.tmA3, A[i], tt, m, tk, tk, sk::kBlkM);
    if (st == SK_OK && use3d)
      st = encode_operand_3d(&pr.tmB3, B[i], tt, n, tk, tk, gp.tile_n / gp.cluster_m);
    if (st != SK_OK) {
      g->table_valid = false;
      return st;
    }
    if (!use3d) {
      pr.tmA3 = pr.tmA;
      pr.tmB3 = pr.tmB;
    }
    const bool c_tma = encode_output(&pr.tmC, C[i], g->c_type, m, n, n);
    if (!c_tma) pr.tmC = pr.tmA;
    pr.C = C[i];
    pr.ldc = n;
    pr.m = static_cast<int32_t>(m);
    pr.n = static_cast<int32_t>(n);
    pr.c_tma = c_tma ? store_path(g->store_req) : 0;
    pr.c_vec = (n * static_cast<int64_t>(dtype_size(g->c_type))) % 16 == 0 ? 1 : 0;
    pr.alpha = al;
    pr.beta = be;
    pr.scale_a = f8 ? SA[i] : nullptr;
    pr.scale_b = f8 ? SB[i] : nullptr;
    pr.ld_scale = static_cast<int32_t>((k + 127) / 128);
    g->enc_sa[i] = pr.scale_a;
    g->enc_sb[i] = pr.scale_b;
    g->enc_a[i] = A[i];
    g->enc_b[i] = B[i];
    g->enc_c[i] = C[i];
    g->enc_alpha[i] = al;
    g->enc_beta[i] = be;
  }
  if (dirty) {
    cudaError_t e = cudaMemcpyAsync(g->d_probs, g->h_probs,
                                    static_cast<size_t>(g->count) * sizeof(sk::GroupProblem),
                                    cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(g->copied, stream);
    if (e != cudaSuccess) return cuda_status(e);
    g->copy_pending = true;
    g->table_valid = true;
  }
  sk::SkArgs a{};
  sk::set_group_walk_args(a, gp);
  a.idesc = make_idesc(g->ab_type, gp.tile_n, gp.cluster_m);
  a.c_tma = 0;
  const bool split = gp.workspace_bytes > 0;
  // co-residency of a split schedule: as for single GEMMs, single CTAs ask
  // for it, CTA pairs rely on the stream order
  const bool cooperative = split && gp.cluster_m == 1;
  a.flags = split ? reinterpret_cast<uint32_t*>(g->ws) : nullptr;
  a.partials = split ? reinterpret_cast<float*>(g->ws + sk::kFlagBytes) : nullptr;
  a.epoch = next_epoch();
  a.err = g->err;
  a.trace = trace;
  a.trace_cap = gp.max_segments;
  a.debug_skip_signal = -1;
  a.timeout_ns = g->timeout_ns;
  a.pdl = g->pdl ? 1 : 0;
  a.gwalk = g->d_walk;
  a.gstart = g->d_start;
  a.gprobs = g->d_probs;
  a.stages = g->stages_req;
  const CUtensorMap& any = g->h_probs[0].tmA;
  const int cm = gp.cluster_m;
  cudaError_t e =
      f8                 ? sk::launch_grouped_f8(g->c_type, gp.tile_n, any, a, cooperative, stream)
      : gp.tile_n == 256 ? sk::launch_grouped_bn256(g->c_type, cm, any, a, cooperative, stream)
      : gp.tile_n == 64  ? sk::launch_grouped_bn64(g->c_type, cm, any, a, cooperative, stream)
                         : sk::launch_grouped_bn128(g->c_type, cm, any, a, cooperative, stream);
  if (e != cudaSuccess) return cuda_status(e);
  g->last_stream = stream;
  g->launched = true;
  return busy_record(g->inflight, stream);
}

}  // namespace

extern "C" {

int sk_grouped_plan(sk_grouped_t* out, int count, const int64_t* m, const int64_t* n,
                    const int64_t* k, sk_dtype ab_type, sk_dtype c_type, int mode) {
  if (out == nullptr) return SK_ERR_INVALID;
  *out = nullptr;
  if (count < 1 || count > (1 << 20) || m == nullptr || n == nullptr || k == nullptr)
    return SK_ERR_INVALID;
  if (!(ab_type == SK_F16 || ab_type == SK_BF16 || ab_type == SK_E4M3)) return SK_ERR_UNSUPPORTED;
  if (!(c_type == SK_F32 || c_type == SK_BF16 || c_type == SK_F16)) return SK_ERR_UNSUPPORTED;
  if (mode != SK_MODE_AUTO && mode != SK_MODE_DP && mode != SK_MODE_SK && mode != SK_MODE_HYBRID)
    return SK_ERR_UNSUPPORTED;
  const int64_t k_align = ab_type == SK_E4M3 ? 16 : 8;
  for (int i = 0; i < count; ++i)  // dense rows of A and B must be 16-byte multiples (TMA)
    if (k[i] < 1 || k[i] % k_align != 0) return SK_ERR_INVALID;
  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SK_ERR_CUDA;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SK_ERR_CUDA;
  if (major != 10 || minor != 3) return SK_ERR_DEVICE;
  sk_grouped_s* g = new (std::nothrow) sk_grouped_s();
  if (g == nullptr) return SK_ERR_NOMEM;
  g->count = count;
  g->m.assign(m, m + count);
  g->n.assign(n, n + count);
  g->k.assign(k, k + count);
  g->ab_type = ab_type;
  g->c_type = c_type;
  g->mode_req = mode;
  g->device = dev;
  g->num_sms = sms;
  g->enc_a.assign(count, nullptr);
  g->enc_b.assign(count, nullptr);
  g->enc_c.assign(count, nullptr);
  g->enc_alpha.assign(count, 0.0f);
  g->enc_beta.assign(count, 0.0f);
  g->enc_sa.assign(count, nullptr);
  g->enc_sb.assign(count, nullptr);
  if (ab_type == SK_E4M3) {
    g->tile_n_req = 128;  // 128 x 128 x 128 tiles by default (SK_ATTR_TILE_N 256: 128 x 256)
    g->cluster_req = 1;   // on single CTAs (grouped E4M3 launches have no CTA pairs)
  }
  size_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  cudaError_t e = sk::prepare_bn128(&s1);
  if (e == cudaSuccess) e = sk::prepare_bn64(&s0);
  if (e == cudaSuccess) e = sk::prepare_bn256(&s2);
  if (e == cudaSuccess) e = sk::prepare_f8(&s3);
  void *errw = nullptr, *probs = nullptr, *hprobs = nullptr;
  const size_t table = static_cast<size_t>(count) * sizeof(sk::GroupProblem);
  if (e == cudaSuccess) e = cudaMalloc(&errw, 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(errw, 0, 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&probs, table);
  if (e == cudaSuccess) e = cudaMallocHost(&hprobs, table);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->copied, cudaEventDisableTiming);
  g->err = static_cast<int32_t*>(errw);
  g->d_probs = static_cast<sk::GroupProblem*>(probs);
  g->h_probs = static_cast<sk::GroupProblem*>(hprobs);
  if (e != cudaSuccess) {
    sk_grouped_destroy(g);
    return cuda_status(e);
  }
  std::memset(static_cast<void*>(g->h_probs), 0, table);
  int st = grouped_replan(g);
  if (st != SK_OK) {
    sk_grouped_destroy(g);
    return st;
  }
  *out = g;
  return SK_OK;
}

int sk_grouped_destroy(sk_grouped_t g) {
  if (g == nullptr) return SK_OK;
  if (g->launched) cudaStreamSynchronize(g->last_stream);
  grouped_free_schedule(g);
  if (g->d_probs) cudaFree(g->d_probs);
  if (g->h_probs) cudaFreeHost(g->h_probs);
  if (g->copied) cudaEventDestroy(g->copied);
  busy_release(g->inflight);
  if (g->ws) cudaFree(g->ws);
  if (g->err) cudaFree(g->err);
  delete g;
  return SK_OK;
}

int sk_grouped_gemm(sk_grouped_t g, const void* const* A, const void* const* B, void* const* C,
                    const float* alpha, const float* beta, void* stream) {
  return grouped_impl(g, A, B, nullptr, nullptr, C, alpha, beta, nullptr, 0, stream);
}

int sk_grouped_gemm_scaled(sk_grouped_t g, const void* const* A, const void* const* B,
                           const float* const* SA, const float* const* SB, void* const* C,
                           const float* alpha, const float* beta, void* stream) {
  if (SA == nullptr || SB == nullptr) return SK_ERR_INVALID;
  return grouped_impl(g, A, B, SA, SB, C, alpha, beta, nullptr, 0, stream);
}

int sk_grouped_gemm_traced(sk_grouped_t g, const void* const* A, const void* const* B,
                           void* const* C, const float* alpha, const float* beta, int32_t* trace,
                           int64_t trace_ints, void* stream) {
  if (trace == nullptr) return SK_ERR_INVALID;
  return grouped_impl(g, A, B, nullptr, nullptr, C, alpha, beta, trace, trace_ints, stream);
}

int sk_grouped_last_error(sk_grouped_t g, int* device_status) {
  if (g == nullptr) return SK_ERR_INVALID;
  if (device_status) *device_status = 0;
  cudaError_t e = g->launched ? cudaStreamSynchronize(g->last_stream) : cudaSuccess;
  if (e != cudaSuccess) return SK_ERR_CUDA;
  int32_t h[4] = {0, 0, 0, 0};
  e = cudaMemcpy(h, g->err, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return SK_ERR_CUDA;
  if (h[0] != 0 || h[3] != 0) {
    e = cudaMemset(g->err, 0, 4 * sizeof(int32_t));
    if (e == cudaSuccess && g->ws != nullptr) e = cudaMemset(g->ws, 0, static_cast<size_t>(sk::kFlagBytes));
    if (e != cudaSuccess) return SK_ERR_CUDA;
  }
  if (device_status) *device_status = h[0];
  return h[0] == 0 ? SK_OK : SK_ERR_TIMEOUT;
}

int sk_grouped_set(sk_grouped_t g, int attr, int64_t v) {
  if (g == nullptr) return SK_ERR_INVALID;
  switch (attr) {
    case SK_ATTR_TILE_N:
    case SK_ATTR_GRID:
    case SK_ATTR_MODE: {
      // E4M3 groups: 128 (the default) or 256, single CTAs either way
      if (attr == SK_ATTR_TILE_N && g->ab_type == SK_E4M3) {
        if (v == 0) v = 128;
        if (v != 128 && v != 256) return SK_ERR_UNSUPPORTED;
      }
      const int t = g->tile_n_req, gr = g->grid_req, md = g->mode_req;
      if (attr == SK_ATTR_TILE_N) g->tile_n_req = static_cast<int>(v);
      if (attr == SK_ATTR_GRID) g->grid_req = static_cast<int>(v);
      if (attr == SK_ATTR_MODE) g->mode_req = static_cast<int>(v);
      const int st = grouped_replan(g);
      if (st != SK_OK) {
        g->tile_n_req = t;
        g->grid_req = gr;
        g->mode_req = md;
        grouped_replan(g);
      }
      return st;
    }
    case SK_ATTR_TIMEOUT_NS:
      if (v <= 0) return SK_ERR_INVALID;
      g->timeout_ns = static_cast<uint64_t>(v);
      return SK_OK;
    case SK_ATTR_PDL:
      if (v != 0 && v != 1) return SK_ERR_INVALID;
      g->pdl = v != 0;
      return SK_OK;
    case SK_ATTR_STORE:
      if (v < 0 || v > 2) return SK_ERR_INVALID;
      g->store_req = static_cast<int>(v);
      g->table_valid = false;
      return SK_OK;
    case SK_ATTR_STAGES:
      if (v != 0 && (v < 2 || v > sk::max_stages(g->plan.tile_n, g->plan.cluster_m)))
        return SK_ERR_INVALID;
      g->stages_req = static_cast<int>(v);
      return SK_OK;
    case SK_ATTR_CLUSTER_M: {
      if (v != 0 && v != 1 && v != 2) return SK_ERR_UNSUPPORTED;
      if (g->ab_type == SK_E4M3) return v == 0 || v == 1 ? SK_OK : SK_ERR_UNSUPPORTED;
      const int old = g->cluster_req;
      g->cluster_req = static_cast<int>(v);
      const int st = grouped_replan(g);
      if (st != SK_OK) {
        g->cluster_req = old;
        grouped_replan(g);
      }
      return st;
    }
    default:
      return SK_ERR_INVALID;
  }
}

int sk_grouped_get(sk_grouped_t g, int attr, int64_t* v) {
  if (g == nullptr || v == nullptr) return SK_ERR_INVALID;
  const sk::GroupPlan& gp = g->plan;
  switch (attr) {
    case SK_ATTR_MODE: *v = gp.mode; return SK_OK;
    case SK_ATTR_TILE_N: *v = gp.tile_n; return SK_OK;
    case SK_ATTR_TILE_M: *v = sk::kBlkM * gp.cluster_m; return SK_OK;
    case SK_ATTR_TILE_K: *v = gp.tile_k; return SK_OK;
    case SK_ATTR_GRID: *v = gp.grid; return SK_OK;
    case SK_ATTR_CTAS: *v = static_cast<int64_t>(gp.grid) * gp.cluster_m; return SK_OK;
    case SK_ATTR_CLUSTER_M: *v = gp.cluster_m; return SK_OK;
    case SK_ATTR_TILES: *v = gp.tiles; return SK_OK;
    case SK_ATTR_SK_TILES: *v = gp.sk_tiles; return SK_OK;
    case SK_ATTR_DP_TILES: *v = gp.tiles - gp.sk_tiles; return SK_OK;
    case SK_ATTR_WORKSPACE_BYTES: *v = gp.workspace_bytes; return SK_OK;
    case SK_ATTR_NUM_SMS: *v = g->num_sms; return SK_OK;
    case SK_ATTR_TRACE_CAP: *v = gp.max_segments; return SK_OK;
    case SK_ATTR_TRACE_INTS:
      *v = static_cast<int64_t>(gp.grid) * gp.cluster_m *
           (sk::kTraceHeaderInts + static_cast<int64_t>(gp.max_segments) * sk::kTraceRecordInts);
      return SK_OK;
    case SK_ATTR_TIMEOUT_NS: *v = static_cast<int64_t>(g->timeout_ns); return SK_OK;
    case SK_ATTR_PDL: *v = g->pdl ? 1 : 0; return SK_OK;
    case SK_ATTR_STORE: *v = g->store_req; return SK_OK;
    case SK_ATTR_SEGMENTS: *v = static_cast<int64_t>(gp.segs.size()); return SK_OK;
    case SK_ATTR_STAGES: {
      const int mx = sk::max_stages(gp.tile_n, gp.cluster_m);
      *v = g->stages_req >= 2 && g->stages_req < mx ? g->stages_req : mx;
      return SK_OK;
    }
    default: return SK_ERR_INVALID;
  }
}

int sk_grouped_schedule(sk_grouped_t g, int32_t* records, int64_t capacity, int64_t* count) {
  if (g == nullptr || count == nullptr) return SK_ERR_INVALID;
  const sk::GroupPlan& gp = g->plan;
  *count = static_cast<int64_t>(gp.segs.size());
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

}  // extern "C"

// ------------------------------------------------------------------ autotuning
namespace {

// Mean device time of `reps` launches of `launch` on `stream` (after one
// untimed launch), in microseconds; negative on a launch or device error.
template <typename F>
double time_launches(F&& launch, int reps, cudaStream_t stream) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
  double us = -1.0;
  if (launch() == SK_OK && cudaEventRecord(e0, stream) == cudaSuccess) {
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) ok = launch() == SK_OK;
    float ms = 0.0f;
    if (ok && cudaEventRecord(e1, stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
      us = 1e3 * ms / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return us;
}

int plan_autotune(sk_plan_t p, const void* A, const void* B, const float* scale_a,
                  const float* scale_b, void* C, int reps, void* stream_v, double* best_us) {
  if (p == nullptr || reps < 1) return SK_ERR_INVALID;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  const int saved[5] = {p->tile_n_req, p->cluster_req, p->mode_req, p->grid_req, p->stages_req};
  const int64_t km = p->swap ? p->n : p->m, kn = p->swap ? p->m : p->n;
  const bool f8 = p->a_type == SK_E4M3;  // BLK_N = 128 (single CTAs or pairs) or 256 (single)
  const int tns[3] = {64, 128, 256}, cms[2] = {1, 2};
  const int modes[3] = {SK_MODE_DP, SK_MODE_HYBRID, SK_MODE_SK};
  double best = -1.0;
  int bt = saved[0], bc = saved[1], bm = saved[2], bs = saved[4];
  for (int tn : tns) {
    if (tn == 256 && kn <= 128) continue;
    if (tn == 64 && f8) continue;
    for (int cm : cms) {
      if (cm == 2 && (km <= sk::kTileM || tn == 64 || (f8 && tn == 256))) continue;
      // pipeline depth: the full ring, and two or three stages
      const int mx = sk::max_stages(tn, cm);
      const int stage_opts[3] = {0, 3, 2};
      for (int md : modes) {
        for (int so : stage_opts) {
          if (so >= mx) continue;
          p->tile_n_req = tn;
          p->cluster_req = cm;
          p->mode_req = md;
          p->grid_req = 0;
          p->stages_req = so;
          if (replan(p) != SK_OK) continue;  // e.g. an attached workspace too small for it
          const double us = time_launches(
              [&] { return gemm_impl(p, A, B, scale_a, scale_b, C, 1.0f, 0.0f, nullptr, 0, stream); },
              reps, stream);
          int dev_status = 0;
          if (us < 0.0 || sk_last_error(p, &dev_status) != SK_OK) continue;
          if (best < 0.0 || us < best) {
            best = us;
            bt = tn;
            bc = cm;
            bm = md;
            bs = so;
          }
        }
      }
    }
  }
  p->tile_n_req = best < 0.0 ? saved[0] : bt;
  p->cluster_req = best < 0.0 ? saved[1] : bc;
  p->mode_req = best < 0.0 ? saved[2] : bm;
  p->grid_req = best < 0.0 ? saved[3] : 0;
  p->stages_req = best < 0.0 ? saved[4] : bs;
  const int st = replan(p);
  if (st != SK_OK) return st;
  if (best_us) *best_us = best;
  return best < 0.0 ? SK_ERR_CUDA : SK_OK;
}

int grouped_autotune(sk_grouped_t g, const void* const* A, const void* const* B,
                     const float* const* SA, const float* const* SB, void* const* C, int reps,
                     void* stream_v, double* best_us) {
  if (g == nullptr || reps < 1) return SK_ERR_INVALID;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  const int saved[5] = {g->tile_n_req, g->mode_req, g->grid_req, g->stages_req, g->cluster_req};
  const int tns[3] = {64, 128, 256}, modes[3] = {SK_MODE_DP, SK_MODE_HYBRID, SK_MODE_SK};
  const int cms[2] = {1, 2};
  const int stage_opts[3] = {0, 3, 2};
  int64_t max_m = 0;
  for (int64_t v : g->m) max_m = std::max(max_m, v);
  double best = -1.0;
  int bt = saved[0], bm = saved[1], bs = saved[3], bc = saved[4];
  for (int tn : tns) {
    if (tn == 64 && g->ab_type == SK_E4M3) continue;
    for (int cm : cms) {
      if (cm == 2 && (tn == 64 || g->ab_type == SK_E4M3 || max_m <= sk::kTileM)) continue;
      for (int md : modes) {
        for (int so : stage_opts) {
          if (so >= sk::max_stages(tn, cm)) continue;
          g->tile_n_req = tn;
          g->cluster_req = cm;
          g->mode_req = md;
          g->grid_req = 0;
          g->stages_req = so;
          if (grouped_replan(g) != SK_OK) continue;
          const double us = time_launches(
              [&] { return grouped_impl(g, A, B, SA, SB, C, nullptr, nullptr, nullptr, 0, stream); },
              reps, stream);
          int dev_status = 0;
          if (us < 0.0 || sk_grouped_last_error(g, &dev_status) != SK_OK) continue;
          if (best < 0.0 || us < best) {
            best = us;
            bt = tn;
            bc = cm;
            bm = md;
            bs = so;
          }
        }
      }
    }
  }
  g->tile_n_req = best < 0.0 ? saved[0] : bt;
  g->mode_req = best < 0.0 ? saved[1] : bm;
  g->grid_req = best < 0.0 ? saved[2] : 0;
  g->stages_req = best < 0.0 ? saved[3] : bs;
  g->cluster_req = best < 0.0 ? saved[4] : bc;
  const int st = grouped_replan(g);
  if (st != SK_OK) return st;
  if (best_us) *best_us = best;
  return best < 0.0 ? SK_ERR_CUDA : SK_OK;
}

}  // namespace

extern "C" {

int sk_plan_autotune(sk_plan_t p, const void* A, const void* B, void* C, int reps, void* stream,
                     double* best_us) {
  return plan_autotune(p, A, B, nullptr, nullptr, C, reps, stream, best_us);
}

int sk_plan_autotune_scaled(sk_plan_t p, const void* A, const void* B, const float* scale_a,
                            const float* scale_b, void* C, int reps, void* stream, double* best_us) {
  if (scale_a == nullptr || scale_b == nullptr) return SK_ERR_INVALID;
  return plan_autotune(p, A, B, scale_a, scale_b, C, reps, stream, best_us);
}

int sk_grouped_autotune(sk_grouped_t g, const void* const* A, const void* const* B, void* const* C,
                        int reps, void* stream, double* best_us) {
  return grouped_autotune(g, A, B, nullptr, nullptr, C, reps, stream, best_us);
}

int sk_grouped_autotune_scaled(sk_grouped_t g, const void* const* A, const void* const* B,
                               const float* const* SA, const float* const* SB, void* const* C,
                               int reps, void* stream, double* best_us) {
  if (SA == nullptr || SB == nullptr) return SK_ERR_INVALID;
  return grouped_autotune(g, A, B, SA, SB, C, reps, stream, best_us);
}

}  // extern "C"
