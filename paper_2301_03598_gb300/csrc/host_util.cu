// Host helpers shared by the C ABI's translation units: TMA descriptor
// encoding, the MMA instruction descriptor, launch epochs, status mapping.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "../../include/streamk.h"
#include "host_util.h"
#include "sk_args.h"

namespace sk {
namespace host {

// Launch epochs are unique per process, so flags left in a workspace by any
// earlier launch (of any plan sharing it) never match a later launch.
static std::atomic<uint32_t> g_epoch{0};

uint32_t next_epoch() {
  uint32_t e = g_epoch.fetch_add(1, std::memory_order_relaxed) + 1;
  while (e == 0) e = g_epoch.fetch_add(1, std::memory_order_relaxed) + 1;
  return e;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

size_t dtype_size(int t) { return t == SK_F32 ? 4 : t == SK_E4M3 ? 1 : 2; }


int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SK_OK;
  if (e == cudaErrorMemoryAllocation) return SK_ERR_NOMEM;
  return SK_ERR_CUDA;
}

int encode_operand(CUtensorMap* tm, const void* ptr, int dtype, int64_t rows, int64_t kdim,
                   int64_t ld, int box_rows) {
  auto fn = encode_fn();
  if (fn == nullptr) return SK_ERR_CUDA;
  const int64_t esz = static_cast<int64_t>(dtype_size(dtype));
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(kdim), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * esz)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / esz), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUtensorMapDataType dt = dtype == SK_BF16   ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                           : dtype == SK_E4M3 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUresult r = fn(tm, dt, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SK_OK : SK_ERR_INVALID;
}

// The same operand viewed as {64, rows, k/64} with strides {ld, 128 B}: one
// box {64, box_rows, 2} holds two consecutive 64-wide k-blocks.  Only the
// k-blocks that lie entirely inside k are addressed through this view (the
// innermost extent is 64 regardless of k); the kernel loads a tail k-block
// through the 2-D map, which fills columns beyond k with zeros.
int encode_operand_3d(CUtensorMap* tm, const void* ptr, int dtype, int64_t rows, int64_t kdim,
                      int64_t ld, int box_rows) {
  auto fn = encode_fn();
  if (fn == nullptr) return SK_ERR_CUDA;
  const int64_t kfull = kdim / sk::kBlkK;
  if (kfull < 2) return SK_ERR_INVALID;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(sk::kBlkK), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(kfull)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld) * 2, static_cast<cuuint64_t>(sk::kBlkK) * 2};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(sk::kBlkK), static_cast<cuuint32_t>(box_rows), 2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMapDataType dt =
      dtype == SK_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUresult r = fn(tm, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SK_OK : SK_ERR_INVALID;
}

// Tensor map of the output for TMA stores: rows x cols (cols contiguous),
// boxes of 32 rows x 128 bytes, 128-byte swizzle (the epilogue's staging
// layout).  Returns false when the layout cannot be stored by TMA.
bool encode_output(CUtensorMap* tm, void* ptr, int c_type, int64_t rows, int64_t cols, int64_t ld) {
  auto fn = encode_fn();
  const int64_t esz = static_cast<int64_t>(dtype_size(c_type));
  if (fn == nullptr || (reinterpret_cast<uintptr_t>(ptr) & 15u) || (ld * esz) % 16 != 0) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * esz)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / esz), 32};
  cuuint32_t estr[2] = {1, 1};
  CUtensorMapDataType dt = c_type == SK_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                           : c_type == SK_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUresult r = fn(tm, dt, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}


// The epilogue's store path for an aligned C (SkArgs::c_tma): the requested
// one, else the default.
int store_path(int req) { return req == 1 ? 1 : req == 2 ? 2 : 1; }

// tcgen05 kind::f16 / kind::f8f6f4 instruction descriptor: FP32
// accumulator, A/B format (F16 0 / BF16 1; E4M3 0),
// both operands K-major, N >> 3 at bit 17, M >> 4 at bit 24.
uint32_t make_idesc(int in_dtype, int tile_n, int cluster_m) {
  const uint32_t fmt = in_dtype == SK_BF16 ? 1u : 0u;
  uint32_t d = 0;
  d |= 1u << 4;                                         // D: F32
  d |= fmt << 7;                                        // A: F16 / BF16
  d |= fmt << 10;                                       // B: F16 / BF16
  d |= static_cast<uint32_t>(tile_n >> 3) << 17;        // N
  d |= static_cast<uint32_t>((sk::kBlkM * cluster_m) >> 4) << 24;  // M (256 for a CTA pair)
  return d;
}



static bool capturing(cudaStream_t stream, bool* ok) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  *ok = cudaStreamIsCapturing(stream, &cs) == cudaSuccess;
  return cs != cudaStreamCaptureStatusNone;
}

int busy_check(const InFlight& f, cudaStream_t stream) {
  if (!f.recorded || f.stream == stream) return SK_OK;  // stream order covers one stream
  // No event query while the stream is being captured (a graph node is not a
  // launch yet, and the query is not allowed under global capture).
  bool ok = true;
  if (capturing(stream, &ok)) return SK_OK;
  if (!ok) return SK_ERR_CUDA;
  const cudaError_t e = cudaEventQuery(f.done);
  if (e == cudaSuccess) return SK_OK;
  if (e == cudaErrorNotReady) {
    cudaGetLastError();  // a query that is not ready leaves no sticky error; clear it anyway
    return SK_ERR_BUSY;
  }
  return cuda_status(e);
}

int busy_record(InFlight& f, cudaStream_t stream) {
  bool ok = true;
  if (capturing(stream, &ok)) return SK_OK;  // a graph node: not tracked
  if (!ok) return SK_ERR_CUDA;
  if (f.done == nullptr) {
    const cudaError_t e = cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
  }
  const cudaError_t e = cudaEventRecord(f.done, stream);
  if (e != cudaSuccess) return cuda_status(e);
  f.stream = stream;
  f.recorded = true;
  return SK_OK;
}

void busy_release(InFlight& f) {
  if (f.done != nullptr) cudaEventDestroy(f.done);
  f = InFlight{};
}

}  // namespace host
}  // namespace sk
