// Host helpers shared by the C ABI's translation units (host_util.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstddef>
#include <cstdint>

#include "../../include/streamk.h"

namespace sk {
namespace host {

constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;  // 2 s per device-side wait

// A launch epoch unique in this process (never 0).
uint32_t next_epoch();
// cuTensorMapEncodeTiled from the driver, or nullptr.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();
size_t dtype_size(int t);
int cuda_status(cudaError_t e);
// 2-D map of a K-contiguous operand (rows x kdim, pitch ld elements), boxes of
// one k-block (128 bytes: 64 16-bit or 128 E4M3 elements) x box_rows rows,
// 128-byte swizzle.
int encode_operand(CUtensorMap* tm, const void* ptr, int dtype, int64_t rows, int64_t kdim,
                   int64_t ld, int box_rows);
// 3-D view {64, rows, k/64} of the same operand: boxes of two k-blocks.
int encode_operand_3d(CUtensorMap* tm, const void* ptr, int dtype, int64_t rows, int64_t kdim,
                      int64_t ld, int box_rows);
// Output map for TMA stores; false when C cannot be stored by TMA.
bool encode_output(CUtensorMap* tm, void* ptr, int c_type, int64_t rows, int64_t cols, int64_t ld);
// The epilogue store path for an aligned C (SkArgs::c_tma) for a request.
int store_path(int req);
// tcgen05 instruction descriptor (kind::f16, or kind::f8f6f4 for E4M3).
uint32_t make_idesc(int in_dtype, int tile_n, int cluster_m);

// A plan's last launch, for refusing a launch on another stream while it is
// still running (SK_ERR_BUSY): both would use the plan's one workspace.
// Launches issued while their stream is being captured are not tracked.
struct InFlight {
  cudaEvent_t done = nullptr;   // recorded after each tracked launch
  cudaStream_t stream = nullptr;
  bool recorded = false;
};
// SK_OK, SK_ERR_BUSY (the last tracked launch runs on a stream other than
// `stream` and has not finished) or SK_ERR_CUDA.
int busy_check(const InFlight& f, cudaStream_t stream);
// Note a launch just issued on `stream` (creates the event on first use).
int busy_record(InFlight& f, cudaStream_t stream);
void busy_release(InFlight& f);

}  // namespace host

// sk_gemm / sk_gemm_scaled (scales null for 16-bit plans) whose launch also
// stores a device failure status into err_host (a device pointer to mapped
// pinned host memory, or nullptr).
int gemm_reporting(sk_plan_t p, const void* A, const void* B, const float* scale_a,
                   const float* scale_b, void* C, float alpha, float beta, void* stream,
                   int32_t* err_host);
}  // namespace sk
