// Instantiations of the persistent Stream-K kernel for BLK_N = 128.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/streamk.h"
#include "launch.h"
#include "sk_kernel.cuh"

namespace sk {

template <typename TC>
static cudaError_t launch_one(const CUtensorMap& ta, const CUtensorMap& tb,
                              const CUtensorMap& tc, const SkArgs& args,
                              bool cooperative, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(args.grid));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = Cfg<128>::kSmemBytes;
  cfg.stream = stream;
  cudaLaunchAttribute attr[2];
  unsigned na = 0;
  if (cooperative) {
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    ++na;
  }
  if (args.pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, sk_gemm_kernel<128, TC>, ta, tb, tc, args);
}

cudaError_t launch_bn128(int c_dtype, const CUtensorMap& ta, const CUtensorMap& tb,
                         const CUtensorMap& tc, const SkArgs& args, bool cooperative,
                         cudaStream_t stream) {
  switch (c_dtype) {
    case SK_F32:
      return launch_one<float>(ta, tb, tc, args, cooperative, stream);
    case SK_BF16:
      return launch_one<__nv_bfloat16>(ta, tb, tc, args, cooperative, stream);
    case SK_F16:
      return launch_one<__half>(ta, tb, tc, args, cooperative, stream);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_bn128(size_t* smem_bytes) {
  const int bytes = Cfg<128>::kSmemBytes;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(sk_gemm_kernel<128, float>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(sk_gemm_kernel<128, __nv_bfloat16>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(sk_gemm_kernel<128, __half>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  *smem_bytes = static_cast<size_t>(bytes);
  return cudaSuccess;
}

}  // namespace sk
