// Instantiations of the persistent Stream-K kernel for E4M3 operands with
// per-128 x 128-block FP32 scales: BLK_N = 128 on single CTAs or CTA pairs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/streamk.h"
#include "launch.h"
#include "sk_kernel.cuh"

namespace sk {

template <int CM, typename TC, bool GROUPED>
static cudaError_t launch_f8_one(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc,
                                 const CUtensorMap& ta3, const CUtensorMap& tb3, const SkArgs& args,
                                 bool cooperative, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(args.grid * CM));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = Cfg<128, CM, true>::kSmemBytes;
  cfg.stream = stream;
  cudaLaunchAttribute attr[3];
  unsigned na = 0;
  if (CM > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = CM;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
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
  return cudaLaunchKernelEx(&cfg, sk_gemm_kernel<128, CM, TC, GROUPED, true>, ta, tb, tc, ta3, tb3,
                            args);
}

template <int CM, bool GROUPED>
static cudaError_t launch_f8_c(int c_dtype, const CUtensorMap& ta, const CUtensorMap& tb,
                               const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                               const SkArgs& args, bool cooperative, cudaStream_t stream) {
  switch (c_dtype) {
    case SK_F32:
      return launch_f8_one<CM, float, GROUPED>(ta, tb, tc, ta3, tb3, args, cooperative, stream);
    case SK_BF16:
      return launch_f8_one<CM, __nv_bfloat16, GROUPED>(ta, tb, tc, ta3, tb3, args, cooperative, stream);
    case SK_F16:
      return launch_f8_one<CM, __half, GROUPED>(ta, tb, tc, ta3, tb3, args, cooperative, stream);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_f8(int c_dtype, int cluster_m, const CUtensorMap& ta, const CUtensorMap& tb,
                      const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                      const SkArgs& args, bool cooperative, cudaStream_t stream) {
  return cluster_m == 2
             ? launch_f8_c<2, false>(c_dtype, ta, tb, tc, ta3, tb3, args, cooperative, stream)
             : launch_f8_c<1, false>(c_dtype, ta, tb, tc, ta3, tb3, args, cooperative, stream);
}

cudaError_t launch_grouped_f8(int c_dtype, const CUtensorMap& tm, const SkArgs& args,
                              bool cooperative, cudaStream_t stream) {
  return launch_f8_c<1, true>(c_dtype, tm, tm, tm, tm, tm, args, cooperative, stream);
}

template <typename TC>
static cudaError_t set_smem_f8() {
  cudaError_t e = cudaFuncSetAttribute(sk_gemm_kernel<128, 1, TC, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg<128, 1, true>::kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sk_gemm_kernel<128, 2, TC, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<128, 2, true>::kSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sk_gemm_kernel<128, 1, TC, true, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Cfg<128, 1, true>::kSmemBytes);
}

cudaError_t prepare_f8(size_t* smem_bytes) {
  cudaError_t e;
  if ((e = set_smem_f8<float>()) != cudaSuccess) return e;
  if ((e = set_smem_f8<__nv_bfloat16>()) != cudaSuccess) return e;
  if ((e = set_smem_f8<__half>()) != cudaSuccess) return e;
  *smem_bytes = static_cast<size_t>(Cfg<128, 1, true>::kSmemBytes);
  return cudaSuccess;
}

}  // namespace sk
