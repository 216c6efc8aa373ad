// Instantiations of the persistent Stream-K kernel for one tile width BLK_N.
// This file is compiled once per tile width with -DSK_BN=<BLK_N>; each object
// defines launch_bn<BLK_N>, launch_grouped_bn<BLK_N> and prepare_bn<BLK_N>.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/streamk.h"
#include "launch.h"
#include "planner.h"
#include "sk_kernel.cuh"

#ifndef SK_BN
#error "compile with -DSK_BN=<tile width>"
#endif
#define SK_CAT2(a, b) a##b
#define SK_CAT(a, b) SK_CAT2(a, b)

namespace sk {

template <int CM, typename TC>
static cudaError_t launch_one(const CUtensorMap& ta, const CUtensorMap& tb,
                              const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                              const SkArgs& args, bool cooperative, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(args.grid * CM));
  cfg.blockDim = dim3(Cfg<SK_BN, CM>::kThreads);
  cfg.dynamicSmemBytes = Cfg<SK_BN, CM>::kSmemBytes;
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
  return cudaLaunchKernelEx(&cfg, sk_gemm_kernel<SK_BN, CM, TC, false, false>, ta, tb, tc, ta3, tb3, args);
}

template <int CM>
static cudaError_t launch_cm(int c_dtype, const CUtensorMap& ta, const CUtensorMap& tb,
                             const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                             const SkArgs& args, bool cooperative, cudaStream_t stream) {
  switch (c_dtype) {
    case SK_F32:
      return launch_one<CM, float>(ta, tb, tc, ta3, tb3, args, cooperative, stream);
    case SK_BF16:
      return launch_one<CM, __nv_bfloat16>(ta, tb, tc, ta3, tb3, args, cooperative, stream);
    case SK_F16:
      return launch_one<CM, __half>(ta, tb, tc, ta3, tb3, args, cooperative, stream);
    default:
      return cudaErrorInvalidValue;
  }
}

// BLK_N = 64 tiles (the narrow configuration for shapes with few tiles) run on
// single CTAs only.
constexpr bool kPairs = SK_BN != 64;
static_assert(Cfg<SK_BN, 1>::kStages == max_stages(SK_BN, 1) &&
                  (!kPairs || Cfg<SK_BN, 2>::kStages == max_stages(SK_BN, 2)),
              "the host's stage count matches the kernel's ring");

template <bool kWithPairs>
static cudaError_t launch_any(int c_dtype, int cluster_m, const CUtensorMap& ta, const CUtensorMap& tb,
                              const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                              const SkArgs& args, bool cooperative, cudaStream_t stream) {
  if (cluster_m == 2) {
    if constexpr (kWithPairs)
      return launch_cm<2>(c_dtype, ta, tb, tc, ta3, tb3, args, cooperative, stream);
    else
      return cudaErrorInvalidValue;
  }
  return launch_cm<1>(c_dtype, ta, tb, tc, ta3, tb3, args, cooperative, stream);
}

cudaError_t SK_CAT(launch_bn, SK_BN)(int c_dtype, int cluster_m, const CUtensorMap& ta, const CUtensorMap& tb,
                         const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                         const SkArgs& args, bool cooperative, cudaStream_t stream) {
  return launch_any<kPairs>(c_dtype, cluster_m, ta, tb, tc, ta3, tb3, args, cooperative, stream);
}

// Grouped launches: the walk table and problem table in args (the
// tensor-map parameters are not read); single CTAs or CTA pairs.
template <int CM, typename TC>
static cudaError_t launch_grouped_one(const CUtensorMap& tm, const SkArgs& args, bool cooperative,
                                      cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(args.grid * CM));
  cfg.blockDim = dim3(Cfg<SK_BN, CM>::kThreads);
  cfg.dynamicSmemBytes = Cfg<SK_BN, CM>::kSmemBytes;
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
  return cudaLaunchKernelEx(&cfg, sk_gemm_kernel<SK_BN, CM, TC, true, false>, tm, tm, tm, tm, tm, args);
}

template <int CM>
static cudaError_t launch_grouped_cm(int c_dtype, const CUtensorMap& tm, const SkArgs& args,
                                     bool cooperative, cudaStream_t stream) {
  switch (c_dtype) {
    case SK_F32:
      return launch_grouped_one<CM, float>(tm, args, cooperative, stream);
    case SK_BF16:
      return launch_grouped_one<CM, __nv_bfloat16>(tm, args, cooperative, stream);
    case SK_F16:
      return launch_grouped_one<CM, __half>(tm, args, cooperative, stream);
    default:
      return cudaErrorInvalidValue;
  }
}

template <bool kWithPairs>
static cudaError_t launch_grouped_any(int c_dtype, int cluster_m, const CUtensorMap& tm,
                                      const SkArgs& args, bool cooperative, cudaStream_t stream) {
  if (cluster_m == 2) {
    if constexpr (kWithPairs)
      return launch_grouped_cm<2>(c_dtype, tm, args, cooperative, stream);
    else
      return cudaErrorInvalidValue;
  }
  return launch_grouped_cm<1>(c_dtype, tm, args, cooperative, stream);
}

cudaError_t SK_CAT(launch_grouped_bn, SK_BN)(int c_dtype, int cluster_m, const CUtensorMap& tm,
                                             const SkArgs& args, bool cooperative,
                                             cudaStream_t stream) {
  return launch_grouped_any<kPairs>(c_dtype, cluster_m, tm, args, cooperative, stream);
}

template <int CM, typename TC>
static cudaError_t set_smem() {
  cudaError_t e = cudaFuncSetAttribute(sk_gemm_kernel<SK_BN, CM, TC, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg<SK_BN, CM>::kSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sk_gemm_kernel<SK_BN, CM, TC, true, false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<SK_BN, CM>::kSmemBytes);
}

template <bool kWithPairs>
static cudaError_t prepare_all() {
  cudaError_t e;
  if ((e = set_smem<1, float>()) != cudaSuccess) return e;
  if ((e = set_smem<1, __nv_bfloat16>()) != cudaSuccess) return e;
  if ((e = set_smem<1, __half>()) != cudaSuccess) return e;
  if constexpr (kWithPairs) {
    if ((e = set_smem<2, float>()) != cudaSuccess) return e;
    if ((e = set_smem<2, __nv_bfloat16>()) != cudaSuccess) return e;
    if ((e = set_smem<2, __half>()) != cudaSuccess) return e;
    static_assert(!kWithPairs || Cfg<SK_BN, 1>::kSmemBytes == Cfg<SK_BN, 2>::kSmemBytes,
                  "one size for both");
  }
  return cudaSuccess;
}

cudaError_t SK_CAT(prepare_bn, SK_BN)(size_t* smem_bytes) {
  const cudaError_t e = prepare_all<kPairs>();
  if (e != cudaSuccess) return e;
  *smem_bytes = static_cast<size_t>(Cfg<SK_BN, 1>::kSmemBytes);
  return cudaSuccess;
}

}  // namespace sk
