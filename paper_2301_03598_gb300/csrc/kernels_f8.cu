// Instantiations of the persistent Stream-K kernel for E4M3 operands with
// per-128 x 128-block FP32 scales, for one tile width BLK_N.  This file is
// compiled once per width with -DSK_F8_BN=<BLK_N>; each object defines
// launch_f8_bn<BLK_N>, launch_grouped_f8_bn<BLK_N> and prepare_f8_bn<BLK_N>.
// BLK_N = 128 runs on single CTAs or CTA pairs (256 x 128 tiles), BLK_N = 256
// on single CTAs (128 x 256 tiles).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>

#include "../../include/streamk.h"
#include "launch.h"
#include "sk_kernel.cuh"

#ifndef SK_F8_BN
#error "compile with -DSK_F8_BN=<tile width>"
#endif
#define SK_CAT2(a, b) a##b
#define SK_CAT(a, b) SK_CAT2(a, b)

namespace sk {

// CTA pairs (256 x 128 tiles) for BLK_N = 128 only
#define SK_F8_PAIRS (SK_F8_BN == 128)

// A kernel that rebalances registers with setmaxnreg (Cfg::kRebalance) must
// have been compiled to the launch register count its split assumes: the
// epilogue's setmaxnreg.inc waits for registers that warpgroup 0 released,
// and a split larger than the launch's allocation would wait forever.  The
// count is read once per kernel; a shortfall refuses the launch.
template <int CM, typename TC, bool GROUPED>
static cudaError_t registers_cover_rebalance() {
  using C_ = Cfg<SK_F8_BN, CM, true>;
  if constexpr (!C_::kRebalance) {
    return cudaSuccess;
  } else {
    // -1 until read; any thread may read it, all store the same value
    static std::atomic<int> ok{-1};
    int v = ok.load(std::memory_order_relaxed);
    if (v < 0) {
      cudaFuncAttributes fa;
      const cudaError_t e = cudaFuncGetAttributes(&fa, sk_gemm_kernel<SK_F8_BN, CM, TC, GROUPED, true>);
      if (e != cudaSuccess) return e;
      v = (C_::kRegsLow + 2 * C_::kRegsHigh <= 3 * fa.numRegs &&
           fa.maxThreadsPerBlock >= C_::kThreads)
              ? 1
              : 0;
      ok.store(v, std::memory_order_relaxed);
    }
    return v == 1 ? cudaSuccess : cudaErrorInvalidConfiguration;
  }
}

template <int CM, typename TC, bool GROUPED>
static cudaError_t launch_f8_one(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc,
                                 const CUtensorMap& ta3, const CUtensorMap& tb3, const SkArgs& args,
                                 bool cooperative, cudaStream_t stream) {
  const cudaError_t regs = registers_cover_rebalance<CM, TC, GROUPED>();
  if (regs != cudaSuccess) return regs;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(args.grid * CM));
  cfg.blockDim = dim3(Cfg<SK_F8_BN, CM, true>::kThreads);
  cfg.dynamicSmemBytes = Cfg<SK_F8_BN, CM, true>::kSmemBytes;
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
  return cudaLaunchKernelEx(&cfg, sk_gemm_kernel<SK_F8_BN, CM, TC, GROUPED, true>, ta, tb, tc, ta3,
                            tb3, args);
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

cudaError_t SK_CAT(launch_f8_bn, SK_F8_BN)(int c_dtype, int cluster_m, const CUtensorMap& ta,
                                           const CUtensorMap& tb, const CUtensorMap& tc,
                                           const CUtensorMap& ta3, const CUtensorMap& tb3,
                                           const SkArgs& args, bool cooperative, cudaStream_t stream) {
  if (cluster_m == 2) {
#if SK_F8_PAIRS
    return launch_f8_c<2, false>(c_dtype, ta, tb, tc, ta3, tb3, args, cooperative, stream);
#else
    return cudaErrorInvalidValue;
#endif
  }
  return launch_f8_c<1, false>(c_dtype, ta, tb, tc, ta3, tb3, args, cooperative, stream);
}

cudaError_t SK_CAT(launch_grouped_f8_bn, SK_F8_BN)(int c_dtype, const CUtensorMap& tm,
                                                   const SkArgs& args, bool cooperative,
                                                   cudaStream_t stream) {
  return launch_f8_c<1, true>(c_dtype, tm, tm, tm, tm, tm, args, cooperative, stream);
}

template <typename TC>
static cudaError_t set_smem_f8() {
  cudaError_t e = cudaFuncSetAttribute(sk_gemm_kernel<SK_F8_BN, 1, TC, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg<SK_F8_BN, 1, true>::kSmemBytes);
#if SK_F8_PAIRS
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sk_gemm_kernel<SK_F8_BN, 2, TC, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg<SK_F8_BN, 2, true>::kSmemBytes);
#endif
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sk_gemm_kernel<SK_F8_BN, 1, TC, true, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Cfg<SK_F8_BN, 1, true>::kSmemBytes);
}

cudaError_t SK_CAT(prepare_f8_bn, SK_F8_BN)(size_t* smem_bytes) {
  cudaError_t e;
  if ((e = set_smem_f8<float>()) != cudaSuccess) return e;
  if ((e = set_smem_f8<__nv_bfloat16>()) != cudaSuccess) return e;
  if ((e = set_smem_f8<__half>()) != cudaSuccess) return e;
  *smem_bytes = static_cast<size_t>(Cfg<SK_F8_BN, 1, true>::kSmemBytes);
  return cudaSuccess;
}

}  // namespace sk
