// Kernel launchers, one object per BLK_N (64, 128, 256) and one for E4M3.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "sk_args.h"

namespace sk {

// c_dtype: SK_F32 / SK_BF16 / SK_F16.  cluster_m: 1, or 2 for CTA pairs along M
// (the grid is args.grid units of cluster_m CTAs).  ta/tb: 2-D operand maps
// (boxes of one 64-wide k-block); ta3/tb3: the 3-D views whose boxes hold two
// k-blocks, used by BLK_N = 64 and 128 (pass the 2-D maps when unused).
// cooperative: CTAs wait on one another, so the launch must guarantee
// co-residency.
// BLK_N = 64: single CTAs only (cluster_m 2 returns cudaErrorInvalidValue).
cudaError_t launch_bn64(int c_dtype, int cluster_m, const CUtensorMap& ta, const CUtensorMap& tb,
                        const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                        const SkArgs& args, bool cooperative, cudaStream_t stream);
cudaError_t launch_bn128(int c_dtype, int cluster_m, const CUtensorMap& ta, const CUtensorMap& tb,
                         const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                         const SkArgs& args, bool cooperative, cudaStream_t stream);
cudaError_t launch_bn256(int c_dtype, int cluster_m, const CUtensorMap& ta, const CUtensorMap& tb,
                         const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                         const SkArgs& args, bool cooperative, cudaStream_t stream);
// A grouped launch (args.grid units of cluster_m CTAs walking args.gwalk; CTA
// pairs for BLK_N 128 and 256 only); tm is any valid tensor map (the kernel's
// tensor-map parameters are unused there).
cudaError_t launch_grouped_bn64(int c_dtype, int cluster_m, const CUtensorMap& tm, const SkArgs& args,
                                bool cooperative, cudaStream_t stream);
cudaError_t launch_grouped_bn128(int c_dtype, int cluster_m, const CUtensorMap& tm,
                                 const SkArgs& args, bool cooperative, cudaStream_t stream);
cudaError_t launch_grouped_bn256(int c_dtype, int cluster_m, const CUtensorMap& tm,
                                 const SkArgs& args, bool cooperative, cudaStream_t stream);
// E4M3 operands with per-128 x 128-block scales (args.scale_a / scale_b):
// BLK_N = 128, single CTAs or CTA pairs (cluster_m 2, 256 x 128 tiles).  The
// operand maps view the rows as 16-bit elements (k/2 per row), 2-D and 3-D as
// for the 16-bit BLK_N = 128 kernels.
cudaError_t launch_f8(int c_dtype, int cluster_m, const CUtensorMap& ta, const CUtensorMap& tb,
                      const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                      const SkArgs& args, bool cooperative, cudaStream_t stream);
cudaError_t launch_grouped_f8(int c_dtype, const CUtensorMap& tm, const SkArgs& args,
                              bool cooperative, cudaStream_t stream);
// Dynamic shared memory of one CTA; also sets the kernels' opt-in limit.
cudaError_t prepare_bn64(size_t* smem_bytes);
cudaError_t prepare_bn128(size_t* smem_bytes);
cudaError_t prepare_bn256(size_t* smem_bytes);
cudaError_t prepare_f8(size_t* smem_bytes);

}  // namespace sk
