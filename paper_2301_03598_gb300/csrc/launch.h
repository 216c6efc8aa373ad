// Kernel launchers, one object per BLK_N (64, 128, 256) and one per E4M3 BLK_N (128, 256).
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
// BLK_N = 128 on single CTAs or CTA pairs (cluster_m 2, 256 x 128 tiles), or
// BLK_N = 256 on single CTAs (128 x 256 tiles; cluster_m 2 returns
// cudaErrorInvalidValue).  The operand maps view the rows as 16-bit elements
// (k/2 per row), 2-D and 3-D as for the 16-bit kernels of the same width.
cudaError_t launch_f8_bn128(int c_dtype, int cluster_m, const CUtensorMap& ta, const CUtensorMap& tb,
                            const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                            const SkArgs& args, bool cooperative, cudaStream_t stream);
cudaError_t launch_f8_bn256(int c_dtype, int cluster_m, const CUtensorMap& ta, const CUtensorMap& tb,
                            const CUtensorMap& tc, const CUtensorMap& ta3, const CUtensorMap& tb3,
                            const SkArgs& args, bool cooperative, cudaStream_t stream);
cudaError_t launch_grouped_f8_bn128(int c_dtype, const CUtensorMap& tm, const SkArgs& args,
                                    bool cooperative, cudaStream_t stream);
cudaError_t launch_grouped_f8_bn256(int c_dtype, const CUtensorMap& tm, const SkArgs& args,
                                    bool cooperative, cudaStream_t stream);
inline cudaError_t launch_f8(int c_dtype, int tile_n, int cluster_m, const CUtensorMap& ta,
                             const CUtensorMap& tb, const CUtensorMap& tc, const CUtensorMap& ta3,
                             const CUtensorMap& tb3, const SkArgs& args, bool cooperative,
                             cudaStream_t stream) {
  if (tile_n == 256)
    return launch_f8_bn256(c_dtype, cluster_m, ta, tb, tc, ta3, tb3, args, cooperative, stream);
  if (tile_n == 128)
    return launch_f8_bn128(c_dtype, cluster_m, ta, tb, tc, ta3, tb3, args, cooperative, stream);
  return cudaErrorInvalidValue;
}
inline cudaError_t launch_grouped_f8(int c_dtype, int tile_n, const CUtensorMap& tm,
                                     const SkArgs& args, bool cooperative, cudaStream_t stream) {
  if (tile_n == 256) return launch_grouped_f8_bn256(c_dtype, tm, args, cooperative, stream);
  if (tile_n == 128) return launch_grouped_f8_bn128(c_dtype, tm, args, cooperative, stream);
  return cudaErrorInvalidValue;
}
// Dynamic shared memory of one CTA; also sets the kernels' opt-in limit.
cudaError_t prepare_bn64(size_t* smem_bytes);
cudaError_t prepare_bn128(size_t* smem_bytes);
cudaError_t prepare_bn256(size_t* smem_bytes);
cudaError_t prepare_f8_bn128(size_t* smem_bytes);
cudaError_t prepare_f8_bn256(size_t* smem_bytes);
// Both E4M3 widths; the larger of their shared-memory sizes.
inline cudaError_t prepare_f8(size_t* smem_bytes) {
  size_t a = 0, b = 0;
  cudaError_t e = prepare_f8_bn128(&a);
  if (e == cudaSuccess) e = prepare_f8_bn256(&b);
  *smem_bytes = a > b ? a : b;
  return e;
}

}  // namespace sk
