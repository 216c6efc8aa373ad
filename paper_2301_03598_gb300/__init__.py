"""GB300-native (sm_103a) Stream-K GEMM library.

C = alpha * A * B + beta * C with the work-centric Stream-K decomposition of
Osama et al. (arXiv 2301.03598): hand-written tcgen05/TMA CUDA kernels behind
the C ABI of include/streamk.h, with a thin Python binding in ``streamk``.

Importing the package loads nothing; the first call into ``streamk`` loads
libstreamk.so and raises if it has not been built (``build.build()``).
"""
__all__ = ["streamk", "inputs", "build"]
