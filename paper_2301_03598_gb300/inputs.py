"""Seeded synthetic inputs for the Stream-K GEMM library.

This module is the one piece shared by the oracle side and the GPU side: it
draws random matrices and shape lists and stores them in the input formats.
It holds none of the GEMM's arithmetic.  Workload recipes follow the paper's
evaluation corpus (Section 6: m, n, k log-sampled in [128, 8192]) and the
synthetic stand-ins named in the repository's design notes.

Random values are drawn in float32 by numpy's PCG64 (host) or by torch's
Philox generator (device pools), then rounded to the storage format by the
library conversions (numpy float16 cast / torch bfloat16 cast, both
round-to-nearest-even).  The float64 copy returned beside a host matrix holds
exactly the stored values, since FP16 and BF16 widen to FP64 without error.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
import torch

DTYPES = {"f16": torch.float16, "bf16": torch.bfloat16, "f32": torch.float32}


def _draw(rng: np.random.Generator, shape, dist: str) -> np.ndarray:
    if dist == "uniform":          # U[-1, 1]
        return rng.uniform(-1.0, 1.0, size=shape).astype(np.float32)
    if dist == "normal":           # N(0, 1)
        return rng.standard_normal(size=shape, dtype=np.float32)
    if dist == "ones":
        return np.ones(shape, np.float32)
    if dist == "smallint":         # integers in [-4, 4]: exact in every format
        return rng.integers(-4, 5, size=shape).astype(np.float32)
    raise ValueError(f"unknown distribution {dist!r}")


def to_storage(values_f32: np.ndarray, dtype: str) -> torch.Tensor:
    """Round float32 values to the storage dtype (RN-even), as a CPU tensor."""
    t = torch.from_numpy(np.ascontiguousarray(values_f32, dtype=np.float32))
    return t.to(DTYPES[dtype]).contiguous()


def widen(t: torch.Tensor) -> np.ndarray:
    """Exact float64 copy of a CPU tensor of FP16 / BF16 / FP32 values."""
    return t.to(torch.float64).numpy()


def host_matrix(rows: int, cols: int, dtype: str, dist: str, seed: int):
    """A rows x cols matrix (row-major storage tensor on the CPU) and the exact
    float64 values it holds."""
    rng = np.random.Generator(np.random.PCG64(seed))
    stor = to_storage(_draw(rng, (rows, cols), dist), dtype)
    return stor, widen(stor)


def device_pool(numel: int, dtype: str, dist: str, seed: int, device) -> torch.Tensor:
    """A flat device tensor of ``numel`` seeded values in ``dtype`` (Philox on
    the device; used where host generation of gigabytes would be too slow)."""
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = torch.empty(numel, dtype=DTYPES[dtype], device=device)
    chunk = 1 << 28
    for s in range(0, numel, chunk):
        e = min(numel, s + chunk)
        if dist == "normal":
            v = torch.randn(e - s, generator=gen, device=device, dtype=torch.float32)
        elif dist == "uniform":
            v = torch.rand(e - s, generator=gen, device=device, dtype=torch.float32) * 2 - 1
        else:
            raise ValueError(dist)
        out[s:e] = v.to(out.dtype)
    return out


def e4m3_quantize(x: torch.Tensor):
    """Block-scaled E4M3 storage of a float32 matrix (any device): one FP32
    scale per 128 x 128 block, amax / 448 (1 for an all-zero block), and the
    codes of x / scale rounded by torch's float8_e4m3fn conversion (RN-even;
    |x / scale| <= 448 by construction).  Returns (codes uint8 rows x cols,
    scales float32 [ceil(rows/128), ceil(cols/128)])."""
    rows, cols = x.shape
    nbr, nbc = -(-rows // 128), -(-cols // 128)
    pad = torch.zeros(nbr * 128, nbc * 128, dtype=torch.float32, device=x.device)
    pad[:rows, :cols] = x
    amax = pad.abs().view(nbr, 128, nbc, 128).amax(dim=(1, 3))
    scales = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax))
    full = scales.repeat_interleave(128, 0).repeat_interleave(128, 1)[:rows, :cols]
    codes = (x / full).to(torch.float8_e4m3fn).view(torch.uint8).contiguous()
    return codes, scales.contiguous()


def host_e4m3_matrix(rows: int, cols: int, dist: str, seed: int):
    """A rows x cols block-scaled E4M3 operand on the CPU: (codes, scales),
    values drawn as in ``host_matrix`` before quantisation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return e4m3_quantize(torch.from_numpy(_draw(rng, (rows, cols), dist)))


def device_e4m3_matrix(rows: int, cols: int, seed: int, device, dist: str = "normal"):
    """The same drawn on the device (Philox), for operands too large to make
    on the host: (codes, scales) device tensors."""
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    if dist == "normal":
        x = torch.randn(rows, cols, generator=gen, device=device, dtype=torch.float32)
    elif dist == "uniform":
        x = torch.rand(rows, cols, generator=gen, device=device, dtype=torch.float32) * 2 - 1
    else:
        raise ValueError(dist)
    return e4m3_quantize(x)


def log_uniform_shapes(count: int, seed: int, lo: int = 128, hi: int = 8192,
                       multiple: int = 16) -> List[Tuple[int, int, int]]:
    """``count`` shapes (m, n, k), each drawn log-uniform in [lo, hi] and rounded
    to the nearest multiple of ``multiple`` (at least ``multiple``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    logs = rng.uniform(math.log(lo), math.log(hi), size=(count, 3))
    vals = np.maximum(multiple, np.rint(np.exp(logs) / multiple).astype(np.int64) * multiple)
    return [tuple(int(v) for v in row) for row in vals]


# The shape-sweep workload: 2,000 single BF16 GEMMs with m, n, k log-uniform
# in [128, 8192], multiples of 16.
SWEEP_SEED = 2301_03598 + 2
SWEEP_COUNT = 2000


def sweep_shapes(count: int = SWEEP_COUNT, seed: int = SWEEP_SEED):
    return log_uniform_shapes(count, seed)


# Extreme-quantisation shapes (m, n, k): square, deep-K skinny, tall-skinny,
# and a tile count near the SM count.
EXTREME_SHAPES = [(8192, 8192, 8192), (256, 256, 65536), (8192, 128, 4096), (1536, 1536, 1536)]


# The grouped workload: 256 problems in one launch, m log-uniform in [16, 4096]
# (rounded to a multiple of 16), n and k drawn uniformly from {1024, 2048,
# 4096, 8192}.
GROUPED_SEED = 2301_03598 + 4
GROUPED_COUNT = 256


def grouped_shapes(count: int = GROUPED_COUNT, seed: int = GROUPED_SEED):
    rng = np.random.Generator(np.random.PCG64(seed))
    ms = np.maximum(16, np.rint(np.exp(rng.uniform(math.log(16), math.log(4096), size=count))
                                / 16).astype(np.int64) * 16)
    choices = np.array([1024, 2048, 4096, 8192])
    ns = rng.choice(choices, size=count)
    ks = rng.choice(choices, size=count)
    return [(int(m), int(n), int(k)) for m, n, k in zip(ms, ns, ks)]
