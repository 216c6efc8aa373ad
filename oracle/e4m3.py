"""Oracle for block-scaled E4M3 GEMMs.  TEST INFRASTRUCTURE ONLY.

The library's E4M3 path multiplies A (m x k) and B (n x k, i.e. B^T of a
k x n operand) stored as 8-bit E4M3 codes, each 128 x 128 block of either
operand carrying one FP32 scale: the operand's value at (r, l) is
scale[r // 128][l // 128] * decode(code[r][l]).  The paper fixes no 8-bit
format (its evaluation is FP16 -> FP32 and FP64, Section 6); this is the
operand model of the library's E4M3 entry points, and the oracle computes
the GEMM of those values exactly as defined:

    C = alpha * Adq @ Bdq^T + beta * C_in,   Adq = dequantize(qA, sA), ...

in FP64 by the same plain GEMM as the 16-bit path (``oracle.gemm``).  Every
dequantized value is exact in FP64 (a 4-bit significand times an FP32 scale).

``decode`` follows the OCP 8-bit floating point specification (E4M3: sign
bit, 4 exponent bits with bias 7, 3 mantissa bits; exponent field 0 encodes
subnormals f * 2^-9; no infinities; S.1111.111 is NaN; the largest finite
magnitude is 1.75 * 2^8 = 448).
"""
from __future__ import annotations

import numpy as np

BLOCK = 128     # scale block edge along rows and along k
MAX_FINITE = 448.0


def decode(codes) -> np.ndarray:
    """float64 value of every E4M3 code (uint8 array of any shape)."""
    c = np.asarray(codes, dtype=np.uint8).astype(np.int64)
    sign = np.where(c >> 7, -1.0, 1.0)
    e = (c >> 3) & 0xF
    f = c & 0x7
    mag = np.where(e == 0, f * 2.0 ** -9, (1.0 + f / 8.0) * np.exp2(e - 7.0))
    out = sign * mag
    return np.where((e == 15) & (f == 7), np.nan, out)


def dequantize_rows(codes, row_scales) -> np.ndarray:
    """Exact float64 values of r rows taken from an E4M3 operand: ``codes`` is
    r x cols, and row i of ``row_scales`` [r, ceil(cols/128)] is the scale row
    of the 128-row block that row i came from."""
    q = decode(codes)
    s = np.asarray(row_scales, dtype=np.float64)
    rows, cols = q.shape
    if s.shape != (rows, -(-cols // BLOCK)):
        raise ValueError(f"row scales shape {s.shape}, expected {(rows, -(-cols // BLOCK))}")
    return q * np.repeat(s, BLOCK, axis=1)[:, :cols]


def dequantize(codes, scales) -> np.ndarray:
    """Exact float64 values of a rows x cols E4M3 operand whose 128 x 128
    blocks carry the FP32 scales ``scales`` [ceil(rows/128), ceil(cols/128)]."""
    codes = np.asarray(codes, dtype=np.uint8)
    s = np.asarray(scales)
    rows, cols = codes.shape
    nbr, nbc = -(-rows // BLOCK), -(-cols // BLOCK)
    if s.shape != (nbr, nbc):
        raise ValueError(f"scales shape {s.shape}, expected {(nbr, nbc)}")
    return dequantize_rows(codes, s[np.arange(rows) // BLOCK])


def gemm(qA, sA, qB, sB, alpha: float = 1.0, beta: float = 0.0, C_in=None, nthreads: int = 0):
    """(C64, absAB) of the block-scaled GEMM: qA m x k codes with sA, qB n x k
    codes with sB; absAB = |Adq| @ |Bdq|^T for the error bound."""
    from . import gemm as gemm64
    A = dequantize(qA, sA)
    B = dequantize(qB, sB)
    return gemm64(A, B.T, alpha, beta, C_in, nthreads)


def gemm_entries(rows, cols, qA, sA, qB, sB, alpha: float = 1.0, beta: float = 0.0, C_in=None,
                 nthreads: int = 0):
    """Entries (rows[e], cols[e]) of the block-scaled GEMM and of |Adq| @ |Bdq|^T.
    For operands too large to bring to the host, pass only the referenced rows
    of qA and qB with ``dequantize_rows``' per-row scales through
    ``gemm_entries_rows``."""
    from . import gemm_entries as entries64
    A = dequantize(qA, sA)
    B = dequantize(qB, sB)
    return entries64(rows, cols, A, B.T, alpha, beta, C_in, nthreads)


def gemm_entries_rows(ri, ci, qA_rows, sA_rows, qB_rows, sB_rows, alpha: float = 1.0,
                      beta: float = 0.0, C_in=None, nthreads: int = 0):
    """Entries (ri[e], ci[e]) of the block-scaled GEMM of row subsets: qA_rows
    (r_a x k) and qB_rows (r_b x k) are rows taken from A and B, sA_rows and
    sB_rows their per-row scale rows (see ``dequantize_rows``); ri and ci index
    into the taken rows."""
    from . import gemm_entries as entries64
    A = dequantize_rows(qA_rows, sA_rows)
    B = dequantize_rows(qB_rows, sB_rows)
    return entries64(ri, ci, A, B.T, alpha, beta, C_in, nthreads)
