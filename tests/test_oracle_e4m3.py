"""Pins of the block-scaled E4M3 oracle (CPU only).

The decoder is pinned by the OCP E4M3 definition's landmark codes and by a
library routine (torch's float8_e4m3fn widening) over all 256 codes; the
block-scaled GEMM by brute force in its other form (a sum over k-blocks of
scale products times block dot products) and by closed forms."""
import numpy as np
import pytest
import torch

from oracle import e4m3
from paper_2301_03598_gb300 import inputs


def test_decode_landmarks():
    cases = {
        0x00: 0.0, 0x80: -0.0, 0x38: 1.0, 0xB8: -1.0, 0x40: 2.0, 0x3C: 1.5,
        0x01: 2.0 ** -9,            # smallest subnormal
        0x07: 7 * 2.0 ** -9,        # largest subnormal
        0x08: 2.0 ** -6,            # smallest normal
        0x7E: 448.0, 0xFE: -448.0,  # largest finite
        0x77: 240.0, 0x30: 0.5,
    }
    for code, v in cases.items():
        got = e4m3.decode(np.array([code], np.uint8))[0]
        assert got == v and np.signbit(got) == np.signbit(v), hex(code)
    assert np.isnan(e4m3.decode(np.array([0x7F, 0xFF], np.uint8))).all()


def test_decode_matches_library_widening_for_every_code():
    codes = np.arange(256, dtype=np.uint8)
    mine = e4m3.decode(codes)
    lib = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(np.isnan(mine), np.isnan(lib))
    ok = ~np.isnan(lib)
    assert np.array_equal(mine[ok], lib[ok])
    assert np.array_equal(np.signbit(mine[ok]), np.signbit(lib[ok]))


def test_decode_is_monotone_over_positive_codes():
    v = e4m3.decode(np.arange(0x7F, dtype=np.uint8))
    assert (np.diff(v) > 0).all()
    assert v[-1] == e4m3.MAX_FINITE


def _brute_block_sum(qA, sA, qB, sB):
    """C[i, j] = sum over k-blocks kb of sA[i//128, kb] * sB[j//128, kb] *
    sum_{l in kb} a[i, l] * b[j, l] -- loops, codes decoded one by one."""
    m, k = qA.shape
    n = qB.shape[0]
    vals = e4m3.decode(np.arange(256, dtype=np.uint8))
    C = np.zeros((m, n))
    for i in range(m):
        for j in range(n):
            tot = 0.0
            for kb in range(-(-k // 128)):
                dot = 0.0
                for l in range(kb * 128, min(k, kb * 128 + 128)):
                    dot += vals[qA[i, l]] * vals[qB[j, l]]
                tot += float(sA[i // 128, kb]) * float(sB[j // 128, kb]) * dot
            C[i, j] = tot
    return C


def test_gemm_equals_block_sum_form_on_ragged_blocks():
    # 2 x 2 row blocks, 3 k-blocks (the last of 44), all ragged
    m, n, k = 131, 129, 300
    qA, sA = inputs.host_e4m3_matrix(m, k, "normal", 11)
    qB, sB = inputs.host_e4m3_matrix(n, k, "normal", 12)
    qA, sA, qB, sB = qA.numpy(), sA.numpy(), qB.numpy(), sB.numpy()
    rows = np.array([0, 5, 127, 128, 130, 64, 129])
    cols = np.array([0, 128, 7, 127, 128, 100, 3])
    C64, _ = e4m3.gemm(qA, sA, qB, sB)
    # brute force on the sampled entries only
    vals = e4m3.decode(np.arange(256, dtype=np.uint8))
    for i, j in zip(rows, cols):
        tot = 0.0
        for kb in range(3):
            dot = sum(vals[qA[i, l]] * vals[qB[j, l]] for l in range(kb * 128, min(k, kb * 128 + 128)))
            tot += float(sA[i // 128, kb]) * float(sB[j // 128, kb]) * dot
        assert C64[i, j] == pytest.approx(tot, rel=1e-12, abs=1e-12)


def test_gemm_small_full_brute_force_with_alpha_beta():
    m, n, k = 5, 4, 272
    qA, sA = inputs.host_e4m3_matrix(m, k, "uniform", 21)
    qB, sB = inputs.host_e4m3_matrix(n, k, "uniform", 22)
    qA, sA, qB, sB = qA.numpy(), sA.numpy(), qB.numpy(), sB.numpy()
    Cin = np.arange(m * n, dtype=np.float64).reshape(m, n) / 7.0
    C64, absAB = e4m3.gemm(qA, sA, qB, sB, alpha=0.5, beta=-2.0, C_in=Cin)
    want = 0.5 * _brute_block_sum(qA, sA, qB, sB) - 2.0 * Cin
    assert np.allclose(C64, want, rtol=1e-12, atol=1e-12)
    vals = np.abs(e4m3.decode(np.arange(256, dtype=np.uint8)))
    absA = vals[qA] * np.repeat(sA.astype(np.float64), 128, 1)[:, :k]
    absB = vals[qB] * np.repeat(sB.astype(np.float64), 128, 1)[:, :k]
    assert np.allclose(absAB, absA @ absB.T, rtol=1e-12)


def test_closed_form_ones_with_power_of_two_scales():
    # every code 1.0 (0x38); scale of block (I, kb) = 2^(I + kb) for A and
    # 2^-(J + 2 kb) for B, so C[i, j] = sum_kb 2^(I - J - kb) * len(kb)
    m, n, k = 260, 130, 400
    qA = np.full((m, k), 0x38, np.uint8)
    qB = np.full((n, k), 0x38, np.uint8)
    nkb = -(-k // 128)
    sA = np.array([[2.0 ** (I + kb) for kb in range(nkb)] for I in range(-(-m // 128))], np.float32)
    sB = np.array([[2.0 ** -(J + 2 * kb) for kb in range(nkb)] for J in range(-(-n // 128))],
                  np.float32)
    C64, _ = e4m3.gemm(qA, sA, qB, sB)
    lens = [min(k, kb * 128 + 128) - kb * 128 for kb in range(nkb)]
    for i in (0, 127, 128, 259):
        for j in (0, 128, 129):
            I, J = i // 128, j // 128
            assert C64[i, j] == sum(2.0 ** (I - J - kb) * L for kb, L in enumerate(lens))


def test_quantizer_scales_and_range():
    x = torch.randn(300, 260)
    q, s = inputs.e4m3_quantize(x)
    deq = e4m3.dequantize(q.numpy(), s.numpy())
    # every block's largest magnitude maps to 448 exactly (amax / scale)
    assert s.shape == (3, 3)
    assert np.abs(deq).max() == pytest.approx(float(np.abs(x.numpy()).max()), rel=1e-6)
    # E4M3 keeps 3 mantissa bits: relative error at most 2^-4 above the subnormals
    big = np.abs(x.numpy()) > float(s.max()) * 2.0 ** -6
    rel = np.abs(deq - x.numpy().astype(np.float64))[big] / np.abs(x.numpy())[big]
    assert rel.max() <= 2.0 ** -4 + 1e-12
    q0, s0 = inputs.e4m3_quantize(torch.zeros(130, 10))
    assert (s0.numpy() == 1.0).all() and (q0.numpy() == 0).all()


def test_row_subset_entries_equal_full_gemm_entries():
    # rows taken across 128-row blocks (with their blocks' scale rows) give the
    # same entries as the whole operands, and each taken value is
    # scale * decode(code) element by element
    m, n, k = 300, 260, 400
    qA, sA = inputs.host_e4m3_matrix(m, k, "normal", 31)
    qB, sB = inputs.host_e4m3_matrix(n, k, "normal", 32)
    qA, sA, qB, sB = qA.numpy(), sA.numpy(), qB.numpy(), sB.numpy()
    ra = np.array([0, 127, 128, 255, 256, 299])
    rb = np.array([3, 128, 259])
    vals = e4m3.decode(np.arange(256, dtype=np.uint8))
    sub = e4m3.dequantize_rows(qA[ra], sA[ra // 128])
    for i, r in enumerate(ra):
        for l in (0, 127, 128, 399):
            assert sub[i, l] == float(sA[r // 128, l // 128]) * vals[qA[r, l]]
    ri = np.array([0, 1, 2, 3, 4, 5, 5])
    ci = np.array([0, 1, 2, 0, 1, 2, 0])
    got, gabs = e4m3.gemm_entries_rows(ri, ci, qA[ra], sA[ra // 128], qB[rb], sB[rb // 128],
                                       alpha=0.5)
    want, wabs = e4m3.gemm_entries(ra[ri], rb[ci], qA, sA, qB, sB, alpha=0.5)
    assert np.array_equal(got, want) and np.array_equal(gabs, wabs)
