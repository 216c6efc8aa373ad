"""Pins of the oracle's RN-even format rounding and ulp.

FP16 and FP32 reduce to library casts (numpy's IEEE conversions); BF16 is
pinned by hand-worked ties and by torch's BF16 cast.
"""
import numpy as np
import pytest
import torch

from oracle import rounding


def _samples(seed, count=20000):
    r = np.random.Generator(np.random.PCG64(seed))
    x = r.standard_normal(count) * np.exp2(r.integers(-30, 30, size=count))
    edge = np.array([0.0, -0.0, 1.0, -1.0, 65504.0, 65520.0, 65519.99, 6.0e-8, 2.9e-8,
                     3.0e-8, 1e-40, 3.4028234663852886e38, 3.4028235677973366e38, 1e39])
    return np.concatenate([x, edge])


def test_f16_matches_ieee_cast():
    x = _samples(1)
    got = rounding.round_rne(x, "f16")
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(got, want, equal_nan=True)


def test_f32_matches_ieee_cast():
    x = _samples(2)
    got = rounding.round_rne(x, "f32")
    with np.errstate(over="ignore"):
        want = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(got, want, equal_nan=True)


def test_bf16_hand_ties():
    # bf16 has 7 fraction bits: spacing 2^-7 on [1, 2).
    cases = {
        1.0 + 2.0 ** -8: 1.0,                       # tie -> even (1.0)
        1.0 + 3 * 2.0 ** -8: 1.0 + 2.0 ** -6,       # tie between odd 1+2^-7 and even 1+2^-6
        1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,  # above the tie
        -(1.0 + 2.0 ** -8): -1.0,
        4096.0 + 8.0: 4096.0,                       # spacing 32 at 2^12: 8 < 16 rounds down
        4096.0 + 16.0: 4096.0,                      # tie -> even
        4096.0 + 48.0: 4096.0 + 64.0,               # tie -> even (odd 32 vs even 64)
        2.0 ** -130: 2.0 ** -130,                   # subnormal (spacing 2^-133), representable
        2.0 ** -134: 0.0,                           # half the smallest subnormal: tie -> even (0)
        3 * 2.0 ** -134: 2.0 ** -132,               # 1.5 * 2^-133: tie -> even (2 * 2^-133)
    }
    for x, want in cases.items():
        assert rounding.round_rne(x, "bf16") == want, x


def test_bf16_matches_torch_cast():
    x = _samples(3)
    x = x[np.abs(x) < 3.0e38]
    got = rounding.round_rne(x, "bf16")
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    # torch rounds from float32, so compare only where float32 holds x exactly
    exact32 = x.astype(np.float32).astype(np.float64) == x
    assert np.array_equal(got[exact32], want[exact32])


def test_ulp_values():
    assert rounding.ulp(1.0, "f32") == 2.0 ** -23
    assert rounding.ulp(1.5, "bf16") == 2.0 ** -7
    assert rounding.ulp(3.0, "bf16") == 2.0 ** -6
    assert rounding.ulp(1024.0, "f16") == 1.0
    assert rounding.ulp(0.0, "f16") == 2.0 ** -24
    assert rounding.ulp(-7.0, "f32") == 2.0 ** -21


@pytest.mark.parametrize("k", [1, 255, 256, 257, 4096, 4097, 65535, 65536])
def test_bf16_of_integer(k):
    # An integer k needs ceil(log2 k) bits; bf16 keeps 8 significant bits.
    got = rounding.round_rne(float(k), "bf16")
    e = int(np.floor(np.log2(k)))
    q = 2.0 ** max(0, e - 7)
    lo = np.floor(k / q) * q
    hi = lo + q
    if k - lo < hi - k:
        want = lo
    elif k - lo > hi - k:
        want = hi
    else:
        want = lo if int(lo / q) % 2 == 0 else hi
    assert got == want
