"""Oracle number formats: round-to-nearest-even onto a binary format's grid,
and the format's unit in the last place.  TEST INFRASTRUCTURE ONLY.

Written from the IEEE 754 definition of a binary format with precision p
(significand bits including the hidden bit) and exponent range [emin, emax]:
the representable magnitudes are 0, the subnormals j * 2^(emin-p+1) and the
normals (1 + f) * 2^e.  A real x rounds to the nearest representable value,
ties to the one with an even last significand bit, and to infinity once it
reaches 2^emax * (2 - 2^-p) (the halfway point above the largest finite
value).

The GPU path never calls this; the tests use it for closed-form expected
outputs (for instance k in BF16) and for the one-output-ulp term of the error
bound on the GPU results.
"""
from __future__ import annotations

import numpy as np

# name: (precision p, emin, emax)
FORMATS = {
    "f32": (24, -126, 127),
    "f16": (11, -14, 15),
    "bf16": (8, -126, 127),
}


def _params(fmt: str):
    try:
        return FORMATS[fmt]
    except KeyError:
        raise ValueError(f"unknown format {fmt!r}") from None


def max_finite(fmt: str) -> float:
    p, _, emax = _params(fmt)
    return (2.0 - 2.0 ** (1 - p)) * 2.0 ** emax


def quantum(x, fmt: str) -> np.ndarray:
    """Spacing of the format's grid at |x|: 2^(max(e, emin) - p + 1) with
    e = floor(log2 |x|); the subnormal spacing for |x| below 2^emin and 0."""
    p, emin, _ = _params(fmt)
    ax = np.abs(np.asarray(x, dtype=np.float64))
    _, E = np.frexp(ax)               # ax = f * 2^E, f in [0.5, 1) (E = 0 for 0)
    e = np.where(ax > 0, E - 1, emin)
    e = np.maximum(e, emin)
    return np.ldexp(1.0, (e - (p - 1)).astype(np.int64))


def ulp(x, fmt: str) -> np.ndarray:
    """Unit in the last place of the format at |x| (same as ``quantum``)."""
    return quantum(x, fmt)


def round_rne(x, fmt: str) -> np.ndarray:
    """Round each double in x to the nearest value of ``fmt``, ties to even,
    overflow to +-inf.  Returned as float64 holding the rounded value."""
    x = np.asarray(x, dtype=np.float64)
    q = quantum(x, fmt)
    ax = np.abs(x)
    # ax / q is an exact power-of-two scaling; rint rounds half to even.
    r = np.rint(ax / q) * q
    r = np.where(r > max_finite(fmt), np.inf, r)
    r = np.where(np.isnan(x), np.nan, r)
    return np.copysign(r, x)
