"""Rounding of FP32 panels to shorter floating-point formats, for the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The sparse x dense products of Section 3.3 gather one panel row per stored
entry, so the bytes of a panel value set the cost of a pass.  Section 3.2
lets the library choose the precision of its numbers; the sparse passes offer
the panel rounded to

* BF16:   8 significant bits (sign, 8-bit exponent, 7 stored mantissa bits);
* 24-bit: 16 significant bits (sign, 8-bit exponent, 15 stored mantissa bits).

Both keep FP32's exponent range, so rounding is to a grid of spacing
``ulp32(x) * 2**(24 - p)`` for p significant bits, where ulp32(x) is the
spacing of FP32 at x (``2**(e - 23)`` for a normal x in [2**e, 2**(e+1)),
``2**-149`` for subnormals), with ties to even -- the plain definition of
round-to-nearest-even into a format with p significant bits and FP32's
exponents, written out with exact FP64 arithmetic (every FP32 value and every
grid point is an FP64 value; dividing by a power of two is exact).
"""

from __future__ import annotations

import numpy as np


def round_significant(x, p: int) -> np.ndarray:
    """Round FP32 values to p significant bits (1 <= p <= 24), ties to even,
    keeping FP32's exponent range.  Returns FP32.  Finite inputs only; a value
    that rounds past the largest finite FP32 becomes inf."""
    if not 1 <= p <= 24:
        raise ValueError("p must be in [1, 24]")
    x = np.asarray(x, dtype=np.float32)
    if not np.all(np.isfinite(x)):
        raise ValueError("finite inputs only")
    xd = x.astype(np.float64)
    mag = np.abs(xd)
    # exponent e with 2**e <= |x| < 2**(e+1); FP32 subnormals use e = -126
    e = np.where(mag > 0, np.floor(np.log2(np.where(mag > 0, mag, 1.0))), -126.0)
    # log2 may land one off at exact powers of two: correct against the bounds
    e = np.where(np.exp2(e) > mag, e - 1, e)
    e = np.where(np.exp2(e + 1) <= mag, e + 1, e)
    e = np.maximum(e, -126.0)
    quantum = np.exp2(e - 23.0 + (24 - p))
    q = np.round(xd / quantum) * quantum  # numpy rounds halves to even
    with np.errstate(over="ignore"):
        return q.astype(np.float32)


def round_bf16(x) -> np.ndarray:
    """FP32 values rounded to BF16 (8 significant bits), returned as FP32."""
    return round_significant(x, 8)


def round_p24(x) -> np.ndarray:
    """FP32 values rounded to the 24-bit format (16 significant bits), as FP32."""
    return round_significant(x, 16)
