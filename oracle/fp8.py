"""FP8 (E4M3) storage of A with per-tile power-of-two scales, for the FP8
variant of the A-passes (products with A of Section 2.1 steps 2 and 5 and of
Eq. (3); the precision choices of Section 3.2 taken one step below half
precision).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

E4M3 as defined by the OCP 8-bit floating point specification (2023): one sign
bit, four exponent bits with bias 7, three mantissa bits; exponent field 0
holds the subnormals m * 2^-9; the largest finite magnitude is
1.75 * 2^8 = 448 (exponent 15, mantissa 110); exponent 15 with mantissa 111 is
NaN; there are no infinities.  Values are rounded to nearest, ties to even
mantissa, and magnitudes beyond 448 saturate to 448 ("satfinite").

Per-tile scale: for a tile with largest magnitude amax > 0 the scale is the
smallest power of two s with amax / s <= 448 (s = 1 for an all-zero tile), and
the tile stores code(x / s); the dequantised value is decode(code) * s.
Tiles are the block-cyclic tiles of Section 3.1: rows [I*qm, ...) x columns
[J*qn, ...).
"""

from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def decode_e4m3(code: int) -> float:
    """Value of one E4M3 byte (NaN for 0x7F / 0xFF)."""
    code = int(code) & 0xFF
    sign = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 15 and m == 7:
        return float("nan")
    if e == 0:
        return sign * m * 2.0 ** -9
    return sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)


DECODE_TABLE = np.array([decode_e4m3(c) for c in range(256)], dtype=np.float64)


def encode_e4m3(x) -> np.ndarray:
    """Round FP64 values to E4M3 codes (nearest, ties to even, saturating)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape, dtype=np.uint8)
    sign = np.signbit(x)
    a = np.abs(x)
    nan = np.isnan(x)
    a = np.where(nan, 0.0, a)
    # spacing of the E4M3 grid around a: 2^(max(floor(log2 a), -6) - 3), with
    # floor(log2 a) = E - 1 for a = f 2^E, f in [0.5, 1) (exact, from frexp)
    _, E = np.frexp(np.where(a > 0, a, 1.0))
    e = np.maximum(E.astype(np.int64) - 1, -6)
    ulp = np.ldexp(1.0, e - 3)
    q = a / ulp                                   # exact: division by a power of two
    fl = np.floor(q)
    frac = q - fl
    up = (frac > 0.5) | ((frac == 0.5) & (np.mod(fl, 2) == 1))
    v = (fl + up) * ulp                          # rounded magnitude (may step to the next binade)
    v = np.minimum(v, E4M3_MAX)                   # satfinite
    # encode v (a point of the E4M3 grid) exactly
    _, Ev = np.frexp(np.where(v > 0, v, 1.0))
    ev = np.maximum(Ev.astype(np.int64) - 1, -6)
    sub = v < 2.0 ** -6
    mant_sub = np.round(v / 2.0 ** -9).astype(np.int64)                  # exact for subnormals
    mant_norm = np.round((v / np.ldexp(1.0, ev) - 1.0) * 8).astype(np.int64)  # exact on the grid
    field = np.where(sub, mant_sub, ((ev + 7) << 3) | mant_norm)
    field = np.where(v == 0, 0, field)
    out = (field.astype(np.int64) | (sign.astype(np.int64) << 7)).astype(np.uint8)
    out = np.where(nan, np.uint8(0x7F), out)
    return out.astype(np.uint8)


def tile_scale(amax: float) -> float:
    """Smallest power of two s with amax / s <= 448 (1 for amax = 0)."""
    if not amax > 0:
        return 1.0
    m, e = np.frexp(amax)          # amax = m 2^e, m in [0.5, 1)
    s = np.ldexp(1.0, int(e) - 9)  # 448 = 0.875 * 2^9: candidate with amax / s = m * 2^9
    if amax / s > E4M3_MAX:        # m > 0.875
        s *= 2.0
    return float(s)


def quantize_tiles(A, qm: int, qn: int):
    """E4M3 codes (uint8, A's shape) and per-tile scales (Tm x Tn) of a dense A."""
    A = np.asarray(A)
    m, n = A.shape
    Tm, Tn = -(-m // qm), -(-n // qn)
    codes = np.zeros((m, n), dtype=np.uint8)
    scales = np.ones((Tm, Tn), dtype=np.float64)
    for I in range(Tm):
        for J in range(Tn):
            blk = A[I * qm:(I + 1) * qm, J * qn:(J + 1) * qn].astype(np.float64)
            s = tile_scale(float(np.max(np.abs(blk))) if blk.size else 0.0)
            scales[I, J] = s
            codes[I * qm:(I + 1) * qm, J * qn:(J + 1) * qn] = encode_e4m3(blk / s)
    return codes, scales


def dequantize_tiles(codes, scales, qm: int, qn: int) -> np.ndarray:
    """FP64 values decode(code) * scale of the tile."""
    codes = np.asarray(codes, dtype=np.uint8)
    m, n = codes.shape
    out = DECODE_TABLE[codes]
    rs = np.repeat(np.asarray(scales, dtype=np.float64), qm, axis=0)[:m]
    return out * np.repeat(rs, qn, axis=1)[:, :n]
