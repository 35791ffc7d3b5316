"""Gaussian test matrix of Section 2.1 step 1 (the matrix O, n x r, i.i.d. N(0,1)).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper only says that every entry of O is drawn independently from N(0,1).
This oracle fixes a reproducible, parallel-friendly reading of that draw:

* Uniform bits come from the counter-based generator Philox4x32-10 (Salmon,
  Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
  ten rounds of the Philox S-box with the published multipliers and Weyl key
  increments.  The key is (seed mod 2^32, seed >> 32).
* Entry (i, j) of O is element e = i*r + j of one global stream, so the
  matrix does not depend on tiling or on how many threads produce it.
  Elements 2g and 2g+1 share one Philox call with counter (g mod 2^32, g >> 32,
  0, 0) and form one Box-Muller pair.
* From the four output words x0..x3: N1 = ((x0 << 32) | x1) >> 11 and
  N2 = ((x2 << 32) | x3) >> 11 are 53-bit integers; u1 = (N1 + 1) * 2^-53 lies
  in (0, 1] and is exact in FP64; the angle is theta = 2*pi*(2*N2 + 1)*2^-54.
* Box-Muller: rho = sqrt(-2 ln u1); even e takes rho*cos(theta), odd e takes
  rho*sin(theta).
* ln, sin and cos are written out below from their Taylor / atanh series with
  a fixed sequence of separately rounded FP64 multiplies and adds (no fused
  multiply-add), so that an independent implementation that performs the same
  IEEE operations in the same order produces the same bits.  The angle is
  reduced to [-pi/4, pi/4] exactly in integer arithmetic before the series.
* The FP64 value is rounded once (round-to-nearest-even) to the working type.
"""

from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

# Philox4x32 round multipliers and Weyl key increments (Salmon et al. 2011).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
PHILOX_ROUNDS = 10

_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32(c0, c1, c2, c3, key0: int, key1: int, rounds: int = PHILOX_ROUNDS):
    """Philox4x32-R on arrays of 32-bit counters (held in uint64 arrays).

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
    the key is advanced by the Weyl increments before every round but the first.
    """
    c0 = np.asarray(c0, dtype=np.uint64)
    c1 = np.asarray(c1, dtype=np.uint64)
    c2 = np.asarray(c2, dtype=np.uint64)
    c3 = np.asarray(c3, dtype=np.uint64)
    k0 = key0 & 0xFFFFFFFF
    k1 = key1 & 0xFFFFFFFF
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for rnd in range(rounds):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
        p0 = c0 * m0  # < 2^64: exact in uint64
        p1 = c2 * m1
        hi0 = p0 >> np.uint64(32)
        lo0 = p0 & _MASK32
        hi1 = p1 >> np.uint64(32)
        lo1 = p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return c0, c1, c2, c3


# ---------------------------------------------------------------------------
# FP64 elementary functions (own series; every operation separately rounded).
# ---------------------------------------------------------------------------

def _recip(q: int) -> float:
    """Correctly rounded FP64 value of 1/q."""
    return float(Fraction(1, q))


# ln 2 split as a 32-significant-bit head (so E*LN2_HI is exact for |E| < 2^21)
# plus the FP64-rounded remainder.
LN2_HI = float.fromhex("0x1.62e42fee00000p-1")
LN2_LO = float.fromhex("0x1.a39ef35793c76p-33")
SQRT2 = float.fromhex("0x1.6a09e667f3bcdp+0")  # fl(sqrt 2), a branch threshold
PI = float.fromhex("0x1.921fb54442d18p+1")     # fl(pi)
PI_2M53 = PI * 2.0 ** -53                       # exact scaling of fl(pi)

# atanh series: ln f = 2 atanh(s) = 2s + 2s * z * sum_k z^k / (2k+3), z = s^2.
ATANH_C = [_recip(2 * k + 3) for k in range(10)]          # 1/3 .. 1/21
# sin x = x + x * z * sum_k (-1)^(k+1) z^k / (2k+3)!, k = 0..8  (3! .. 19!)
SIN_C = [(-1.0 if k % 2 == 0 else 1.0) * _recip(math.factorial(2 * k + 3)) for k in range(9)]
# cos x = 1 + z * sum_k (-1)^(k+1) z^k / (2k+2)!, k = 0..8     (2! .. 18!)
COS_C = [(-1.0 if k % 2 == 0 else 1.0) * _recip(math.factorial(2 * k + 2)) for k in range(9)]


def _horner(coeffs, z):
    """c0 + z*(c1 + z*(c2 + ...)), each multiply and add rounded separately."""
    acc = np.full_like(z, coeffs[-1])
    for c in reversed(coeffs[:-1]):
        acc = c + z * acc
    return acc


def ln(u):
    """Natural log of positive normal FP64 values.

    u = f * 2^E with f in [sqrt(2)/2, sqrt(2)]; s = (f-1)/(f+1);
    ln u = E*LN2_HI + (E*LN2_LO + (h + h*(z*P(z)))) with h = 2s, z = s^2.
    """
    u = np.asarray(u, dtype=np.float64)
    mant, ex = np.frexp(u)            # exact: u = mant * 2^ex, mant in [0.5, 1)
    f = mant * 2.0                    # exact
    E = (ex - 1).astype(np.int64)
    big = f > SQRT2
    f = np.where(big, f * 0.5, f)     # exact
    E = np.where(big, E + 1, E)
    s = (f - 1.0) / (f + 1.0)
    z = s * s
    P = _horner(ATANH_C, z)
    h = 2.0 * s                       # exact
    t1 = z * P
    t2 = h * t1
    lnf = h + t2
    Ef = E.astype(np.float64)
    t3 = Ef * LN2_LO
    t4 = t3 + lnf
    t5 = Ef * LN2_HI                  # exact
    return t5 + t4


def sin_reduced(phi):
    """sin(phi) for |phi| <= pi/4: phi + phi*(z*S(z))."""
    z = phi * phi
    S = _horner(SIN_C, z)
    t1 = z * S
    t2 = phi * t1
    return phi + t2


def cos_reduced(phi):
    """cos(phi) for |phi| <= pi/4: 1 + z*C(z)."""
    z = phi * phi
    C = _horner(COS_C, z)
    t = z * C
    return 1.0 + t


def sincos_2pi(n2):
    """(sin theta, cos theta) for theta = 2*pi*(2*n2 + 1)*2^-54, n2 a 53-bit integer.

    Exact reduction: t = 2*n2 + 1, quadrant q = round(t / 2^52), remainder
    d = t - q*2^52 (|d| < 2^51, exact in FP64), phi = d * fl(pi) * 2^-53.
    """
    t = np.asarray(n2, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    q = (t + np.uint64(1 << 51)) >> np.uint64(52)
    d = t.astype(np.int64) - (q << np.uint64(52)).astype(np.int64)
    phi = d.astype(np.float64) * PI_2M53
    s = sin_reduced(phi)
    c = cos_reduced(phi)
    qm = (q & np.uint64(3)).astype(np.int64)
    sin_t = np.select([qm == 0, qm == 1, qm == 2], [s, c, -s], -c)
    cos_t = np.select([qm == 0, qm == 1, qm == 2], [c, -s, -c], s)
    return sin_t, cos_t


def gaussian_stream(e0: int, count: int, seed: int) -> np.ndarray:
    """FP64 values of stream elements e0 .. e0+count-1 (see module docstring)."""
    if count <= 0:
        return np.zeros(0, dtype=np.float64)
    return gaussian_elements(np.arange(e0, e0 + count, dtype=np.uint64), seed)


def gaussian_elements(e, seed: int) -> np.ndarray:
    """FP64 values of the stream elements with the given indices (any order,
    repeats allowed); element e is the one ``gaussian_stream`` gives at e."""
    e = np.asarray(e, dtype=np.uint64)
    g = e >> np.uint64(1)
    x0, x1, x2, x3 = philox4x32(g & _MASK32, g >> np.uint64(32),
                                np.zeros_like(g), np.zeros_like(g),
                                seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    n1 = ((x0 << np.uint64(32)) | x1) >> np.uint64(11)
    n2 = ((x2 << np.uint64(32)) | x3) >> np.uint64(11)
    u1 = (n1 + np.uint64(1)).astype(np.float64) * 2.0 ** -53   # exact, in (0, 1]
    L = ln(u1)
    rho = np.sqrt(-2.0 * L)
    sin_t, cos_t = sincos_2pi(n2)
    odd = (e & np.uint64(1)).astype(bool)
    return np.where(odd, rho * sin_t, rho * cos_t)


def to_bf16_bits(x) -> np.ndarray:
    """Round FP64 values once to bfloat16 (round-to-nearest-even); returns uint16 bits.

    Valid for zero and for normal values inside the bfloat16 range, which is
    all a Gaussian entry can take.
    """
    x = np.asarray(x, dtype=np.float64)
    b = x.view(np.uint64)
    sign = (b >> np.uint64(63)).astype(np.uint16)
    mag = b & np.uint64((1 << 63) - 1)            # exponent | mantissa
    lsb = (mag >> np.uint64(45)) & np.uint64(1)
    rounded = (mag + np.uint64((1 << 44) - 1) + lsb) >> np.uint64(45)  # 11 exp + 7 mant bits
    exp64 = (rounded >> np.uint64(7)).astype(np.int64)
    mant7 = (rounded & np.uint64(0x7F)).astype(np.uint16)
    exp16 = exp64 - 1023 + 127
    zero = mag == 0
    if np.any(~zero & ((exp16 <= 0) | (exp16 >= 255))):
        raise ValueError("value outside the normal bfloat16 range")
    bits = (sign << np.uint16(15)) | (np.where(zero, 0, exp16).astype(np.uint16) << np.uint16(7)) | np.where(zero, 0, mant7).astype(np.uint16)
    return bits.astype(np.uint16)


def bf16_bits_to_f64(bits) -> np.ndarray:
    bits = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)
    return bits.view(np.float32).astype(np.float64)


def gaussian_matrix(n: int, r: int, seed: int, dtype: str = "f64") -> np.ndarray:
    """The n x r Gaussian matrix O of Section 2.1 step 1, row-major.

    dtype "f64" returns the FP64 values, "f32" their RNE rounding to FP32,
    "bf16" their RNE rounding to bfloat16 returned as uint16 bit patterns.
    """
    vals = gaussian_stream(0, n * r, seed).reshape(n, r)
    if dtype == "f64":
        return vals
    if dtype == "f32":
        return vals.astype(np.float32)
    if dtype == "bf16":
        return to_bf16_bits(vals)
    raise ValueError(dtype)


def gaussian_rows(rows, r: int, seed: int, dtype: str = "f64") -> np.ndarray:
    """Rows ``rows`` of the n x r matrix O (entry (i, j) is element i*r + j),
    rounded to ``dtype`` and widened back to FP64, without forming O: for
    checks that touch a few rows of a test matrix with many rows."""
    rows = np.asarray(rows, dtype=np.uint64)
    e = (rows[:, None] * np.uint64(r) + np.arange(r, dtype=np.uint64)[None, :]).ravel()
    vals = gaussian_elements(e, seed).reshape(len(rows), r)
    if dtype == "f64":
        return vals
    if dtype == "f32":
        return vals.astype(np.float32).astype(np.float64)
    if dtype == "bf16":
        return bf16_bits_to_f64(to_bf16_bits(vals))
    raise ValueError(dtype)


def gaussian_matrix_as_f64(n: int, r: int, seed: int, dtype: str = "f64") -> np.ndarray:
    """O rounded to ``dtype`` and widened back to FP64 (the values a path of that type uses)."""
    o = gaussian_matrix(n, r, seed, dtype)
    if dtype == "bf16":
        return bf16_bits_to_f64(o)
    return o.astype(np.float64)
