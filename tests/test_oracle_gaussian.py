"""Pins for the oracle's Gaussian test matrix (Section 2.1 step 1)."""

import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from oracle import gaussian as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for row in rows:
        ctr, key, want = row[:4], row[4:6], row[6:]
        out = G.philox4x32(*[np.array([c], dtype=np.uint64) for c in ctr], key[0], key[1])
        assert [int(o[0]) for o in out] == want


def test_philox_vectorised_matches_scalar_calls():
    ctr = np.arange(17, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15 & 0xFFFFFFFF)
    ctr &= np.uint64(0xFFFFFFFF)
    batch = G.philox4x32(ctr, ctr ^ np.uint64(5), ctr, ctr, 123, 456)
    for i in range(17):
        one = G.philox4x32(ctr[i:i + 1], ctr[i:i + 1] ^ np.uint64(5), ctr[i:i + 1], ctr[i:i + 1], 123, 456)
        assert [int(o[0]) for o in one] == [int(b[i]) for b in batch]


def test_ln2_split_against_decimal():
    getcontext().prec = 50
    ln2 = Fraction(Decimal(2).ln())
    hi, lo = Fraction(G.LN2_HI), Fraction(G.LN2_LO)
    # head has at most 32 significant bits, so E*LN2_HI is exact for |E| < 2^21
    assert (hi * 2 ** 32).denominator == 1
    assert abs(hi + lo - ln2) < Fraction(1, 2 ** 85)


def _mp():
    return pytest.importorskip("mpmath")


def _ulp_err(got, ref):
    return abs(got - ref) / math.ulp(ref)


def test_ln_within_2ulp_of_high_precision():
    mp = _mp()
    mp.mp.prec = 120
    rng = np.random.default_rng(7)
    u = np.concatenate([rng.random(1500), 2.0 ** -np.arange(1, 54),
                        1.0 - 2.0 ** -np.arange(1, 53), [0.5 + 2 ** -52, G.SQRT2 / 2]])
    got = G.ln(u)
    worst = max(_ulp_err(float(g), float(mp.log(mp.mpf(float(x))))) for g, x in zip(got, u))
    assert worst <= 2.0
    assert G.ln(np.array([1.0]))[0] == 0.0


def test_sincos_within_2ulp_of_high_precision():
    mp = _mp()
    mp.mp.prec = 120
    rng = np.random.default_rng(8)
    n2 = np.concatenate([rng.integers(0, 2 ** 53, 1500, dtype=np.uint64),
                         np.array([0, 2 ** 53 - 1, 2 ** 51, 2 ** 51 - 1, 2 ** 52, 2 ** 52 - 1,
                                   3 * 2 ** 51, 3 * 2 ** 51 - 1, 2 ** 50, 2 ** 50 - 1],
                                  dtype=np.uint64)])
    s, c = G.sincos_2pi(n2)
    ws = wc = 0.0
    for i, v in enumerate(n2):
        th = 2 * mp.pi * mp.mpf(2 * int(v) + 1) / mp.mpf(2) ** 54
        ws = max(ws, _ulp_err(float(s[i]), float(mp.sin(th))))
        wc = max(wc, _ulp_err(float(c[i]), float(mp.cos(th))))
    assert ws <= 2.0 and wc <= 2.0


def test_box_muller_assembly_against_high_precision():
    """Rebuild a few stream elements from the Philox words with 120-bit math."""
    mp = _mp()
    mp.mp.prec = 120
    seed = 0x1234_5678_9ABC_DEF0
    vals = G.gaussian_stream(0, 64, seed)
    for e in range(64):
        g = e >> 1
        x = G.philox4x32(np.array([g & 0xFFFFFFFF], dtype=np.uint64), np.array([g >> 32], dtype=np.uint64),
                         np.zeros(1, np.uint64), np.zeros(1, np.uint64), seed & 0xFFFFFFFF, seed >> 32)
        x0, x1, x2, x3 = (int(w[0]) for w in x)
        n1 = ((x0 << 32) | x1) >> 11
        n2 = ((x2 << 32) | x3) >> 11
        u1 = mp.mpf(n1 + 1) / mp.mpf(2) ** 53
        th = 2 * mp.pi * mp.mpf(2 * n2 + 1) / mp.mpf(2) ** 54
        rho = mp.sqrt(-2 * mp.log(u1))
        ref = float(rho * (mp.sin(th) if e % 2 else mp.cos(th)))
        assert abs(vals[e] - ref) <= 4 * math.ulp(ref) + 1e-300


def test_gaussian_distribution():
    scipy_stats = pytest.importorskip("scipy.stats")
    v = G.gaussian_stream(0, 1_000_000, 2002)
    assert abs(v.mean()) < 5 / 1000
    assert abs(v.var() - 1) < 5 * math.sqrt(2 / 1e6)
    kurt = ((v - v.mean()) ** 4).mean() / v.var() ** 2
    assert abs(kurt - 3) < 5 * math.sqrt(24 / 1e6)
    assert scipy_stats.kstest(v, "norm").pvalue > 1e-4
    # the two halves of a Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(v[0::2], v[1::2])[0, 1]) < 5 / 1000


def test_stream_is_tiling_invariant():
    full = G.gaussian_stream(0, 1000, 99)
    parts = np.concatenate([G.gaussian_stream(0, 333, 99), G.gaussian_stream(333, 667, 99)])
    assert np.array_equal(full, parts)
    M = G.gaussian_matrix(40, 25, 99)
    assert np.array_equal(M.reshape(-1), full)


def _bf16_nearest_exact(x: float) -> float:
    """Nearest bfloat16 to x by exhaustive search over neighbours (ties to even)."""
    if x == 0:
        return 0.0
    f = Fraction(x)
    e = math.floor(math.log2(abs(x)))
    best = None
    for ee in (e - 1, e, e + 1):
        step = Fraction(2) ** (ee - 7)
        base = (abs(f) / step).__floor__()
        for mnt in (base - 1, base, base + 1, base + 2):
            if not (128 <= mnt < 256):
                continue
            cand = mnt * step
            d = abs(cand - abs(f))
            key = (d, mnt % 2)
            if best is None or key < best[0]:
                best = (key, cand)
    return float(best[1]) * (1 if x > 0 else -1)


def test_bf16_rounding_is_nearest_even():
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.standard_normal(3000) * 3, [1.0, -1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8,
                                                         1 + 2 ** -8 + 2 ** -40, 255.5, 0.0]])
    got = G.bf16_bits_to_f64(G.to_bf16_bits(xs))
    for x, g in zip(xs, got):
        assert g == _bf16_nearest_exact(float(x)), x


def test_matrix_dtypes_round_once():
    v = G.gaussian_matrix(30, 7, 5, "f64")
    assert np.array_equal(G.gaussian_matrix(30, 7, 5, "f32"), v.astype(np.float32))
    assert np.array_equal(G.gaussian_matrix_as_f64(30, 7, 5, "bf16"),
                          G.bf16_bits_to_f64(G.to_bf16_bits(v)).reshape(30, 7))


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_rows_of_o_without_forming_it(dtype):
    """gaussian_rows gives the rows of the full matrix, in any order and with
    repeats, for even and odd r (odd r splits Box-Muller pairs across rows)."""
    for n, r in ((50, 8), (37, 7)):
        full = G.gaussian_matrix_as_f64(n, r, 31, dtype)
        rows = np.array([36, 0, 5, 5, 17, 1])
        assert np.array_equal(G.gaussian_rows(rows, r, 31, dtype), full[rows])
