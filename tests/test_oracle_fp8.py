"""Pins for the oracle's E4M3 rounding and per-tile scales (OCP FP8 definition)."""

import numpy as np
import pytest

from oracle import fp8 as F


def test_decode_table_matches_the_format():
    v = F.DECODE_TABLE
    assert np.isnan(v[0x7F]) and np.isnan(v[0xFF])
    finite = v[~np.isnan(v)]
    assert finite.max() == 448.0 and finite.min() == -448.0
    assert v[0x01] == 2.0 ** -9 and v[0x07] == 7 * 2.0 ** -9      # subnormals
    assert v[0x08] == 2.0 ** -6                                    # smallest normal
    assert v[0x38] == 1.0 and v[0x39] == 1.125 and v[0x7E] == 448.0
    assert v[0x80] == 0.0 and np.signbit(v[0x80])                 # negative zero
    pos = np.sort(v[:0x7F])
    assert np.all(np.diff(pos) > 0)                               # 127 distinct non-negative values


def test_every_code_round_trips():
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF, 0x80)], dtype=np.uint8)
    assert np.array_equal(F.encode_e4m3(F.DECODE_TABLE[codes]), codes)


def test_round_to_nearest_even_at_every_midpoint():
    pos = np.sort(F.DECODE_TABLE[:0x7F])          # 0 .. 448
    mids = (pos[:-1] + pos[1:]) / 2
    got = F.DECODE_TABLE[F.encode_e4m3(mids)]
    lo_codes = F.encode_e4m3(pos[:-1])
    even_lo = (lo_codes & 1) == 0
    assert np.array_equal(got, np.where(even_lo, pos[:-1], pos[1:]))
    # just off the midpoints rounding goes to the nearer neighbour
    assert np.array_equal(F.DECODE_TABLE[F.encode_e4m3(np.nextafter(mids, 0))], pos[:-1])
    assert np.array_equal(F.DECODE_TABLE[F.encode_e4m3(np.nextafter(mids, 1e9))], pos[1:])


def test_saturation_and_signs():
    x = np.array([448.0, 460.0, 480.0, 1e6, -1e6, -3.3, 0.0, -0.0, 2.0 ** -11, 2.0 ** -10 + 2.0 ** -20])
    got = F.DECODE_TABLE[F.encode_e4m3(x)]
    assert got[0] == 448 and got[1] == 448 and got[2] == 448 and got[3] == 448 and got[4] == -448
    assert got[5] == -3.25                      # nearest of -3.25 / -3.5
    assert got[6] == 0 and got[7] == 0 and np.signbit(got[7])
    assert got[8] == 0.0                        # below half the smallest subnormal
    assert got[9] == 2.0 ** -9                  # just above half of it
    assert F.encode_e4m3(np.array([np.nan]))[0] == 0x7F


@pytest.mark.parametrize("amax,scale", [(448.0, 1.0), (448.0001, 2.0), (449.0, 2.0), (1.0, 2.0 ** -8),
                                        (0.875, 2.0 ** -9), (0.8751, 2.0 ** -8), (0.0, 1.0), (3e5, 1024.0)])
def test_tile_scale_is_the_smallest_power_of_two(amax, scale):
    s = F.tile_scale(amax)
    assert s == scale
    if amax > 0:
        assert amax / s <= 448 and amax / (s / 2) > 448


def test_quantize_tiles_bounds_and_round_trip():
    rng = np.random.default_rng(3)
    A = (rng.standard_normal((300, 260)) * np.logspace(-3, 2, 260)).astype(np.float32)
    codes, scales = F.quantize_tiles(A, 128, 128)
    assert scales.shape == (3, 3)
    D = F.dequantize_tiles(codes, scales, 128, 128)
    # each entry within half a unit of E4M3 precision (2^-4 relative) or below the subnormal step
    rel = np.abs(D - A) / np.maximum(np.abs(A), 1e-300)
    ok = (rel <= 2.0 ** -4 + 1e-12) | (np.abs(D - A) <= np.repeat(np.repeat(scales, 128, 0)[:300], 128, 1)[:, :260] * 2.0 ** -10)
    assert np.all(ok)
    # the largest entry of every tile uses the top of the range
    for I in range(3):
        for J in range(3):
            blk = D[I * 128:(I + 1) * 128, J * 128:(J + 1) * 128]
            assert 224 <= np.max(np.abs(blk)) / scales[I, J] <= 448
