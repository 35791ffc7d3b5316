"""Pins of oracle.panel (rounding of FP32 panels to BF16 and to 24-bit floats)
against values fixed by the formats' definitions."""

import numpy as np
import pytest

from oracle import panel as OP


def f32(bits):
    return np.array(bits, dtype=np.uint32).view(np.float32)


def test_exact_values_stay():
    # values with at most p significant bits are fixed points
    x = np.array([0.0, -0.0, 1.0, -2.5, 0.75, 3.0 * 2.0 ** -100, 2.0 ** 127], dtype=np.float32)
    assert np.array_equal(OP.round_bf16(x), x)
    assert np.array_equal(OP.round_p24(x), x)
    y = np.float32(1.0 + 2.0 ** -15)  # 16 significant bits
    assert OP.round_p24(y) == y and OP.round_bf16(y) == np.float32(1.0)


def test_ties_go_to_even():
    # 24-bit format: the spacing at 1 is 2^-15; 1 + 2^-16 is halfway -> 1 (even)
    assert OP.round_p24(np.float32(1.0 + 2.0 ** -16)) == np.float32(1.0)
    # 1 + 3 * 2^-16 is halfway between 1 + 2^-15 (odd) and 1 + 2^-14 (even)
    assert OP.round_p24(np.float32(1.0 + 3 * 2.0 ** -16)) == np.float32(1.0 + 2.0 ** -14)
    # BF16: spacing 2^-7 at 1; 1 + 2^-8 -> 1, 1 + 3 * 2^-8 -> 1 + 2^-6
    assert OP.round_bf16(np.float32(1.0 + 2.0 ** -8)) == np.float32(1.0)
    assert OP.round_bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == np.float32(1.0 + 2.0 ** -6)
    # just above halfway rounds up, just below rounds down
    assert OP.round_p24(np.float32(1.0 + 2.0 ** -16 + 2.0 ** -23)) == np.float32(1.0 + 2.0 ** -15)
    assert OP.round_p24(np.float32(1.0 + 2.0 ** -16 - 2.0 ** -23)) == np.float32(1.0)


def test_bit_patterns_of_the_formats():
    # the 24-bit result keeps the top 24 bits of the FP32 word: bits 0..7 are zero
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-60, 60, 20000))).astype(np.float32)
    b24 = OP.round_p24(x).view(np.uint32)
    b16 = OP.round_bf16(x).view(np.uint32)
    assert np.all(b24 & 0xFF == 0) and np.all(b16 & 0xFFFF == 0)
    # nearest: the neighbours on the grid are no closer
    for b, step in ((b24, 1 << 8), (b16, 1 << 16)):
        r = b.view(np.float32).astype(np.float64)
        up = (b + step).view(np.float32).astype(np.float64)
        dn = (b - step).view(np.float32).astype(np.float64)
        d = np.abs(r - x)
        assert np.all(d <= np.abs(up - x)) and np.all(d <= np.abs(dn - x))


def test_relative_error_bounds_and_idempotence():
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(50000) * np.exp(rng.uniform(-80, 80, 50000))).astype(np.float32)
    for fn, p in ((OP.round_bf16, 8), (OP.round_p24, 16)):
        y = fn(x)
        rel = np.abs(y.astype(np.float64) - x) / np.abs(x.astype(np.float64))
        assert rel.max() <= 2.0 ** -p
        assert np.array_equal(fn(y), y)
        assert np.array_equal(fn(-x), -y)  # symmetric


def test_carry_into_the_exponent_and_subnormals():
    # the largest value below 2 with 24 significant bits rounds up to 2
    x = np.float32(2.0 - 2.0 ** -23)
    assert OP.round_p24(x) == np.float32(2.0) and OP.round_bf16(x) == np.float32(2.0)
    # subnormals: the grid spacing is 2^-149 * 2^8 (24-bit) and 2^-149 * 2^16 (BF16)
    s = f32([0x00000180])  # 384 * 2^-149: halfway between 256 and 512 units -> 512 (even)
    assert OP.round_p24(s)[0] == f32([0x00000200])[0]
    s2 = f32([0x00000080])  # 128 units: halfway between 0 and 256 -> 0 (even)
    assert OP.round_p24(s2)[0] == 0.0


def test_rejects_bad_precision_and_non_finite():
    with pytest.raises(ValueError):
        OP.round_significant(np.float32(1.0), 0)
    with pytest.raises(ValueError):
        OP.round_bf16(np.array([np.inf], dtype=np.float32))
