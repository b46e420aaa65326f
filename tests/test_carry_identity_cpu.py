"""The identity behind the FP64-accuracy byte-carry recombination, on the CPU.

The slice GEMM sums the levels d = s+1 .. 2 (weights 2^(8(s+1-d))) in one
int32 register per output: after each level but the last it keeps the low
byte b_l of the running sum (final, since every later level adds multiples of
2^8 at that weight) and carries the rest, an arithmetic shift by 8, into the
next level. The total is then X = S 2^(8(s-1)) + sum_l b_l 2^(8l), rounded
once (half up) to the fixed point 2^shift. Here random level sums within the
kernel's bounds check that X is the exact total, that the running sum stays
inside int32, and that the rounding equals rounding the exact total.
"""
import random

import pytest

SEG_CHUNKS = 120
CHUNK_MAX = 2 ** 24          # |one chunk's exact f32 sum| <= 2^24


def carry_total(levels, s, shift):
    """levels[d] for d = s+1 .. 2 -> (rounded total, largest |running sum|)."""
    W = 8 * (s - 1)
    S, R, peak = 0, 0, 0
    for d in range(s + 1, 1, -1):
        S += levels[d]
        peak = max(peak, abs(S))
        if d > 2:
            l = s + 1 - d
            R |= (S & 255) << (8 * l)      # Python & on negatives is two's complement
            S >>= 8                        # floor division, the arithmetic shift
    if shift == 0:
        return (S << W) + R, peak
    return (S << (W - shift)) + ((R + (1 << (shift - 1))) >> shift), peak


@pytest.mark.parametrize("s", [3, 4, 5, 6, 7])
def test_byte_carry_is_the_exact_total(s):
    rng = random.Random(1000 + s)
    for trial in range(4000):
        # extremes included: every level at +-SEG_CHUNKS full chunks
        if trial < 4:
            sign = 1 if trial % 2 == 0 else -1
            levels = {d: sign * SEG_CHUNKS * CHUNK_MAX for d in range(2, s + 2)}
        else:
            levels = {d: rng.randint(-SEG_CHUNKS * CHUNK_MAX, SEG_CHUNKS * CHUNK_MAX) for d in range(2, s + 2)}
        X = sum(levels[d] << (8 * (s + 1 - d)) for d in levels)
        for shift in sorted({0, 1, 5, 8 * (s - 1)}):
            got, peak = carry_total(levels, s, shift)
            want = X if shift == 0 else (X + (1 << (shift - 1))) >> shift
            assert got == want, (s, shift, levels)
            assert peak < 2 ** 31


def test_a_dropped_carry_is_caught():
    # the same check with the carry left out (bytes kept, sum not shifted) fails
    s, shift = 5, 0
    levels = {d: 3 * 2 ** 20 + d for d in range(2, s + 2)}
    X = sum(levels[d] << (8 * (s + 1 - d)) for d in levels)
    W = 8 * (s - 1)
    S, R = 0, 0
    for d in range(s + 1, 1, -1):
        S += levels[d]
        if d > 2:
            R |= (S & 255) << (8 * (s + 1 - d))
    assert (S << W) + R != X
