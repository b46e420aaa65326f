"""Shared helpers of the GPU tests (no method arithmetic)."""
import math

import numpy as np


def bf16_bits_of(values) -> np.ndarray:
    """bfloat16 bit patterns of values that are exactly bfloat16 (ints or doubles)."""
    f = np.asarray(values, dtype=np.float64).astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def fixed_shift(s: int, k: int) -> int:
    """The right shift the FP64-accuracy epilogue applies so the int64 total of
    sum_d 2^(8(s+1-d)) L_d (|L_d| <= k (d-1) 2^14) stays below 2^62."""
    tot = sum(j * 2.0 ** (8 * (s - j)) for j in range(1, s + 1))
    bits = math.log2(2.0 ** 14 * max(k, 1) * tot)
    return max(0, math.ceil(bits + 1e-9) - 62)


def bound_ok(C, C_ref, D, gamma):
    """|C - C_ref| <= gamma * |A||B| elementwise (NaN-free)."""
    return np.all(np.abs(C - C_ref) <= gamma * D)


def max_ratio(C, C_ref, D, gamma):
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.abs(C - C_ref) / (gamma * D)
    r[(D == 0) & (C == C_ref)] = 0.0
    return float(np.nanmax(r)) if r.size else 0.0
