"""Pins for the INT8 digit form of the FP64-accuracy oracle.

The INT8 form holds every digit in a signed byte: its scale exponent is one
larger (offset 3), so the top digit stays within [-64, 64]. Checked against
exact rational digits, the byte range on rows whose entries sit at the very
top of their binade, the level products by brute force, the emulated result
within half the bound of the exact product at the INT8 form's automatic
slice count, and a planted mistake (the bfloat16 form's offset) that breaks
the byte range.
"""
import math

import numpy as np
import pytest

from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

from test_oracle_emulation import pin_digits, pin_levels
from test_oracle_slice_count import DISTS, emulated_ratio, exact_product


def extreme_rows(m, k, seed):
    """Rows whose largest entry is the largest double below a power of two (the
    case that sends a bfloat16-form top digit to 128)."""
    A = inputs.uniform(m, k, seed, inputs.STREAM_A)
    for i in range(m):
        j = i % k
        A[i, j] = math.copysign(math.ldexp(1.0 - 2.0 ** -53, i % 5 - 2), A[i, j] if A[i, j] != 0 else 1.0)
    return A


def test_int8_digits_exact_and_in_byte_range():
    A = extreme_rows(24, 40, 3)
    for s in (3, 5, 7):
        E, sig = em.fp64_slices_A(A, s, offset=em.OFFSET_INT8)
        assert pin_digits(A, E, sig, s)
        assert sig.min() >= -128 and sig.max() <= 127
        assert np.all(np.abs(sig[0]) <= 64)


def test_int8_columns_of_B():
    B = np.ascontiguousarray(extreme_rows(12, 30, 4).T)
    F, sig = em.fp64_slices_B(B, 4, offset=em.OFFSET_INT8)
    assert sig.min() >= -128 and sig.max() <= 127
    assert pin_digits(B.T.copy(), F, np.transpose(sig, (0, 2, 1)), 4)


def test_bfloat16_offset_would_leave_the_byte_range():
    # planted: the bfloat16 form's exponent offset sends some top digit to 128
    A = extreme_rows(24, 40, 3)
    _, sig = em.fp64_slices_A(A, 5, offset=em.OFFSET_BF16)
    assert sig.max() == 128


def test_int8_level_products_brute_force():
    A = inputs.row_scaled(4, 7, 9)
    B = inputs.col_scaled(7, 3, 9)
    s = 4
    _, sA = em.fp64_slices_A(A, s, offset=em.OFFSET_INT8)
    _, sB = em.fp64_slices_B(B, s, offset=em.OFFSET_INT8)
    assert pin_levels(sA, sB, em.level_products(sA, sB, s), s)


@pytest.mark.parametrize("dist", ["uniform", "normal", "spread"])
@pytest.mark.parametrize("k", [96, 700, 4096])
def test_int8_count_keeps_half_the_bound(dist, k):
    m = 16 if k < 4096 else 10
    A = DISTS[dist](m, k, 300 + k, inputs.STREAM_A)
    B = DISTS[dist](k, m, 300 + k, inputs.STREAM_B)
    s = em.slice_count_int8(A, B)
    assert s >= em.slice_count(A, B)        # a coarser grid never needs fewer slices
    if s <= em.S_MAX:
        C = em.gemm_fp64_emu(A, B, s, offset=em.OFFSET_INT8)
        bound = em.gamma(k, "fp64_emu") * (np.abs(A) @ np.abs(B))
        assert np.max(np.abs(C - exact_product(A, B)) / bound) <= em.THETA, (dist, k, s)
    else:
        assert emulated_ratio(A, B, s) <= em.THETA
