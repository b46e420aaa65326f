"""Pins for the automatic FP64-accuracy slice count of the oracle.

The spread statistic is checked against hand-derived values; the slice count
against the property it exists for: the emulated product at the chosen s stays
within half the componentwise bound 4k 2^-53 |A||B| of the exact product, on
the workload distributions and on heavy-tailed ones, with the plain FP64
product taken where no s <= 7 qualifies. The exact products come from an
error-free product (Veltkamp splitting) summed by math.fsum, itself pinned
against rational arithmetic. Planted mistakes in copies of the statistic are
caught by the same property.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import emulation as em
from paper_2408_15384_gb300 import inputs


# ------------------------------------------------------------ exact products
def _split(x):
    """Veltkamp splitting: x = hi + lo with hi, lo of at most 26 significant bits."""
    c = 134217729.0 * x            # 2^27 + 1
    hi = c - (c - x)
    return hi, x - hi


def exact_product(A, B):
    """sum_k a_ik b_kj rounded once to double: every a*b is split error-free
    into p + e (Dekker's product), and math.fsum rounds the exact sum once."""
    A = np.asarray(A, float)
    B = np.asarray(B, float)
    m, n = A.shape[0], B.shape[1]
    C = np.zeros((m, n))
    Bh, Bl = _split(B)
    for i in range(m):
        a = A[i][:, None]
        ah, al = _split(a)
        p = a * B
        e = ((ah * Bh - p) + ah * Bl + al * Bh) + al * Bl
        for j in range(n):
            C[i, j] = math.fsum(np.concatenate([p[:, j], e[:, j]]))
    return C


def test_exact_product_against_rationals():
    A = inputs.box_muller(3, 37, 5, inputs.STREAM_A) * 1e3
    B = inputs.wide_spread(37, 4, 5, inputs.STREAM_B)
    C = exact_product(A, B)
    for i in range(3):
        for j in range(4):
            tot = sum(Fraction(float(A[i, x])) * Fraction(float(B[x, j])) for x in range(37))
            assert C[i, j] == float(tot)


def emulated_ratio(A, B, s):
    """max over outputs of |C_emu - C_exact| / (4k 2^-53 |A||B|)."""
    k = A.shape[1]
    C = em.gemm_fp64_emu(A, B, s) if s <= em.S_MAX else exact_product(A, B)
    bound = em.gamma(k, "fp64_emu") * (np.abs(A) @ np.abs(B))
    return float(np.max(np.abs(C - exact_product(A, B)) / bound))


# ------------------------------------------------------------ the statistic
def test_spread_closed_forms():
    k = 10
    A = np.zeros((5, k))
    A[0] = 3.0 * np.array([1, -1] * 5)            # |a| = 3: E = 1 + 2, alpha = 3/8
    A[1, 4] = -0.75                               # one entry: E = -1 + 2, alpha = 0.75 / (10 * 2)
    A[3] = 2.0 ** -1060                           # subnormal row: E = -1060 + 2, alpha = 1/4
    A[4, 2] = np.nan                              # non-finite: no constraint
    E = em.row_exponents(A, 2)
    al = em.row_spread(A, E)
    assert al[0] == 3.0 / 8.0
    assert al[1] == 0.75 / 20.0
    assert al[2] == math.inf                      # zero row: no constraint
    assert al[3] == 0.25
    assert al[4] == math.inf
    B = np.ascontiguousarray(A.T)
    assert np.array_equal(em.col_spread(B, em.col_exponents(B, 2)), al)


def test_spread_is_between_zero_and_a_half():
    A = inputs.wide_spread(16, 300, 3, inputs.STREAM_A)
    al = em.row_spread(A, em.row_exponents(A, 2))
    # |a| < 2^(E-1) for every entry, and the largest is at least 2^(E-2)
    assert np.all(al < 0.5) and np.all(al >= 0.25 / 300)


def test_rule_edges():
    assert em.slice_count_from_spread(100, math.inf, math.inf) == em.S_MIN
    assert em.slice_count_from_spread(100, 0.0, 0.25) == em.S_PLAIN
    # more terms or wider-spread rows never ask for fewer slices
    prev = em.S_PLAIN
    for k in [8, 64, 512, 4096, 32768, 1 << 20]:
        s = em.slice_count_from_spread(k, 0.25, 0.25)
        assert s <= prev
        prev = s
        assert em.slice_count_from_spread(k, 0.05, 0.25) >= s


def test_uniform_workload_at_8192_takes_five_slices():
    # the benchmark workload: rows and columns uniform[-1,1) * 2^e
    A = inputs.row_scaled(32, 8192, 3)
    B = inputs.col_scaled(8192, 32, 3)
    assert em.slice_count(A, B) == 5


# ------------------------------------------------------------ the property
DISTS = {
    "uniform": lambda r, c, seed, st: inputs.uniform(r, c, seed, st),
    "normal": lambda r, c, seed, st: inputs.box_muller(r, c, seed, st),
    "t3": lambda r, c, seed, st: inputs.student_t3(r, c, seed, st),
    "spread": lambda r, c, seed, st: inputs.wide_spread(r, c, seed, st),
}


@pytest.mark.parametrize("dist", sorted(DISTS))
@pytest.mark.parametrize("k", [7, 96, 700, 4096])
def test_chosen_count_keeps_half_the_bound(dist, k):
    m = 24 if k < 4096 else 12
    A = DISTS[dist](m, k, 100 + k, inputs.STREAM_A)
    B = DISTS[dist](k, m, 100 + k, inputs.STREAM_B)
    s = em.slice_count(A, B)
    assert emulated_ratio(A, B, s) <= em.THETA, (dist, k, s)


def test_cauchy_takes_the_plain_product():
    A = inputs.cauchy(12, 1000, 9, inputs.STREAM_A)
    B = inputs.cauchy(1000, 12, 9, inputs.STREAM_B)
    s = em.slice_count(A, B)
    assert s == em.S_PLAIN
    # with seven slices the bound would not hold
    assert emulated_ratio(A, B, em.S_MAX) > 1.0


def test_normal_rows_at_4096_need_six():
    # rows of normal deviates stand about 5 times above their mean: five
    # slices (enough for uniform rows at this k) leave the bound
    A = inputs.box_muller(12, 4096, 21, inputs.STREAM_A)
    B = inputs.box_muller(4096, 12, 21, inputs.STREAM_B)
    assert em.slice_count(A, B) == 6
    assert emulated_ratio(A, B, 5) > em.THETA


# ------------------------------------------------------------ planted mistakes
def _count_with(spread, A, B):
    k = A.shape[1]
    a = spread(A, em.row_exponents(A, 2))
    b = spread(np.ascontiguousarray(B.T), em.col_exponents(B, 2))
    return em.slice_count_from_spread(k, float(a.min()), float(b.min()))


def test_property_catches_planted_mistakes():
    k = 4096
    A = inputs.box_muller(12, k, 21, inputs.STREAM_A)
    B = inputs.box_muller(k, 12, 21, inputs.STREAM_B)

    def no_mean(X, E):       # sum instead of mean: the division by k dropped
        return em.row_spread(X, E) * X.shape[1]

    def max_not_mean(X, E):  # the largest entry instead of the mean
        return np.max(np.abs(X), axis=1) / np.ldexp(1.0, E)

    assert _count_with(em.row_spread, A, B) == em.slice_count(A, B)
    for bad in (no_mean, max_not_mean):
        s = _count_with(bad, A, B)
        assert emulated_ratio(A, B, s) > em.THETA, bad.__name__
