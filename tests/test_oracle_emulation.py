"""Pins for the split-precision oracle (oracle/emulation.py).

The FP64-accuracy splitting is checked against hand-worked digits, exact
rational arithmetic (round-half-even of the scaled entry), the digit bounds,
brute-force integer level products, and closed forms where the emulation is
exact (small integers). The FP32-accuracy splitting is checked against
hand-worked bfloat16 splits and brute-force nearest-bfloat16 search. A last
group plants plausible mistakes in copies of the oracle functions and checks
that these pins catch them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

T = em.T_BITS


# ---------------------------------------------------------------- pin helpers
def pin_exponents(A, E, offset):
    """2^(E-offset) <= max|a_i| < 2^(E-offset+1) row by row, E=0 for zero rows."""
    for i in range(A.shape[0]):
        mx = max((abs(Fraction(x)) for x in A[i]), default=Fraction(0))
        if mx == 0:
            if E[i] != 0:
                return False
            continue
        lo = Fraction(2) ** (int(E[i]) - offset)
        if not (lo <= mx < 2 * lo):
            return False
    return True


def rne(fr: Fraction) -> int:
    return round(fr)  # Python rounds Fractions half to even


def pin_digits(A, E, sig, s):
    """R = rne(a*2^(ts-E)) exactly, R = sum sigma_p 2^(t(s-p)), digit bounds."""
    half = 1 << (T - 1)
    for i in range(A.shape[0]):
        for c in range(A.shape[1]):
            R = rne(Fraction(A[i, c]) * Fraction(2) ** (T * s - int(E[i])))
            val = sum(int(sig[p, i, c]) << (T * (s - 1 - p)) for p in range(s))
            if val != R:
                return False
            if abs(int(sig[0, i, c])) > half:
                return False
            for p in range(1, s):
                if not (-half <= int(sig[p, i, c]) < half):
                    return False
    return True


def pin_levels(sA, sB, L, s):
    """Brute force: L_d[i,j] = sum over p+q=d and k of sA[p][i,k]*sB[q][k,j]."""
    m, k = sA.shape[1], sA.shape[2]
    n = sB.shape[2]
    for d in range(2, s + 2):
        for i in range(m):
            for j in range(n):
                tot = 0
                for p in range(1, d):
                    q = d - p
                    if p <= s and q <= s:
                        tot += sum(int(sA[p - 1, i, x]) * int(sB[q - 1, x, j]) for x in range(k))
                if tot != int(L[d - 2, i, j]):
                    return False
    return True


def pin_recombine(sA, sB, E, F, C, s):
    """Pair form: C_ij = RN(sum_{p+q<=s+1} sA_p.sB_q 2^(E_i+F_j-t(p+q))), exact rationals."""
    m, k = sA.shape[1], sA.shape[2]
    n = sB.shape[2]
    for i in range(m):
        for j in range(n):
            tot = Fraction(0)
            for p in range(1, s + 1):
                for q in range(1, s + 2 - p):
                    dotpq = sum(int(sA[p - 1, i, x]) * int(sB[q - 1, x, j]) for x in range(k))
                    tot += Fraction(dotpq) * Fraction(2) ** (int(E[i]) + int(F[j]) - T * (p + q))
            if float(tot) != C[i, j]:
                return False
    return True


# ---------------------------------------------------------------- golden
def test_digits_golden(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "digits_t8.json")))
    assert g["t"] == T
    for case in g["cases"]:
        row = np.array([case["row"]], float)
        s = case["s"]
        E = em.row_exponents(row, 2)
        assert int(E[0]) == case["E"], case["why"]
        R = em.integer_repr(row, E, s)
        assert R[0].tolist() == case["R"], case["why"]
        sig = em.balanced_digits(R, s)
        assert [[int(sig[p, 0, c]) for p in range(s)] for c in range(row.shape[1])] == case["digits"], case["why"]


def test_bf16_golden(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "bf16_slices.json")))
    for case in g["cases"]:
        sl = em.fp32_slices(np.array([case["r"]]))
        assert [float(x[0]) for x in sl] == case["slices"], case["why"]


# ---------------------------------------------------------------- exponents
def test_exponents_brackets_and_special_rows():
    A = inputs.row_scaled(20, 13, 4)
    A[3] = 0.0
    A[5, :] = 0.0
    A[5, 7] = 5e-324  # smallest subnormal
    A[6, :] = 0.0
    A[6, 2] = -2.0 ** 1000
    for off in (1, 2):
        E = em.row_exponents(A, off)
        assert pin_exponents(A, E, off)
    assert em.row_exponents(A, 2)[5] == -1074 + 2
    assert em.row_exponents(A, 2)[6] == 1002
    Bm = inputs.col_scaled(13, 9, 4)
    assert pin_exponents(Bm.T, em.col_exponents(Bm, 2), 2)


# ---------------------------------------------------------------- digits
@pytest.mark.parametrize("s", [1, 2, 5, 7])
def test_digits_exact_rational(s):
    A = inputs.row_scaled(6, 11, 30 + s)
    A[2, 3] = 0.0
    A[4, 0] = 1e-300
    E, sig = em.fp64_slices_A(A, s)
    assert pin_digits(A, E, sig, s)


def test_digits_columns_of_B():
    B = inputs.col_scaled(9, 5, 3)
    F, sig = em.fp64_slices_B(B, 3)
    assert sig.shape == (3, 9, 5)
    assert pin_digits(B.T.copy(), F, np.transpose(sig, (0, 2, 1)), 3)


def test_digits_fit_bfloat16_exactly():
    A = inputs.row_scaled(16, 64, 9)
    _, sig = em.fp64_slices_A(A, 6)
    assert np.all(np.abs(sig) <= 128)
    # every integer of magnitude <= 256 is a bfloat16 value
    assert np.array_equal(em.bf16_round(sig.astype(float)), sig.astype(float))


# ---------------------------------------------------------------- levels
def test_level_products_brute_force():
    A = inputs.row_scaled(4, 6, 5)
    B = inputs.col_scaled(6, 3, 5)
    s = 4
    E, sA = em.fp64_slices_A(A, s)
    F, sB = em.fp64_slices_B(B, s)
    L = em.level_products(sA, sB, s)
    assert pin_levels(sA, sB, L, s)


def test_recombine_pair_form():
    A = inputs.row_scaled(3, 5, 6)
    B = inputs.col_scaled(5, 4, 6)
    s = 3
    E, sA = em.fp64_slices_A(A, s)
    F, sB = em.fp64_slices_B(B, s)
    C = em.recombine_exact(em.level_products(sA, sB, s), E, F, s)
    assert pin_recombine(sA, sB, E, F, C, s)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("s", [5, 6, 7])
def test_small_integer_products_exact(s):
    rng = np.random.default_rng(s)
    A = rng.integers(-8, 9, (9, 40)).astype(float)
    B = rng.integers(-8, 9, (40, 7)).astype(float)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(float)
    assert np.array_equal(em.gemm_fp64_emu(A, B, s), exact)
    assert np.array_equal(em.gemm_fp32_emu(A, B), exact)


def test_two_digit_integers_exact():
    # entries up to 2^12 need two digits; s >= 3 keeps every level they reach
    rng = np.random.default_rng(1)
    A = rng.integers(-4096, 4097, (5, 17)).astype(float)
    B = rng.integers(-4096, 4097, (17, 6)).astype(float)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(float)
    assert np.array_equal(em.gemm_fp64_emu(A, B, 3), exact)


def test_identity_and_permutation_dyadic():
    # dyadic entries of <= 24 significant bits relative to the row max are exact
    rng = np.random.default_rng(2)
    A = rng.integers(-2 ** 20, 2 ** 20, (6, 6)) / 2.0 ** 20
    I = np.eye(6)
    assert np.array_equal(em.gemm_fp64_emu(A, I, 5), A)
    assert np.array_equal(em.gemm_fp32_emu(A, I), A)
    P = np.eye(6)[[3, 0, 5, 1, 4, 2]]
    assert np.all(em.gemm_fp64_emu(P, A, 5) == A[[3, 0, 5, 1, 4, 2]])


def test_transpose_identity_emulated():
    A = inputs.row_scaled(7, 12, 8)
    B = inputs.col_scaled(12, 5, 8)
    C = em.gemm_fp64_emu(A, B, 6)
    Ct = em.gemm_fp64_emu(np.ascontiguousarray(B.T), np.ascontiguousarray(A.T), 6)
    # row scaling of A becomes column scaling of A^T: the same integers meet
    assert np.array_equal(C, Ct.T)


def test_within_bound_on_workload_inputs():
    # the acceptance bound against the triple-loop oracle, k spanning the slice rule
    for k, s in [(5, 7), (40, 7), (100, 6), (700, 6)]:
        A = inputs.row_scaled(6, k, k)
        B = inputs.col_scaled(k, 5, k)
        C = oracle.gemm(A, B)
        D = oracle.absprod(A, B)
        Ce = em.gemm_fp64_emu(A, B, s)
        assert np.all(np.abs(Ce - C) <= em.gamma(k, "fp64") * D), k
        Cf = em.gemm_fp32_emu(A, B)
        assert np.all(np.abs(Cf - C) <= em.gamma(k, "fp32") * D), k


# ---------------------------------------------------------------- bfloat16
def _bf16_neighbours(x):
    """All bfloat16 values adjacent to x (brute force on the float32 bit grid)."""
    f = np.float32(x)
    bits = int(np.array([f], np.float32).view(np.uint32)[0]) & 0xFFFF0000
    out = []
    for d in (-2, -1, 0, 1, 2):
        b = (bits + d * 0x10000) & 0xFFFFFFFF
        out.append(float(np.array([b], np.uint32).view(np.float32)[0]))
    return out


def test_bf16_round_is_nearest():
    xs = inputs.uniform(1, 400, 77, inputs.STREAM_A)[0] * 2.0 ** np.arange(-60, 40, 0.25)
    r = em.bf16_round(xs)
    for x, y in zip(xs, r):
        cands = [c for c in _bf16_neighbours(x) if math.isfinite(c)]
        best = min(abs(Fraction(c) - Fraction(x)) for c in cands)
        assert abs(Fraction(y) - Fraction(x)) == best
        assert y in cands


def test_fp32_slices_reconstruct():
    r = inputs.uniform(1, 500, 3, inputs.STREAM_A)[0]
    sl = em.fp32_slices(r)
    rec = sl[0] + sl[1] + sl[2]
    assert np.all(np.abs(rec - r) <= 2.0 ** -24 * np.abs(r))
    for p in range(3):
        assert np.array_equal(em.bf16_round(sl[p]), sl[p])


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes():
    A = inputs.row_scaled(4, 6, 12)
    B = inputs.col_scaled(6, 3, 12)
    s = 3
    E, sA = em.fp64_slices_A(A, s)
    F, sB = em.fp64_slices_B(B, s)
    L = em.level_products(sA, sB, s)
    C = em.recombine_exact(L, E, F, s)
    assert pin_exponents(A, E, 2) and pin_digits(A, E, sA, s)
    assert pin_levels(sA, sB, L, s) and pin_recombine(sA, sB, E, F, C, s)
    # off-by-one scale exponent
    assert not pin_exponents(A, E + 1, 2)
    # a digit with the wrong sign
    bad = sA.copy(); bad[1] = -bad[1]
    assert not pin_digits(A, E, bad, s)
    # digits in reversed significance order
    assert not pin_digits(A, E, sA[::-1].copy(), s)
    # a dropped pair in one level
    Lbad = L.copy(); Lbad[1] -= sA[0] @ sB[1]
    assert not pin_levels(sA, sB, Lbad, s)
    # a transposed operand in the level product
    Lt = L.copy(); Lt[0] = (sA[0] @ sB[0])
    assert pin_levels(sA, sB, Lt, s)  # unchanged is fine ...
    Lt[0] = (sA[0][:, :3] @ sB[0][:3, :])  # ... a truncated k range is not
    assert not pin_levels(sA, sB, Lt, s)
    # a wrong level weight in the recombination
    Cbad = em.recombine_exact(L[::-1].copy(), E, F, s)
    assert not pin_recombine(sA, sB, E, F, Cbad, s)


# ---------------------------------------------------------------- FP32-accuracy pair count
def test_fp32_pair_count_by_k():
    assert em.fp32_pairs(511) == em.FP32_PAIRS and len(em.FP32_PAIRS) == 6
    assert em.fp32_pairs(512) == [(0, 0), (0, 1), (1, 0)]


@pytest.mark.parametrize("k", [500, 512, 2048])
def test_fp32_within_half_the_bound_worst_signs(k):
    # all entries positive: the left-out products all add up, nothing cancels
    from test_oracle_slice_count import exact_product
    A = np.abs(inputs.wide_spread(6, k, 70 + k, inputs.STREAM_A)) + 2.0 ** -30
    B = np.abs(inputs.uniform(k, 5, 70 + k, inputs.STREAM_B)) + 2.0 ** -30
    ratio = np.max(np.abs(em.gemm_fp32_emu(A, B) - exact_product(A, B)) / (em.gamma(k, "fp32_emu") * (A @ B)))
    assert ratio <= 0.5, (k, ratio)


def test_fp32_planted_single_pair_fails():
    # planted: only (0, 0) kept -- the 2^-8 rounding of the first slice shows
    from test_oracle_slice_count import exact_product
    k = 512
    A = np.abs(inputs.uniform(4, k, 5, inputs.STREAM_A)) + 0.1
    B = np.abs(inputs.uniform(k, 3, 5, inputs.STREAM_B)) + 0.1
    E, sA = em.fp32_slices_A(A)
    F, sB = em.fp32_slices_B(B)
    C = np.ldexp(np.ldexp(sA[0] @ sB[0], E[:, None]), F[None, :])
    ratio = np.max(np.abs(C - exact_product(A, B)) / (em.gamma(k, "fp32_emu") * (A @ B)))
    assert ratio > 1.0
