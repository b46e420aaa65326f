"""Pins for the FP64 triple-loop oracle (Sec. III definition, Sec. V program).

Each check compares the oracle with something it does not compute itself:
hand-worked products, closed forms (identity, permutation, rank one),
exactness of small-integer products, the transpose identity, and exact
rational brute force on tiny shapes with the standard inner-product bound.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2408_15384_gb300 import inputs

U = 2.0 ** -53


def test_textbook_golden(golden_dir):
    for case in json.load(open(os.path.join(golden_dir, "textbook.json"))):
        C = oracle.gemm(np.array(case["A"], float), np.array(case["B"], float))
        assert np.array_equal(C, np.array(case["C"], float)), case["cite"]


@pytest.mark.parametrize("m,k", [(1, 1), (5, 7), (33, 17), (64, 64)])
def test_identity(m, k):
    A = inputs.uniform(m, k, 11, inputs.STREAM_A)
    assert np.array_equal(oracle.gemm(A, np.eye(k)), A)
    assert np.array_equal(oracle.gemm(np.eye(m), A), A)


def test_permutation():
    rng = np.random.default_rng(3)
    A = inputs.uniform(23, 19, 12, inputs.STREAM_A)
    perm = rng.permutation(23)
    P = np.zeros((23, 23))
    P[np.arange(23), perm] = 1.0
    # (P A)[i] = A[perm[i]]; compare with == so -0 and +0 agree
    assert np.all(oracle.gemm(P, A) == A[perm])
    # column permutation from the right
    cperm = rng.permutation(19)
    Q = np.zeros((19, 19))
    Q[cperm, np.arange(19)] = 1.0
    assert np.all(oracle.gemm(A, Q) == A[:, cperm])


@pytest.mark.parametrize("m,n,k", [(4, 5, 1), (7, 3, 64), (16, 16, 1000)])
def test_rank_one_closed_form(m, n, k):
    # A = u 1^T, B = 1 w^T with dyadic u, w of few bits: C_ij = k u_i w_j exactly
    rng = np.random.default_rng(m * n + k)
    u = rng.integers(-64, 65, m) / 64.0
    w = rng.integers(-64, 65, n) / 16.0
    A = np.repeat(u[:, None], k, axis=1)
    B = np.repeat(w[None, :], k, axis=0)
    assert np.array_equal(oracle.gemm(A, B), k * np.outer(u, w))


def test_k1_is_rounded_product():
    a = inputs.uniform(9, 1, 5, inputs.STREAM_A)
    b = inputs.uniform(1, 11, 5, inputs.STREAM_B)
    C = oracle.gemm(a, b)
    for i in range(9):
        for j in range(11):
            assert C[i, j] == float(Fraction(a[i, 0]) * Fraction(b[0, j]))


@pytest.mark.parametrize("m,n,k", [(8, 8, 8), (31, 17, 300), (5, 40, 2048)])
def test_small_integers_exact(m, n, k):
    rng = np.random.default_rng(k)
    A = rng.integers(-8, 9, (m, k)).astype(float)
    B = rng.integers(-8, 9, (k, n)).astype(float)
    exact = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(oracle.gemm(A, B), exact.astype(float))


def test_transpose_identity():
    A = inputs.uniform(13, 29, 21, inputs.STREAM_A)
    B = inputs.uniform(29, 7, 21, inputs.STREAM_B)
    C = oracle.gemm(A, B)
    Ct = oracle.gemm(np.ascontiguousarray(B.T), np.ascontiguousarray(A.T))
    # same products in the same k order: bit-identical
    assert np.array_equal(C, Ct.T)


def test_brute_force_rational_tiny():
    rng = np.random.default_rng(7)
    for trial in range(300):
        m, n, k = rng.integers(1, 9, 3)
        A = inputs.uniform(m, k, 100 + trial, inputs.STREAM_A)
        B = inputs.uniform(k, n, 100 + trial, inputs.STREAM_B)
        C = oracle.gemm(A, B)
        D = oracle.absprod(A, B)
        for i in range(m):
            for j in range(n):
                exact = sum(Fraction(A[i, p]) * Fraction(B[p, j]) for p in range(k))
                err = abs(Fraction(C[i, j]) - exact)
                # standard inner-product bound |fl - exact| <= gamma_k |A||B|
                gk = k * U / (1 - k * U)
                assert err <= Fraction(gk) * Fraction(D[i, j]) + Fraction(0), (m, n, k, i, j)


def test_absprod_matches_definition():
    A = inputs.uniform(6, 9, 3, inputs.STREAM_A)
    B = inputs.uniform(9, 4, 3, inputs.STREAM_B)
    D = oracle.absprod(A, B)
    assert np.all(D >= 0)
    # |A||B| >= |AB| entrywise (triangle inequality), equality for nonnegative inputs
    assert np.all(D >= np.abs(oracle.gemm(A, B)) * (1 - 1e-15))
    assert np.array_equal(oracle.absprod(np.abs(A), np.abs(B)), oracle.gemm(np.abs(A), np.abs(B)))


def test_rows_dot_and_omp_agree_with_full():
    A = inputs.uniform(40, 33, 8, inputs.STREAM_A)
    B = inputs.uniform(33, 21, 8, inputs.STREAM_B)
    C = oracle.gemm(A, B)
    assert np.array_equal(oracle.gemm_rows(A, B, [0, 39, 17]), C[[0, 39, 17]])
    assert oracle.dot(A, B, 12, 20) == C[12, 20]
    Cr, used = oracle.gemm_omp_rows(A, B, 5, 35, 4)
    assert np.array_equal(Cr, C[5:35]) and used >= 1
    D = oracle.absprod(A, B)
    assert np.array_equal(oracle.absprod_rows(A, B, [3, 9]), D[[3, 9]])
    # the parallel sampled-row helpers give the serial loop's bits
    assert np.array_equal(oracle.gemm_rows_par(A, B, [39, 2, 17]), C[[39, 2, 17]])
    assert np.array_equal(oracle.absprod_rows_par(A, B, [39, 2, 17]), D[[39, 2, 17]])


def test_ieee_special_values_propagate():
    A = np.array([[np.inf, 1.0], [np.nan, 0.0], [1.0, 2.0]])
    B = np.array([[1.0, 0.0], [2.0, 3.0]])
    C = oracle.gemm(A, B)
    assert C[0, 0] == np.inf and np.isnan(C[0, 1])  # inf*0 = nan
    assert np.isnan(C[1, 0]) and np.isnan(C[1, 1])
    assert C[2, 0] == 5.0 and C[2, 1] == 6.0


def test_empty_shapes():
    assert oracle.gemm(np.zeros((0, 3)), np.zeros((3, 4))).shape == (0, 4)
    assert np.array_equal(oracle.gemm(np.zeros((2, 0)), np.zeros((0, 3))), np.zeros((2, 3)))


@pytest.mark.parametrize("m,n,k", [(37, 300, 261), (64, 17, 1000), (5, 513, 3)])
def test_cpu_variants_equal_the_oracle(m, n, k):
    # the paper's column-prefetching and cache-tiling loops take each element's
    # products in the oracle's order, so they return the oracle's bits
    from paper_2408_15384_gb300 import inputs
    A = inputs.row_scaled(m, k, 51)
    B = inputs.col_scaled(k, n, 51)
    ref = oracle.gemm(A, B)
    for fn in (oracle.gemm_colprefetch_rows, oracle.gemm_tiled_rows):
        C, used = fn(A, B, 0, m, 3)
        assert used >= 1 and np.array_equal(C, ref), fn.__name__
        part, _ = fn(A, B, 2, m - 1, 2)
        assert np.array_equal(part, ref[2:m - 1])
