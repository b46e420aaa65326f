"""Pins for the modular (Chinese-remainder) form of the FP64-accuracy product
in the oracle (Ozaki scheme II).

Each step is pinned against something other than itself: residues against
hand-derived values and a brute-force congruence check, the rebuild against
exact Python-integer matrix products (and hand-derived values), the rounding
against closed forms, the whole product against exact integer products and
against the exact product within half the componentwise bound 4k 2^-53 |A||B|,
and the parameter rule against the inequalities that define it. Planted
mistakes (a missing modulus, no centring, too few bits) fail these pins.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import emulation as em
from paper_2408_15384_gb300 import inputs
from test_oracle_slice_count import emulated_ratio, exact_product

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "crt_residues.json")))


# ------------------------------------------------------------ the moduli
def test_moduli_pairwise_coprime_and_exact_in_bf16():
    ms = em.CRT_MODULI
    assert all(2 <= m <= 256 for m in ms)
    for i in range(len(ms)):
        for j in range(i + 1, len(ms)):
            assert math.gcd(ms[i], ms[j]) == 1, (ms[i], ms[j])
    # every centred residue lies in [-128, 127]; all of those are bfloat16 values
    vals = np.arange(-128, 128, dtype=np.float64)
    assert np.array_equal(em.bf16_round(vals), vals)
    # greedy: no larger integer <= 256 is coprime to all the chosen ones before it
    chosen = []
    for m in ms:
        for c in range(m + 1, 257):
            if c not in chosen:
                assert any(math.gcd(c, x) > 1 for x in chosen), (c, m)
        chosen.append(m)


# ------------------------------------------------------------ residues
def test_golden_residues():
    for r in GOLDEN["residues"]:
        l = em.CRT_MODULI.index(r["m"])
        got = em.crt_residues(np.array([r["R"]]), l + 1)[l, 0]
        assert got == r["rho"], r


def test_residues_brute_force():
    R = np.arange(-3000, 3001, dtype=np.int64)
    rho = em.crt_residues(R, em.CRT_N_MAX)
    for l, m in enumerate(em.CRT_MODULI):
        assert np.all((R - rho[l]) % m == 0)
        assert np.all(rho[l] >= -(m // 2)) and np.all(rho[l] <= (m + 1) // 2 - 1)


def test_residues_of_the_largest_scaled_integers():
    b = em.CRT_B_MAX
    R = np.array([2 ** (b - 1), -(2 ** (b - 1)), 2 ** (b - 1) - 1, 123456789012345], dtype=np.int64)
    rho = em.crt_residues(R, em.CRT_N_MAX)
    for l, m in enumerate(em.CRT_MODULI):
        for i in range(R.size):
            assert (int(R[i]) - int(rho[l, i])) % m == 0


# ------------------------------------------------------------ rebuild
def test_golden_rebuilds():
    for r in GOLDEN["rebuild"]:
        N = len(r["moduli"])
        assert tuple(r["moduli"]) == em.CRT_MODULI[:N]
        P = np.array(r["residues"], dtype=np.int64).reshape(N, 1, 1)
        assert em.crt_reconstruct(P)[0, 0] == r["Y"]


def _int_matmul(RA, RB):
    m, k = RA.shape
    n = RB.shape[1]
    return np.array([[sum(int(RA[i, x]) * int(RB[x, j]) for x in range(k)) for j in range(n)] for i in range(m)],
                    dtype=object)


def _rand_ints(rows, cols, b, seed, stream):
    """integers uniform on [-2^(b-1), 2^(b-1)] from the seeded words"""
    w = inputs.words(seed, stream, rows * cols).astype(object)
    span = (1 << b) + 1
    return np.array([int(x) % span - (1 << (b - 1)) for x in w], dtype=object).reshape(rows, cols).astype(np.int64)


@pytest.mark.parametrize("b,k", [(8, 5), (20, 37), (37, 64), (45, 300), (53, 3)])
def test_rebuild_equals_the_exact_integer_product(b, k):
    N = next(n for n in range(1, em.CRT_N_MAX + 1) if em.crt_fits(k, b, n))
    RA = _rand_ints(5, k, b, 7 + b, inputs.STREAM_A)
    RB = _rand_ints(k, 4, b, 7 + b, inputs.STREAM_B)
    RA[0, :] = 1 << (b - 1)           # the extremes: row 0 x column 0 is the largest sum,
    RB[:, 0] = 1 << (b - 1)           # row 1 x column 0 the most negative
    RA[1, :] = -(1 << (b - 1))
    Y = em.crt_reconstruct(em.crt_products(em.crt_residues(RA, N), em.crt_residues(RB, N)))
    want = _int_matmul(RA, RB)
    assert np.array_equal(Y, want)
    assert Y[0, 0] == k << (2 * b - 2) and Y[1, 0] == -(k << (2 * b - 2))


def test_rebuild_planted_mistakes():
    b, k = 37, 64
    N = next(n for n in range(1, em.CRT_N_MAX + 1) if em.crt_fits(k, b, n))
    assert not em.crt_fits(k, b, N - 1)
    RA = _rand_ints(5, k, b, 3, inputs.STREAM_A)
    RB = _rand_ints(k, 4, b, 3, inputs.STREAM_B)
    P = em.crt_products(em.crt_residues(RA, N), em.crt_residues(RB, N))
    want = _int_matmul(RA, RB)
    assert np.array_equal(em.crt_reconstruct(P), want)
    # one modulus dropped: the sums no longer fit and the rebuild wraps
    assert not np.array_equal(em.crt_reconstruct(P[: N - 1]), want)

    # no centring: the rebuild's [0, M) value is wrong for every negative output
    def uncentred(P):
        M = em.crt_modulus_product(P.shape[0])
        Y = em.crt_reconstruct(P)
        return np.vectorize(lambda y: y % M, otypes=[object])(Y)

    assert any(w < 0 for w in want.ravel())
    assert not np.array_equal(uncentred(P), want)


# ------------------------------------------------------------ rounding
def test_round_closed_forms():
    E = np.array([0])
    F = np.array([0])

    def rnd(Y, e):     # Y * 2^e with b = 0: the exponent is E + F - 2b = e
        return em.crt_round(np.array([[Y]], dtype=object), E + e, F, 0)[0, 0]

    assert rnd(3, -1) == 1.5
    assert rnd(-3, -1) == -1.5
    assert rnd((1 << 54) + 2, 0) == 2.0 ** 54                      # tie, even significand below
    assert rnd((1 << 54) + 6, 0) == 2.0 ** 54 + 8                  # tie, even significand above
    assert rnd((1 << 54) + 3, 0) == 2.0 ** 54 + 4
    assert rnd(1, -1074) == 5e-324
    assert rnd(1, -1075) == 0.0                                    # half the least subnormal: to even (zero)
    assert rnd(3, -1075) == 2 * 5e-324                             # 1.5 units: to even (two)
    assert rnd(0, 10) == 0.0


# ------------------------------------------------------------ the whole product
def test_golden_product():
    g = GOLDEN["product"]
    A = np.array(g["A"])
    B = np.array(g["B"])
    b, N = g["b"], g["N"]
    assert em.crt_fits(A.shape[1], b, N) and not em.crt_fits(A.shape[1], b, N - 1)
    E = em.row_exponents(A, 2)
    F = em.col_exponents(B, 2)
    assert list(E) == g["E"] and list(F) == g["F"]
    RA = em.crt_integer_repr(A, E, b)
    RB = em.crt_integer_repr(B.T, F, b).T
    assert RA.tolist() == g["RA"] and RB.tolist() == g["RB"]
    P = em.crt_products(em.crt_residues(RA, N), em.crt_residues(RB, N))
    assert [int(P[l, 0, 0]) for l in range(N)] == g["P"]
    assert [int(P[l, 0, 0]) % em.CRT_MODULI[l] for l in range(N)] == g["c"]
    assert em.crt_reconstruct(P)[0, 0] == g["Y"]
    assert em.gemm_fp64_crt(A, B, b, N).tolist() == g["C"]


def test_small_integers_exact():
    k = 700
    A = np.round(inputs.uniform(9, k, 5, inputs.STREAM_A) * 8)
    B = np.round(inputs.uniform(k, 6, 5, inputs.STREAM_B) * 8)
    b, N = em.crt_params(A, B)
    assert np.array_equal(em.gemm_fp64_crt(A, B, b, N), A @ B)   # integer sums below 2^53: exact in numpy


def test_identity_exact_for_short_entries():
    # entries with at most b - 2 bits below their row maximum's leading bit
    # survive the scaling, so A * I reproduces A bit for bit
    k = 40
    b = 30
    A = np.ldexp(np.round(inputs.uniform(6, k, 11, inputs.STREAM_A) * 2 ** 20), -20)
    N = next(n for n in range(1, em.CRT_N_MAX + 1) if em.crt_fits(k, b, n))
    assert np.array_equal(em.gemm_fp64_crt(A, np.eye(k), b, N), A)


DISTS = {
    "uniform": lambda r, c, seed, st: inputs.uniform(r, c, seed, st),
    "normal": lambda r, c, seed, st: inputs.box_muller(r, c, seed, st),
    "t3": lambda r, c, seed, st: inputs.student_t3(r, c, seed, st),
    "spread": lambda r, c, seed, st: inputs.wide_spread(r, c, seed, st),
}


def crt_ratio(A, B, b, N):
    k = A.shape[1]
    bound = em.gamma(k, "fp64_emu") * (np.abs(A) @ np.abs(B))
    return float(np.max(np.abs(em.gemm_fp64_crt(A, B, b, N) - exact_product(A, B)) / bound))


@pytest.mark.parametrize("dist", sorted(DISTS))
@pytest.mark.parametrize("k", [7, 96, 700, 2048])
def test_chosen_parameters_keep_half_the_bound(dist, k):
    m = 12 if k < 2048 else 6
    A = DISTS[dist](m, k, 300 + k, inputs.STREAM_A)
    B = DISTS[dist](k, m, 300 + k, inputs.STREAM_B)
    d = em.fp64_scheme(A, B)
    if d[0] == "crt":
        r = crt_ratio(A, B, d[1], d[2])
    else:
        # the modular form cannot reach the target (short sums need more than
        # its 53 bits, or more moduli than it has): the digit form decides
        assert em.crt_params(A, B) is None
        r = emulated_ratio(A, B, d[1] if d[0] == "digits" else em.S_PLAIN)
    assert r <= em.THETA, (dist, k, d)


def test_too_few_bits_leave_the_bound():
    k = 2048
    A = inputs.box_muller(6, k, 41, inputs.STREAM_A)
    B = inputs.box_muller(k, 6, 41, inputs.STREAM_B)
    b, N = em.crt_params(A, B)
    assert crt_ratio(A, B, b, N) <= em.THETA
    # the rule's smallest qualifying bit count, then five bits fewer (the
    # estimate covers 2^30 outputs, so with these 36 the margin is wide)
    al = float(em.row_spread(A, em.row_exponents(A, 2)).min())
    be = float(em.col_spread(B, em.col_exponents(B, 2)).min())
    rhs = em.THETA * 4.0 * k * math.sqrt(k) * al * be
    b0 = next(x for x in range(em.CRT_B_MIN, em.CRT_B_MAX + 1)
              if em.CRT_KAPPA * em.Z_MAX * math.ldexp(1.0, 53 - x) <= rhs)
    assert b0 <= b
    assert crt_ratio(A, B, b0 - 5, N) > em.THETA


def test_workload_parameters():
    # uniform[-1,1) * 2^e rows and columns at k = 8192: spreads near 1/4. On
    # 16 rows and columns the smallest are above 0.2437 and 37 bits do (11
    # moduli); over all 8192 rows and columns the smallest are near 0.2436,
    # which asks for 38 bits, one more than 11 moduli hold: 12 moduli, and
    # then 41 bits (12 residue products against the digit form's 15 pairs)
    A = inputs.row_scaled(16, 8192, 3)
    B = inputs.col_scaled(8192, 16, 3)
    assert em.crt_params(A, B) == (37, 11)
    assert em.crt_params_from_spread(8192, 0.2436, 0.2435) == (41, 12)
    assert not em.crt_fits(8192, 38, 11) and em.crt_fits(8192, 37, 11)


# ------------------------------------------------------------ the rule
@pytest.mark.parametrize("k", [1, 5, 64, 1000, 8192, 100000])
@pytest.mark.parametrize("spread", [0.4, 0.25, 0.05, 0.003])
def test_rule_inequalities(k, spread):
    r = em.crt_params_from_spread(k, spread, spread)
    rhs = em.THETA * 4.0 * k * math.sqrt(k) * spread * spread
    ok = lambda b: em.CRT_KAPPA * em.Z_MAX * math.ldexp(1.0, 53 - b) <= rhs
    if r is None:
        # no bit count in range qualifies, or no modulus count holds the smallest
        b0 = next((b for b in range(em.CRT_B_MIN, em.CRT_B_MAX + 1) if ok(b)), None)
        assert b0 is None or not em.crt_fits(k, b0, em.CRT_N_MAX)
        return
    b, N = r
    assert ok(b) and em.CRT_B_MIN <= b <= em.CRT_B_MAX
    assert em.crt_fits(k, b, N)
    b0 = next(x for x in range(em.CRT_B_MIN, em.CRT_B_MAX + 1) if ok(x))
    assert N == 1 or not em.crt_fits(k, b0, N - 1)                  # the fewest moduli
    assert b == em.CRT_B_MAX or not em.crt_fits(k, b + 1, N)         # the most bits they hold


def test_fits_is_the_exact_integer_comparison():
    # k 2^(2b-1) < M_N, checked against the sums' extreme |Y| = k 2^(2b-2) < M/2
    for N in range(1, em.CRT_N_MAX + 1):
        M = em.crt_modulus_product(N)
        for b in range(1, 60):
            for k in (1, 3, 1000, 8192):
                assert em.crt_fits(k, b, N) == (2 * (k << (2 * b - 2)) < M)
