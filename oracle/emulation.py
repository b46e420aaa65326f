"""CPU reference for the split-precision (emulated) products -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this module. The GPU library never calls it and shares no code with it.

The paper itself measures only the plain FP64 triple loop (Sec. III, Sec. V);
it prints no emulation scheme. The two emulated modes below restate published
methods from their mathematics:

* FP64-accuracy ("fp64_emu"): the error-free splitting of a matrix product of
  Ozaki, Ogita, Oishi and Rump (2012), in the integer-slice form of Ootomo,
  Ozaki and Yokota (2024): after a power-of-two scaling per row of A and per
  column of B, every entry becomes an integer R (the scaled value rounded to
  t*s bits), written as s signed radix-2^t digits ("slices"). Slice products
  are integer matrix products; products whose digit levels add to more than
  s+1 are dropped; the kept levels are recombined with their powers of two.
  The modular form (Ozaki, Uchino, Imamura 2025, "Ozaki scheme II") keeps the
  same scaled integers but multiplies their residues modulo N small coprime
  moduli and rebuilds the exact integer product by the Chinese remainder
  theorem (N products instead of s(s+1)/2).
* FP32-accuracy ("fp32_emu"): three bfloat16 slices per entry, each the
  round-to-nearest bfloat16 of the residual left by the slices before it, and
  the six slice products whose slice indices add to at most 2; from k = 512
  on the first two slices and the three products with indices adding to at
  most 1 (the bound is wide enough there, see FP32_TWO_SLICE_K).

Notation (row-major, A is m x k, B is k x n):
  t      digit width in bits (8 here: every digit fits in a bfloat16 exactly)
  s      number of slices
  E_i    scale exponent of row i of A; F_j of column j of B
  R      integer representation of a scaled entry
  sigma_p  slice p (p = 1 .. s), an integer with |sigma_p| <= 2^(t-1)
  L_d    level-d product sum_{p+q=d} sigma^A_p . sigma^B_q  (d = 2 .. s+1)

Readings taken where no source fixes the detail (each is listed in the design
notes):
  * E_i = floor(log2 max_k |a_ik|) + 2 for FP64-accuracy, so |a/2^E| < 1/2 and
    every balanced digit stays within [-2^(t-1), 2^(t-1)]; +1 for FP32-accuracy.
    A zero row (or column) takes E = 0 and all-zero slices.
  * R = round-half-even(a * 2^(t*s - E)); the digits are its balanced radix-2^t
    expansion, taken from the least significant digit up, with the top digit
    keeping whatever remains.
  * The emulated FP64-accuracy result is the exactly computed kept sum, rounded
    once to the nearest double.

Integer work uses numpy int64 (exact: |R| < 2^62) or Python integers.
Every function is plain and unblocked so it can be checked against the method
by eye.
"""
from __future__ import annotations

from fractions import Fraction
import math

import numpy as np

T_BITS = 8  # digit width t


# ---------------------------------------------------------------------------
# Step 1: power-of-two scale exponents (per row of A, per column of B)
# ---------------------------------------------------------------------------
def _floor_log2(x: float) -> int:
    """floor(log2 x) for a finite x > 0, exact (frexp gives x = f*2^e, f in [1/2,1))."""
    f, e = math.frexp(x)
    return e - 1


def row_exponents(A: np.ndarray, offset: int) -> np.ndarray:
    """E_i = floor(log2 max_k |a_ik|) + offset; 0 for an all-zero row.

    offset is 2 for the FP64-accuracy digits and 1 for the FP32-accuracy slices.
    """
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    E = np.zeros(m, dtype=np.int64)
    for i in range(m):
        mx = float(np.max(np.abs(A[i]))) if A.shape[1] else 0.0
        if mx > 0.0:
            E[i] = _floor_log2(mx) + offset
    return E


def col_exponents(B: np.ndarray, offset: int) -> np.ndarray:
    """F_j = floor(log2 max_k |b_kj|) + offset; 0 for an all-zero column."""
    return row_exponents(np.asarray(B, dtype=np.float64).T, offset)


def has_nonfinite(X: np.ndarray) -> bool:
    return not bool(np.all(np.isfinite(X)))


# ---------------------------------------------------------------------------
# Step 1b (FP64-accuracy): slice count from the operands' spread
# ---------------------------------------------------------------------------
# Error estimate behind the automatic slice count. With digit width 8 and
# s slices, every kept product is formed exactly; the error of output (i, j)
# comes from (a) rounding each entry to the grid 2^(E-8s) (row i of A) or
# 2^(F-8s) (column j of B) and (b) the dropped levels d >= s+2, led by level
# s+2 with its s-1 digit pairs. Taking the digits below the leading ones as
# independent and uniform on [-128, 128), one term a_ik*b_kj carries an error
# of standard deviation at most KAPPA * 2^(E_i+F_j-8s): (a) gives at most
# sqrt(2/12 * 1/4) = 0.204 (|a| < 2^(E-1)), (b) gives sqrt(s-1) * 128^2/3 *
# 2^-16 = 0.083 sqrt(s-1), and for s <= 7 the two together stay below 0.3.
# Over k terms with independent signs the error grows like sqrt(k); the
# largest of up to 2^30 outputs stays within Z = 6.5 standard deviations.
# The componentwise bound is 4k 2^-53 sum_k |a_ik||b_kj|, which for rows and
# columns spread independently of each other is about
# 4k 2^-53 * k * alpha_i * beta_j * 2^(E_i+F_j), where
#     alpha_i = mean_k |a_ik| / 2^E_i,   beta_j = mean_k |b_kj| / 2^F_j.
# So the error stays within THETA of the bound for every output when
#     KAPPA * Z * 2^(53-8s) <= THETA * 4 * k * sqrt(k) * alpha_min * beta_min.
# The slice count is the smallest s in 3..7 that passes; when none does the
# product runs through the plain FP64 kernel (returned as s = 8).
KAPPA = 0.3
Z_MAX = 6.5
THETA = 0.5
S_MIN, S_MAX, S_PLAIN = 3, 7, 8


def row_spread(A: np.ndarray, E: np.ndarray) -> np.ndarray:
    """alpha_i = (sum_k |a_ik|) / (k * 2^E_i) in fp64; +inf for a row that is all
    zero or holds Inf/NaN (such rows put no constraint on the slice count)."""
    A = np.asarray(A, dtype=np.float64)
    m, k = A.shape
    out = np.full(m, np.inf)
    for i in range(m):
        row = A[i]
        if not np.all(np.isfinite(row)):
            continue
        total = math.fsum(abs(float(x)) for x in row)
        if total > 0.0:
            out[i] = total / (k * math.ldexp(1.0, int(E[i])))
    return out


def col_spread(B: np.ndarray, F: np.ndarray) -> np.ndarray:
    """beta_j = (sum_k |b_kj|) / (k * 2^F_j), as row_spread on the columns."""
    return row_spread(np.asarray(B, dtype=np.float64).T, F)


def slice_count_from_spread(k: int, alpha_min: float, beta_min: float) -> int:
    """Smallest s in S_MIN..S_MAX with KAPPA*Z_MAX*2^(53-8s) <= THETA*4*k*sqrt(k)*alpha_min*beta_min,
    else S_PLAIN. Evaluated in double (k*sqrt(k) with a correctly rounded sqrt)."""
    rhs = THETA * 4.0 * float(k) * math.sqrt(float(k)) * float(alpha_min) * float(beta_min)
    for s in range(S_MIN, S_MAX + 1):
        if KAPPA * Z_MAX * math.ldexp(1.0, 53 - 8 * s) <= rhs:
            return s
    return S_PLAIN


def slice_count(A: np.ndarray, B: np.ndarray) -> int:
    """The automatic FP64-accuracy slice count of the product A*B (S_PLAIN:
    the plain FP64 product)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    k = A.shape[1]
    alpha = row_spread(A, row_exponents(A, 2))
    beta = col_spread(B, col_exponents(B, 2))
    amin = float(alpha.min()) if alpha.size else math.inf
    bmin = float(beta.min()) if beta.size else math.inf
    return slice_count_from_spread(k, amin, bmin)


# ---------------------------------------------------------------------------
# Step 2 (FP64-accuracy): integer representation and balanced digits
# ---------------------------------------------------------------------------
def integer_repr(A: np.ndarray, E: np.ndarray, s: int, t: int = T_BITS) -> np.ndarray:
    """R_ik = round-half-even(a_ik * 2^(t*s - E_i)) as int64 (rows scaled by E)."""
    A = np.asarray(A, dtype=np.float64)
    shift = (t * s - np.asarray(E, dtype=np.int64))[:, None]
    scaled = np.ldexp(A, shift)            # exact: a power-of-two scaling
    R = np.rint(scaled)                    # numpy rint rounds half to even
    assert np.all(np.abs(R) <= 2.0 ** (t * s - 1)), "scaled entry out of range"
    return R.astype(np.int64)


def balanced_digits(R: np.ndarray, s: int, t: int = T_BITS) -> np.ndarray:
    """Digits sigma[p-1] (p = 1..s, most significant first) with
    R = sum_p sigma_p * 2^(t*(s-p)); sigma_p in [-2^(t-1), 2^(t-1)) for p >= 2
    and |sigma_1| <= 2^(t-1)."""
    R = np.asarray(R, dtype=np.int64).copy()
    half = 1 << (t - 1)
    base = 1 << t
    sig = np.zeros((s,) + R.shape, dtype=np.int64)
    for p in range(s, 1, -1):                  # least significant digit first
        d = np.mod(R + half, base) - half      # balanced remainder
        sig[p - 1] = d
        R = (R - d) >> t                       # exact division by 2^t
    sig[0] = R
    return sig


# Exponent offset of the digit forms: 2 for digits held in bfloat16 (every
# digit in [-128, 128]); 3 for digits held in signed bytes (the INT8 form):
# with |a / 2^E| < 1/4 the top digit stays within [-64, 64] and every other
# digit within [-128, 128), so all fit in [-128, 127].
OFFSET_BF16, OFFSET_INT8 = 2, 3


def fp64_slices_A(A: np.ndarray, s: int, t: int = T_BITS, offset: int = OFFSET_BF16):
    """(E, sigma) for A: sigma has shape (s, m, k)."""
    E = row_exponents(A, offset)
    return E, balanced_digits(integer_repr(A, E, s, t), s, t)


def fp64_slices_B(B: np.ndarray, s: int, t: int = T_BITS, offset: int = OFFSET_BF16):
    """(F, sigma) for B: sigma has shape (s, k, n) (column j scaled by F_j)."""
    F = col_exponents(B, offset)
    RT = integer_repr(np.asarray(B, dtype=np.float64).T, F, s, t)   # (n, k)
    return F, np.transpose(balanced_digits(RT, s, t), (0, 2, 1))     # (s, k, n)


# ---------------------------------------------------------------------------
# Step 3 (FP64-accuracy): level products of the slices
# ---------------------------------------------------------------------------
def level_products(sigA: np.ndarray, sigB: np.ndarray, s: int) -> np.ndarray:
    """L[d-2] = sum_{p+q=d} sigma^A_p @ sigma^B_q for d = 2..s+1 (int64, exact).

    numpy's integer matmul is exact while |L| < 2^63 (here |L| <= k*s*2^14)."""
    m, n = sigA.shape[1], sigB.shape[2]
    L = np.zeros((s, m, n), dtype=np.int64)
    for d in range(2, s + 2):
        for p in range(1, d):
            q = d - p
            if p > s or q > s:
                continue
            L[d - 2] += sigA[p - 1] @ sigB[q - 1]
    return L


# ---------------------------------------------------------------------------
# Step 4 (FP64-accuracy): recombination, rounded once to double
# ---------------------------------------------------------------------------
def recombine_exact(L: np.ndarray, E: np.ndarray, F: np.ndarray, s: int,
                    t: int = T_BITS) -> np.ndarray:
    """C_ij = RN( 2^(E_i+F_j) * sum_{d=2}^{s+1} 2^(-t d) L_d[i,j] ).

    The sum is formed exactly as the integer X = sum_d 2^(t(s+1-d)) L_d (Python
    integers), then X * 2^(E_i+F_j-t(s+1)) is rounded once (Fraction -> float
    rounds to nearest-even, subnormals included)."""
    m, n = L.shape[1], L.shape[2]
    C = np.zeros((m, n), dtype=np.float64)
    for i in range(m):
        for j in range(n):
            X = 0
            for d in range(2, s + 2):
                X += int(L[d - 2, i, j]) << (t * (s + 1 - d))
            e = int(E[i]) + int(F[j]) - t * (s + 1)
            C[i, j] = float(Fraction(X) * (Fraction(2) ** e))
    return C


def gemm_fp64_emu(A: np.ndarray, B: np.ndarray, s: int, t: int = T_BITS, offset: int = OFFSET_BF16) -> np.ndarray:
    """The FP64-accuracy emulated product, steps 1-4 in order (offset 3: the
    INT8 digit form)."""
    E, sA = fp64_slices_A(A, s, t, offset)
    F, sB = fp64_slices_B(B, s, t, offset)
    L = level_products(sA, sB, s)
    return recombine_exact(L, E, F, s, t)


def slice_count_int8(A: np.ndarray, B: np.ndarray) -> int:
    """The automatic slice count of the INT8 digit form: its digit grid is twice
    as coarse relative to the row maximum, so the spreads enter the rule halved."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    alpha = row_spread(A, row_exponents(A, 2))
    beta = col_spread(B, col_exponents(B, 2))
    amin = float(alpha.min()) if alpha.size else math.inf
    bmin = float(beta.min()) if beta.size else math.inf
    return slice_count_from_spread(A.shape[1], 0.5 * amin, 0.5 * bmin)


# ---------------------------------------------------------------------------
# FP64-accuracy, modular form (Ozaki scheme II: Ozaki, Uchino, Imamura 2025)
# ---------------------------------------------------------------------------
# Instead of splitting each scaled integer into digits and multiplying digit
# pairs, the modular form takes the scaled integers' residues modulo N pairwise
# coprime moduli m_1 .. m_N, multiplies the residue matrices (one product a
# modulus), reduces each product modulo its own modulus and rebuilds the exact
# integer product by the Chinese remainder theorem. With M = m_1 ... m_N the
# rebuilt value is exact as long as every output's integer product lies in
# (-M/2, M/2). N products replace the s(s+1)/2 digit-pair products.
#
# Notation (E_i, F_j as for the digit form, floor(log2 max) + 2):
#   b        bits of the scaled integers: R = round-half-even(a * 2^(b - E_i)),
#            so |R| <= 2^(b-1) (|a| < 2^(E_i - 1))
#   rho^(l)  centred residue of R modulo m_l, in [-floor(m_l/2), ceil(m_l/2) - 1]
#   P^(l)    rho_A^(l) @ rho_B^(l), an exact integer matrix product
#   c^(l)    P^(l) mod m_l, in [0, m_l)
#   Y        the integer in [-M/2, M/2) congruent to c^(l) modulo every m_l
#   C_ij     round-to-nearest(Y_ij * 2^(E_i + F_j - 2b))
# Readings taken here: moduli no larger than 256, so every centred residue
# lies in [-128, 127] and is exact in bfloat16 (and each residue product is at
# most 2^14, as for the digit form); the moduli are the largest pairwise
# coprime integers <= 256, taken greedily from 256 down; Y in [-M/2, M/2).
CRT_MODULI = (256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199)
CRT_N_MAX = len(CRT_MODULI)
CRT_B_MIN, CRT_B_MAX = 24, 53

# The error of the modular form comes only from rounding each scaled entry to
# its integer (the products and the rebuild are exact): one term a_ik b_kj
# carries an error of standard deviation at most sqrt(2/12 * 1/4) * 2^(E_i +
# F_j - b) = 0.204 * ... for digits uniform in their rounding interval, so the
# rule of the digit form applies with this constant and 8s replaced by b.
CRT_KAPPA = 0.21


def crt_modulus_product(N: int) -> int:
    """M_N = m_1 * ... * m_N (exact integer)."""
    M = 1
    for m in CRT_MODULI[:N]:
        M *= m
    return M


def crt_fits(k: int, b: int, N: int) -> bool:
    """Whether every output of an inner dimension k product of b-bit scaled
    integers lies strictly inside (-M_N/2, M_N/2): |Y| <= k 2^(2b-2) < M_N / 2."""
    return k * (1 << (2 * b - 1)) < crt_modulus_product(N)


def crt_params_from_spread(k: int, alpha_min: float, beta_min: float):
    """(b, N) of the modular form for inner dimension k and the smallest row and
    column spreads, or None when it cannot reach the estimate's target.

    b0 = the smallest b in CRT_B_MIN..CRT_B_MAX with
         CRT_KAPPA * Z_MAX * 2^(53-b) <= THETA * 4 * k * sqrt(k) * alpha_min * beta_min
    (evaluated in double, as the digit form's rule), N = the smallest count
    whose moduli hold k-term sums of b0-bit integers, and b = the largest bit
    count (at most CRT_B_MAX) those N moduli still hold."""
    rhs = THETA * 4.0 * float(k) * math.sqrt(float(k)) * float(alpha_min) * float(beta_min)
    b0 = None
    for b in range(CRT_B_MIN, CRT_B_MAX + 1):
        if CRT_KAPPA * Z_MAX * math.ldexp(1.0, 53 - b) <= rhs:
            b0 = b
            break
    if b0 is None:
        return None
    N = next((n for n in range(1, CRT_N_MAX + 1) if crt_fits(k, b0, n)), None)
    if N is None:
        return None
    b = b0
    while b + 1 <= CRT_B_MAX and crt_fits(k, b + 1, N):
        b += 1
    return b, N


def crt_params(A: np.ndarray, B: np.ndarray):
    """(b, N) of the product A*B from its operands' spreads (None: no fit)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    alpha = row_spread(A, row_exponents(A, 2))
    beta = col_spread(B, col_exponents(B, 2))
    amin = float(alpha.min()) if alpha.size else math.inf
    bmin = float(beta.min()) if beta.size else math.inf
    return crt_params_from_spread(A.shape[1], amin, bmin)


def fp64_scheme(A: np.ndarray, B: np.ndarray, modular: bool = True):
    """The automatic FP64-accuracy decision for A*B: ("crt", b, N) when the
    modular form fits (and is allowed), else ("digits", s) for a digit count
    s <= S_MAX, else ("plain",)."""
    if modular:
        bN = crt_params(A, B)
        if bN is not None:
            return ("crt",) + tuple(bN)
    s = slice_count(A, B)
    return ("digits", s) if s <= S_MAX else ("plain",)


def crt_integer_repr(X: np.ndarray, E: np.ndarray, b: int) -> np.ndarray:
    """R = round-half-even(x * 2^(b - E)) per row of X, as int64 (|R| <= 2^(b-1) <= 2^52)."""
    X = np.asarray(X, dtype=np.float64)
    R = np.rint(np.ldexp(X, (b - np.asarray(E, dtype=np.int64))[:, None]))
    assert np.all(np.abs(R) <= 2.0 ** (b - 1)), "scaled entry out of range"
    return R.astype(np.int64)


def crt_residues(R: np.ndarray, N: int) -> np.ndarray:
    """rho[l] = R mod m_l, centred into [-floor(m/2), ceil(m/2) - 1]; shape (N,) + R.shape."""
    R = np.asarray(R, dtype=np.int64)
    out = np.zeros((N,) + R.shape, dtype=np.int64)
    for l, m in enumerate(CRT_MODULI[:N]):
        h = m // 2
        out[l] = np.mod(R + h, m) - h
    return out


def crt_products(rhoA: np.ndarray, rhoB: np.ndarray) -> np.ndarray:
    """P[l] = rhoA[l] @ rhoB[l], exact in int64 (|P| <= k 2^14)."""
    return np.stack([rhoA[l] @ rhoB[l] for l in range(rhoA.shape[0])])


def crt_reconstruct(P: np.ndarray) -> np.ndarray:
    """Y: the integer in [-M/2, M/2) with Y = P[l] (mod m_l) for every l, from
    the textbook CRT sum X = sum_l c_l * W_l mod M, W_l = (M/m_l) * ((M/m_l)^-1
    mod m_l). Python integers (object array)."""
    N = P.shape[0]
    M = crt_modulus_product(N)
    W = []
    for m in CRT_MODULI[:N]:
        Ml = M // m
        W.append(Ml * pow(Ml % m, -1, m))
    Y = np.empty(P.shape[1:], dtype=object)
    for idx in np.ndindex(*P.shape[1:]):
        X = sum((int(P[(l,) + idx]) % CRT_MODULI[l]) * W[l] for l in range(N)) % M
        Y[idx] = X if 2 * X < M else X - M
    return Y


def crt_round(Y: np.ndarray, E: np.ndarray, F: np.ndarray, b: int) -> np.ndarray:
    """C_ij = round-to-nearest(Y_ij * 2^(E_i + F_j - 2b)) (Fraction -> float)."""
    m, n = Y.shape
    C = np.zeros((m, n), dtype=np.float64)
    for i in range(m):
        for j in range(n):
            C[i, j] = float(Fraction(int(Y[i, j])) * (Fraction(2) ** (int(E[i]) + int(F[j]) - 2 * b)))
    return C


def gemm_fp64_crt(A: np.ndarray, B: np.ndarray, b: int, N: int) -> np.ndarray:
    """The FP64-accuracy product in the modular form with b-bit scaled integers
    and N moduli (k 2^(2b-1) < M_N), the steps above in order."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    assert crt_fits(A.shape[1], b, N), "moduli too few for this b and k"
    E = row_exponents(A, 2)
    F = col_exponents(B, 2)
    RA = crt_integer_repr(A, E, b)                    # (m, k)
    RB = crt_integer_repr(B.T, F, b).T                # (k, n), column j scaled by F_j
    P = crt_products(crt_residues(RA, N), crt_residues(RB, N))
    return crt_round(crt_reconstruct(P), E, F, b)


# ---------------------------------------------------------------------------
# FP32-accuracy: three bfloat16 slices
# ---------------------------------------------------------------------------
def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round doubles to the nearest bfloat16 value (ties to even), returned as
    doubles. bfloat16 keeps 8 significant bits and float32's exponent range;
    below 2^-126 its spacing is the subnormal step 2^-133."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0.0
    _, e = np.frexp(x[nz])                       # |x| in [2^(e-1), 2^e)
    ulp_exp = np.maximum(e - 8, -133)            # spacing of bfloat16 there
    out[nz] = np.ldexp(np.rint(np.ldexp(x[nz], -ulp_exp)), ulp_exp)
    return out


def fp32_slices(R: np.ndarray):
    """a0 = bf16(r), a1 = bf16(r - a0), a2 = bf16(r - a0 - a1); the residuals
    are exact in double (each slice is within a factor two of its residual)."""
    a0 = bf16_round(R)
    r1 = R - a0
    a1 = bf16_round(r1)
    r2 = r1 - a1
    a2 = bf16_round(r2)
    return np.stack([a0, a1, a2])


def fp32_slices_A(A: np.ndarray):
    E = row_exponents(A, 1)
    r = np.ldexp(np.asarray(A, dtype=np.float64), -E[:, None])
    return E, fp32_slices(r)


def fp32_slices_B(B: np.ndarray):
    F = col_exponents(B, 1)
    r = np.ldexp(np.asarray(B, dtype=np.float64), -F[None, :])
    return F, fp32_slices(r)


FP32_PAIRS = [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]

# Two slices suffice once the bound is wide enough. Rounding to the nearest
# bfloat16 keeps 8 significant bits, so |a - a0| <= 2^-8 |a| and
# |a - a0 - a1| <= 2^-16 |a|. Writing a = a0 + a1 + da and b likewise, the
# products left out beside (0,0), (0,1), (1,0) are a1 b1, a0 db, da b0 and
# smaller terms, together at most 3.03 * 2^-16 |a b| for every term of the
# sum, whatever the signs. That is at most half of 4k 2^-24 |A||B| when
# k >= 3.03 * 2^8 / 2 = 388; from k = 512 on (0.38 of the bound) the product
# takes two slices a operand and the three pairs with p + q <= 1.
FP32_TWO_SLICE_K = 512
FP32_PAIRS_TWO = [(0, 0), (0, 1), (1, 0)]


def fp32_pairs(k: int):
    """The slice pairs of the FP32-accuracy product of inner dimension k."""
    return FP32_PAIRS_TWO if k >= FP32_TWO_SLICE_K else FP32_PAIRS


def gemm_fp32_emu(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """sum over the slice pairs of fp32_pairs(k) (the six with p+q <= 2, or
    from k = 512 the three with p+q <= 1) of slice products, scaled back.

    Products of bfloat16 values are exact in double; the k-sums here are in
    double, so this is the FP32-accuracy value without the float32 rounding the
    tensor cores add."""
    E, sA = fp32_slices_A(A)
    F, sB = fp32_slices_B(B)
    acc = np.zeros((sA.shape[1], sB.shape[2]))
    for p, q in fp32_pairs(np.asarray(A).shape[1]):
        acc += sA[p] @ sB[q]
    return np.ldexp(np.ldexp(acc, E[:, None]), F[None, :])


# ---------------------------------------------------------------------------
# Acceptance bound (componentwise)
# ---------------------------------------------------------------------------
def gamma(k: int, mode: str) -> float:
    """gamma = 4k*2^-53 for FP64-accuracy modes, 4k*2^-24 for FP32-accuracy."""
    u = 2.0 ** -53 if mode in ("fp64", "fp64_emu") else 2.0 ** -24
    return 4.0 * max(k, 1) * u
