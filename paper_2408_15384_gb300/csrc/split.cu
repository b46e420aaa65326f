// split.cu -- exponent scan and operand splitting for the emulated modes, and
// the seeded input filler.
//
// GB300's FP64 pipe is narrow, so every step here works on the IEEE-754 bit
// patterns with integer instructions: the row/column maxima are maxima of the
// magnitude bits (order-preserving for non-negative doubles), the scale
// exponent is read from the exponent field, and the slices are produced by
// integer rounding of the significand.
//
// FP64-accuracy splitting (Ozaki, Ogita, Oishi, Rump 2012; integer-slice form
// of Ootomo, Ozaki, Yokota 2024), digit width t = 8:
//   E_i = floor(log2 max_k |a_ik|) + 2      (0 for a zero row)
//   R   = round-half-even(a * 2^(t*s - E_i))          |R| <= 2^(t*s-1)
//   R   = sum_p sigma_p 2^(t(s-p)), balanced digits taken from the least
//         significant up: sigma in [-2^(t-1), 2^(t-1)), the top digit keeps
//         the rest (|sigma_1| <= 2^(t-1)).
// FP32-accuracy splitting: E_i = floor(log2 max|a|) + 1, r = a*2^-E_i,
//   a0 = bf16_rn(r), a1 = bf16_rn(r - a0), a2 = bf16_rn(r - a0 - a1); the
//   residuals are exact (kept as integers scaled by 2^e).
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "ptx.cuh"

namespace mmdev {

static constexpr uint64_t ABS_MASK = 0x7FFFFFFFFFFFFFFFull;
static constexpr uint64_t INF_BITS = 0x7FF0000000000000ull;

__device__ __forceinline__ uint64_t dbits(double x) { return static_cast<uint64_t>(__double_as_longlong(x)); }

// floor(log2 |x|) for finite nonzero magnitude bits.
__device__ __forceinline__ int floor_log2_bits(uint64_t ab) {
  int ex = static_cast<int>(ab >> 52);
  if (ex) return ex - 1023;
  return (63 - __clzll(static_cast<long long>(ab))) - 1074;
}

// Scale exponent from a magnitude maximum: offset + floor(log2 max), 0 for a
// zero maximum, EXP_NONFINITE for Inf/NaN.
__device__ __forceinline__ int32_t exponent_from_max(uint64_t mx, int offset) {
  if (mx == 0) return 0;
  if (mx >= INF_BITS) return EXP_NONFINITE;
  return floor_log2_bits(mx) + offset;
}

// Split |x| into an integer significand and exponent: |x| = mant * 2^e.
__device__ __forceinline__ void decompose(uint64_t ab, uint64_t& mant, int& e) {
  int ex = static_cast<int>(ab >> 52);
  mant = ab & 0xFFFFFFFFFFFFFull;
  if (ex) {
    mant |= (1ull << 52);
    e = ex - 1075;
  } else {
    e = -1074;
  }
}

// round-half-even(x * 2^sh) for x given by its bits; caller guarantees the
// result magnitude is below 2^62.
__device__ __forceinline__ int64_t scaled_rne(uint64_t bits, int sh) {
  uint64_t ab = bits & ABS_MASK;
  if (ab == 0) return 0;
  uint64_t mant;
  int e;
  decompose(ab, mant, e);
  int total = e + sh;
  uint64_t q;
  if (total >= 0) {
    q = mant << total;
  } else {
    int rs = -total;
    if (rs >= 64) {
      q = 0;
    } else {
      q = mant >> rs;
      uint64_t rem = mant & ((1ull << rs) - 1ull);
      uint64_t half = 1ull << (rs - 1);
      if (rem > half || (rem == half && (q & 1ull))) ++q;
    }
  }
  int64_t r = static_cast<int64_t>(q);
  return (bits >> 63) ? -r : r;
}

// bfloat16 bit pattern of a small integer (|d| < 2^22, at most 8 significant
// bits): the float built by adding d to the pattern of 1.5*2^23 and
// subtracting 1.5*2^23 is exact, and its upper half is the bfloat16.
__device__ __forceinline__ uint16_t bf16_of_small_int(int32_t d) {
  float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return static_cast<uint16_t>(__float_as_uint(f) >> 16);
}

// Round the value M * 2^e (M signed) to the nearest bfloat16 (ties to even,
// bfloat16 subnormals below 2^-126 with step 2^-133); subtract the rounded
// value from M (exact) and return its bit pattern.
__device__ __forceinline__ uint16_t bf16_rne_take(int64_t& M, int e) {
  if (M == 0) return 0;
  uint32_t sgn = M < 0 ? 0x8000u : 0u;
  uint64_t a = M < 0 ? static_cast<uint64_t>(-M) : static_cast<uint64_t>(M);
  int nb = 64 - __clzll(static_cast<long long>(a));
  int sh = nb - 8;
  if (e + sh < -133) sh = -133 - e;
  uint64_t q;
  int L;
  if (sh <= 0) {
    q = a;
    L = e;
    M = 0;
  } else {
    if (sh >= 64) {
      q = 0;
    } else {
      // round half to even: add half - 1, plus one more when the kept part is odd
      q = (a + ((1ull << (sh - 1)) - 1ull) + ((a >> sh) & 1ull)) >> sh;
    }
    L = e + sh;
    uint64_t taken = (sh >= 64) ? 0ull : (q << sh);
    M = (M < 0) ? (M + static_cast<int64_t>(taken)) : (M - static_cast<int64_t>(taken));
  }
  if (q == 0) return static_cast<uint16_t>(sgn);
  if (q == 256) {
    q = 128;
    ++L;
  }
  // normalise q into [128, 256) unless that would pass below 2^-133
  if (q < 128) {
    int up = __clz(static_cast<uint32_t>(q)) - 24;   // shifts that bring the top bit to bit 7
    if (L - up < -133) up = L + 133;
    q <<= up;
    L -= up;
  }
  if (q < 128) return static_cast<uint16_t>(sgn | q);  // subnormal bfloat16, L == -133
  int biased = L + 7 + 127;
  return static_cast<uint16_t>(sgn | (static_cast<uint32_t>(biased) << 7) | static_cast<uint32_t>(q - 128));
}

// The first S (2 or 3) FP32-accuracy slices of one entry (the third is not
// formed for two slices).
template <int S>
__device__ __forceinline__ void fp32_slices(uint64_t bits, int E, uint32_t& s0, uint32_t& s1, uint32_t& s2) {
  uint64_t ab = bits & ABS_MASK;
  s2 = 0u;
  if (ab == 0) {
    s0 = s1 = 0u;
    return;
  }
  uint64_t mant;
  int e;
  decompose(ab, mant, e);
  e -= E;
  const bool neg = (bits >> 63) != 0;
  int64_t M;
  // the first slice of a normal entry rounds at a fixed bit (45 of the 53-bit
  // significand): round half to even, the residual kept exact
  if ((mant >> 52) != 0 && e + 45 >= -126) {
    const uint64_t q = (mant + ((1ull << 44) - 1ull) + ((mant >> 45) & 1ull)) >> 45;   // 128 .. 256
    const int64_t rest = static_cast<int64_t>(mant) - static_cast<int64_t>(q << 45);
    M = neg ? -rest : rest;
    const int L = e + 45 + (q == 256 ? 1 : 0);
    const uint32_t q8 = (q == 256) ? 128u : static_cast<uint32_t>(q);
    s0 = (neg ? 0x8000u : 0u) | (static_cast<uint32_t>(L + 7 + 127) << 7) | (q8 - 128u);
  } else {
    M = neg ? -static_cast<int64_t>(mant) : static_cast<int64_t>(mant);
    s0 = bf16_rne_take(M, e);
  }
  s1 = bf16_rne_take(M, e);
  if (S >= 3) s2 = bf16_rne_take(M, e);
}

// Slice modes: 0 FP64-accuracy digits as bfloat16, 1 FP32-accuracy bfloat16
// slices, 2 FP64-accuracy digits as signed bytes (the INT8 form: one more
// bit of headroom in the scale exponent keeps every digit within [-128, 127]).
template <int MODE>
struct SliceElem {
  using T = uint16_t;
};
template <>
struct SliceElem<2> {
  using T = int8_t;
};
__host__ __device__ constexpr int exp_offset(int mode) { return mode == 1 ? 1 : (mode == 2 ? 3 : 2); }

// The slices of 8 consecutive entries (bit patterns vb, scale exponent X of
// their row or column), stored to dst + P * plane for P = 0 .. S-1 (plane 0
// the most significant): one 16-byte vector per plane when the run is whole
// and aligned, else element by element. Everything stays in registers.
//
// FP64-accuracy digits from the biased integer Rb = R + B,
// B = sum_{j=0}^{s-2} 128 * 256^j: digit j (least significant first) is
// ((Rb >> 8j) & 255) - 128 for j < s-1 and the top digit is Rb >> 8(s-1)
// (arithmetic shift), the same digits the one-at-a-time expansion
// d = ((R + 128) mod 256) - 128, R = (R - d) / 256 produces.
template <int MODE>
__device__ __forceinline__ void slice8_store(const uint64_t (&vb)[8], int32_t X, int s,
                                             typename SliceElem<MODE>::T* __restrict__ dst, size_t plane, int cnt) {
  const bool vec = (cnt == 8) && ((reinterpret_cast<uintptr_t>(dst) & (MODE == 2 ? 7u : 15u)) == 0);
  if constexpr (MODE == 2) {
    int64_t bias = 0;
    for (int j = 0; j < s - 1; ++j) bias = (bias << 8) | 128;
    int64_t Rb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) Rb[u] = scaled_rne(vb[u], 8 * s - X) + bias;
#pragma unroll
    for (int P = 0; P < 7; ++P) {
      if (P >= s) break;
      const int sh = 8 * (s - 1 - P);
      uint32_t lo = 0u, hi = 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int32_t d = (P == 0) ? static_cast<int32_t>(Rb[u] >> sh)
                                   : static_cast<int32_t>((Rb[u] >> sh) & 255) - 128;
        const uint32_t byte = static_cast<uint32_t>(d) & 255u;
        if (u < 4) lo |= byte << (8 * u); else hi |= byte << (8 * (u - 4));
      }
      int8_t* o = dst + P * plane;
      if (vec) {
        *reinterpret_cast<uint2*>(o) = make_uint2(lo, hi);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < cnt) o[u] = static_cast<int8_t>(((u < 4 ? lo : hi) >> (8 * (u & 3))) & 255u);
      }
    }
  } else if constexpr (MODE == 0) {
    int64_t bias = 0;
    for (int j = 0; j < s - 1; ++j) bias = (bias << 8) | 128;
    int64_t Rb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) Rb[u] = scaled_rne(vb[u], 8 * s - X) + bias;
#pragma unroll
    for (int P = 0; P < 7; ++P) {
      if (P >= s) break;
      const int sh = 8 * (s - 1 - P);
      uint32_t h[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int32_t d = (P == 0) ? static_cast<int32_t>(Rb[u] >> sh)
                                   : static_cast<int32_t>((Rb[u] >> sh) & 255) - 128;
        h[u] = bf16_of_small_int(d);
      }
      uint16_t* o = dst + P * plane;
      if (vec) {
        *reinterpret_cast<uint4*>(o) =
            make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < cnt) o[u] = static_cast<uint16_t>(h[u]);
      }
    }
  } else {
    uint32_t h[3][8];
    if (s >= 3) {
#pragma unroll
      for (int u = 0; u < 8; ++u) fp32_slices<3>(vb[u], X, h[0][u], h[1][u], h[2][u]);
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) fp32_slices<2>(vb[u], X, h[0][u], h[1][u], h[2][u]);
    }
#pragma unroll
    for (int P = 0; P < 3; ++P) {
      if (P >= s) break;   // two slices: the third is not stored
      uint16_t* o = dst + P * plane;
      if (vec) {
        *reinterpret_cast<uint4*>(o) = make_uint4(h[P][0] | (h[P][1] << 16), h[P][2] | (h[P][3] << 16),
                                                  h[P][4] | (h[P][5] << 16), h[P][6] | (h[P][7] << 16));
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < cnt) o[u] = static_cast<uint16_t>(h[P][u]);
      }
    }
  }
}

// The modular form's residues of 8 consecutive entries: R = round-half-even(
// x 2^(b - X)), |R| <= 2^(b-1) <= 2^52, and for every modulus m_l (l < N) the
// centred residue rho = ((R + h) mod m) - h, h = floor(m/2), as bfloat16 in
// plane l. With the biased u = R + 2^55 = u2 2^40 + u1 2^20 + u0 (pieces below
// 2^20, u < 2^56), (R + h) mod m is the remainder of
//   v = u2 (2^40 mod m) + u1 (2^20 mod m) + u0 + ((h - 2^55) mod m) < 2^29,
// whose quotient is floor(v * M / 2^39) with M = floor(2^39 / m) + 1 < 2^32
// (m > 128): v M / 2^39 exceeds v / m by less than v / 2^39 < 2^-10 < 1/m, so
// the floor is exact. Modulus 256 divides 2^55: its residue is u's low byte.
__host__ __device__ constexpr uint32_t pow2_mod(int e, uint32_t m) {
  uint32_t r = 1u % m;
  for (int i = 0; i < e; ++i) r = (2u * r) % m;
  return r;
}

// R + 2^55 for R = round-half-even(x 2^sh), |R| <= 2^52 (the caller's scaling
// guarantees it): normal entries shift their significand right by at least
// one place and round half to even; zero and subnormal entries take the
// general path.
__device__ __forceinline__ uint64_t biased_rne(uint64_t bits, int sh) {
  const uint32_t ex = static_cast<uint32_t>(bits >> 52) & 0x7FFu;
  if (ex == 0u) return static_cast<uint64_t>(scaled_rne(bits, sh) + (1ll << 55));
  const uint64_t mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int rs = 1075 - static_cast<int>(ex) - sh;   // >= 1: |x| 2^sh < 2^52
  uint64_t q = 0;
  if (rs < 64) q = (mant + ((1ull << (rs - 1)) - 1ull) + ((mant >> rs) & 1ull)) >> rs;
  return (bits >> 63) ? (1ull << 55) - q : (1ull << 55) + q;
}

template <int L>
__device__ __forceinline__ void crt_plane(const uint32_t (&u0)[8], const uint32_t (&u1)[8], const uint32_t (&u2)[8],
                                          uint16_t* __restrict__ o, bool vec, int cnt) {
  constexpr uint32_t m = static_cast<uint32_t>(crt_modulus(L));
  constexpr uint32_t h = m / 2u;
  uint32_t f[8];   // float bit patterns of the residues (exact small integers)
  if constexpr (m == 256u) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
      f[u] = __float_as_uint(__int_as_float(static_cast<int32_t>(0x4B400000u + ((u0[u] & 255u) ^ 128u) - 128u)) -
                             12582912.0f);
  } else {
    constexpr uint32_t c1 = pow2_mod(20, m), c2 = pow2_mod(40, m);
    constexpr uint32_t cb = (h + m - pow2_mod(55, m)) % m;
    constexpr uint32_t M = static_cast<uint32_t>((1ull << 39) / m + 1ull);
    static_assert(m > 128u, "the quotient step needs m > 128");
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const uint32_t v = u2[u] * c2 + u1[u] * c1 + (u0[u] + cb);
      const uint32_t q = __umulhi(v, M) >> 7;
      // rho = v - q m - h, placed in the float 1.5 * 2^23 + rho and read back exactly
      const uint32_t r = (v + (0x4B400000u - h)) - q * m;
      f[u] = __float_as_uint(__uint_as_float(r) - 12582912.0f);
    }
  }
  // bfloat16 = upper half of each float
  const uint4 w = make_uint4(__byte_perm(f[0], f[1], 0x7632), __byte_perm(f[2], f[3], 0x7632),
                             __byte_perm(f[4], f[5], 0x7632), __byte_perm(f[6], f[7], 0x7632));
  if (vec) {
    *reinterpret_cast<uint4*>(o) = w;
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (u < cnt) o[u] = static_cast<uint16_t>(f[u] >> 16);
  }
}

template <int... Ls>
__device__ __forceinline__ void crt_planes(std::integer_sequence<int, Ls...>, int N, const uint32_t (&u0)[8],
                                           const uint32_t (&u1)[8], const uint32_t (&u2)[8],
                                           uint16_t* __restrict__ dst, size_t plane, bool vec, int cnt) {
  ((Ls < N ? crt_plane<Ls>(u0, u1, u2, dst + Ls * plane, vec, cnt) : void()), ...);
}

__device__ __forceinline__ void slice8_crt_store(const uint64_t (&vb)[8], int32_t X, int N, int b,
                                                 uint16_t* __restrict__ dst, size_t plane, int cnt) {
  const bool vec = (cnt == 8) && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0);
  uint32_t u0[8], u1[8], u2[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const uint64_t ub = biased_rne(vb[u], b - X);
    u0[u] = static_cast<uint32_t>(ub) & 0xFFFFFu;
    u1[u] = static_cast<uint32_t>(ub >> 20) & 0xFFFFFu;
    u2[u] = static_cast<uint32_t>(ub >> 40);
  }
  crt_planes(std::make_integer_sequence<int, CRT_N_MAX>{}, N, u0, u1, u2, dst, plane, vec, cnt);
}

// Mode 3: the FP64-accuracy form the decision names -- the modular form's
// residues (code SLICE_CRT_BASE + N, bits b) or digits (code s <= 7); nothing
// for the plain fallback.
__device__ __forceinline__ void slice8_auto_store(const uint64_t (&vb)[8], int32_t X, int code, int bits,
                                                  uint16_t* __restrict__ dst, size_t plane, int cnt) {
  if (code > SLICE_CRT_BASE)
    slice8_crt_store(vb, X, code - SLICE_CRT_BASE, bits, dst, plane, cnt);
  else if (code <= SLICE_S_MAX)
    slice8_store<0>(vb, X, code, dst, plane, cnt);
}

// ------------------------------------------------------ spread statistic
// 2^x as a float for x <= 127 (0 below the normal range).
__device__ __forceinline__ float pow2f(int x) {
  return x >= -126 ? __uint_as_float(static_cast<uint32_t>(x + 127) << 23) : 0.0f;
}

// Running sum of |x| / 2^(ref - 1023) in float, ref the largest biased
// exponent seen so far (subnormals count at exponent 1). A larger exponent
// first rescales the sum by a power of two (exact); each term keeps the top 23
// bits of its significand (truncated), entries more than 2^126 below the
// reference add nothing. With SPREAD = false everything compiles away.
struct SpreadAcc {
  int ref = 1;
  float sum = 0.0f;
};

template <bool SPREAD>
__device__ __forceinline__ void spread_add(SpreadAcc& a, uint64_t ab) {
  if constexpr (SPREAD) {
    const int e = static_cast<int>(ab >> 52);
    const int ee = e > 1 ? e : 1;
    if (ee > a.ref) {
      a.sum *= pow2f(a.ref - ee);
      a.ref = ee;
    }
    float f;
    if (e != 0) {
      const int x = e - a.ref;
      f = x >= -126 ? __uint_as_float((static_cast<uint32_t>(x + 127) << 23) |
                                      static_cast<uint32_t>((ab >> 29) & 0x7FFFFFull))
                    : 0.0f;
    } else {
      // |x| = mant 2^-1074 = mant 2^(-51 - ref) in units of 2^(ref - 1023)
      f = __ull2float_rn(static_cast<unsigned long long>(ab)) * pow2f(-51 - a.ref);
    }
    a.sum += f;
  }
}

__device__ __forceinline__ SpreadAcc spread_merge(const SpreadAcc& a, const SpreadAcc& b) {
  SpreadAcc r;
  r.ref = max(a.ref, b.ref);
  r.sum = a.sum * pow2f(a.ref - r.ref) + b.sum * pow2f(b.ref - r.ref);
  return r;
}

// alpha = (sum |x|) / (k 2^E) with E = floor(log2 max) + 2, from a sum whose
// reference is the maximum's exponent; +inf (no constraint on the slice count)
// for an all-zero or non-finite row or column.
__device__ __forceinline__ float spread_final(const SpreadAcc& a, uint64_t mx, int64_t k) {
  if (mx == 0 || mx >= INF_BITS) return __uint_as_float(0x7F800000u);
  return a.sum * pow2f(a.ref - 1023 - (floor_log2_bits(mx) + 2)) / static_cast<float>(k);
}

// A warp's row spread (every lane holds it), merged into the decision word
// *dst as its distance below +inf by lane 0 (no block barrier: the minimum
// does not depend on the order).
__device__ __forceinline__ void warp_min_to(float v, uint32_t* dst) {
  if ((threadIdx.x & 31u) == 0 && v < __uint_as_float(0x7F800000u))
    atomicMax(dst, 0x7F800000u - __float_as_uint(v));
}

// Minimum over the block's threads of v (non-negative), merged into the
// decision word *dst as its distance below +inf (atomicMax). Every thread of
// the block calls it.
__device__ __forceinline__ void block_min_to(float v, uint32_t* dst) {
  __shared__ float wmin[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = static_cast<int>(threadIdx.x >> 5), nw = static_cast<int>((blockDim.x + 31) >> 5);
  if ((threadIdx.x & 31u) == 0) wmin[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = wmin[0];
    for (int i = 1; i < nw; ++i) m = fminf(m, wmin[i]);
    if (m < __uint_as_float(0x7F800000u)) atomicMax(dst, 0x7F800000u - __float_as_uint(m));
  }
  __syncthreads();
}

// ---------------------------------------------------------- kernel bodies
// Row maximum of |a| bits for one row by one warp (16-byte loads when the row
// start is 16-byte aligned). With SPREAD, returns the row's alpha (every lane),
// else +inf.
template <bool SPREAD>
__device__ __forceinline__ float row_absmax_body(const double* __restrict__ A, int64_t k, int64_t lda, int64_t row,
                                                 uint64_t* __restrict__ rowmax) {
  const double* a = A + row * lda;
  uint64_t mx = 0;
  SpreadAcc acc;
  const uint32_t lane = threadIdx.x & 31u;
  int64_t c0 = 0;
  if ((reinterpret_cast<uintptr_t>(a) & 15u) == 0) {
    const double2* a2 = reinterpret_cast<const double2*>(a);
    const int64_t k2 = k >> 1;   // whole pairs
    int64_t c = lane;
    for (; c + 96 < k2; c += 128) {
      const double2 v0 = __ldg(a2 + c), v1 = __ldg(a2 + c + 32), v2 = __ldg(a2 + c + 64), v3 = __ldg(a2 + c + 96);
      const uint64_t b[8] = {dbits(v0.x) & ABS_MASK, dbits(v0.y) & ABS_MASK, dbits(v1.x) & ABS_MASK,
                             dbits(v1.y) & ABS_MASK, dbits(v2.x) & ABS_MASK, dbits(v2.y) & ABS_MASK,
                             dbits(v3.x) & ABS_MASK, dbits(v3.y) & ABS_MASK};
      mx = max(mx, max(max(max(b[0], b[1]), max(b[2], b[3])), max(max(b[4], b[5]), max(b[6], b[7]))));
#pragma unroll
      for (int u = 0; u < 8; ++u) spread_add<SPREAD>(acc, b[u]);
    }
    for (; c < k2; c += 32) {
      const double2 v = __ldg(a2 + c);
      const uint64_t b0 = dbits(v.x) & ABS_MASK, b1 = dbits(v.y) & ABS_MASK;
      mx = max(mx, max(b0, b1));
      spread_add<SPREAD>(acc, b0);
      spread_add<SPREAD>(acc, b1);
    }
    c0 = 2 * k2;   // an odd last entry is left for the scalar loop
  }
  for (int64_t c = c0 + lane; c < k; c += 32) {
    const uint64_t b = dbits(__ldg(a + c)) & ABS_MASK;
    mx = max(mx, b);
    spread_add<SPREAD>(acc, b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, static_cast<uint64_t>(__shfl_xor_sync(0xffffffffu, static_cast<unsigned long long>(mx), o)));
    if constexpr (SPREAD) {
      SpreadAcc other;
      other.ref = __shfl_xor_sync(0xffffffffu, acc.ref, o);
      other.sum = __shfl_xor_sync(0xffffffffu, acc.sum, o);
      acc = spread_merge(acc, other);
    }
  }
  if (lane == 0) rowmax[row] = mx;
  if constexpr (SPREAD) return spread_final(acc, mx, k);
  return __uint_as_float(0x7F800000u);
}

// Column maximum of |b| bits for column j over rows [r0, r1), merged with
// atomicMax; with part != nullptr also the column's partial spread sum over
// these rows, stored as (reference exponent, float bits) at *part. The sum is
// formed in the grouped kernel's order: eight running sums, one per row
// residue mod 8 (r0 is a multiple of 8), each in row order, merged in residue
// order, so single and grouped products decide the same slice count.
template <bool SPREAD>
__device__ __forceinline__ void col_absmax_body(const double* __restrict__ B, int64_t ldb, int64_t j, int64_t r0,
                                                int64_t r1, unsigned long long* __restrict__ colmax,
                                                uint2* __restrict__ part) {
  uint64_t mx = 0;
  SpreadAcc acc[8];
  int64_t r = r0;
  for (; r + 7 < r1; r += 8) {
    uint64_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = dbits(__ldg(B + (r + u) * ldb + j)) & ABS_MASK;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      mx = max(mx, v[u]);
      spread_add<SPREAD>(acc[u], v[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 7; ++u) {
    if (r + u < r1) {
      const uint64_t v = dbits(__ldg(B + (r + u) * ldb + j)) & ABS_MASK;
      mx = max(mx, v);
      spread_add<SPREAD>(acc[u], v);
    }
  }
  if (mx) atomicMax(colmax + j, static_cast<unsigned long long>(mx));
  if constexpr (SPREAD) {
    SpreadAcc t;
#pragma unroll
    for (int u = 0; u < 8; ++u) t = spread_merge(t, acc[u]);
    *part = make_uint2(static_cast<uint32_t>(t.ref), __float_as_uint(t.sum));
  }
}

// beta of column j from its final maximum and its partial sums (parts records
// of stride n, summed in order).
__device__ __forceinline__ float col_spread_body(const uint64_t* __restrict__ colmax, const uint2* __restrict__ part,
                                                 int64_t n, int64_t k, int64_t parts, int64_t j) {
  const uint64_t mx = colmax[j];
  SpreadAcc acc;
  if (mx != 0 && mx < INF_BITS) {
    acc.ref = max(static_cast<int>(mx >> 52), 1);
    for (int64_t p = 0; p < parts; ++p) {
      const uint2 r = part[p * n + j];
      acc.sum += __uint_as_float(r.y) * pow2f(static_cast<int>(r.x) - acc.ref);
    }
  }
  return spread_final(acc, mx, k);
}

// The slice count a splitting kernel uses: the automatic rule's when dec is
// set (the block's thread 0 evaluates it, in double, and shares it; the thread
// with first set also records it), else s. scale 1/2: the INT8 form, whose
// digit grid is twice as coarse. Every thread of the block calls it.
__device__ __forceinline__ int decided_slices(SliceDecision* dec, int s, int64_t k, bool first, float scale = 1.0f) {
  if (dec == nullptr) return s;
  __shared__ int shared_s;
  __syncthreads();   // an earlier call's value has been read by every thread
  if (threadIdx.x == 0) {
    shared_s = slice_count_rule(k, scale * spread_from_room(dec->amin_room), scale * spread_from_room(dec->bmin_room));
    if (first) dec->s = shared_s;
  }
  __syncthreads();
  return shared_s;
}

// Mode 3 (automatic FP64-accuracy with the modular form allowed): the decision
// code and bit count decide_fp64_kernel recorded (uniform loads).
__device__ __forceinline__ int decided_fp64(const SliceDecision* dec, int* bits) {
  *bits = dec->bits;
  return dec->s;
}

// One thread: the automatic FP64-accuracy decision of a product from the
// scan's spreads, with the modular form allowed (fp64_decision).
__global__ void decide_fp64_kernel(SliceDecision* dec, int64_t k) {
  if (threadIdx.x != 0) return;
  int b = 0;
  const int code = fp64_decision(k, spread_from_room(dec->amin_room), spread_from_room(dec->bmin_room), true, &b);
  dec->s = code;
  dec->bits = b;
}

// Slices of 8 consecutive entries A[row][c0 .. c0+8) (rows scaled by E).
template <int MODE>  // see SliceElem
__device__ __forceinline__ void slice_rows_body(const double* __restrict__ A, int64_t plane_rows, int64_t k,
                                                int64_t lda, const uint64_t* __restrict__ rowmax, int s, int64_t kp,
                                                typename SliceElem<MODE>::T* __restrict__ slices,
                                                int32_t* __restrict__ E,
                                                uint32_t* __restrict__ err, int64_t row, int64_t c0,
                                                int bits = 0) {
  const uint64_t mx = rowmax[row];
  const int32_t Ei = exponent_from_max(mx, exp_offset(MODE));
  if (c0 == 0) {
    E[row] = Ei;
    if (Ei == EXP_NONFINITE) atomicOr(err, MM_DEV_ERR_NONFINITE);
  }
  if (MODE != 1 && MODE != 3 && s > SLICE_S_MAX) return;   // the product runs through the plain FP64 kernel
  if (MODE == 3 && s > SLICE_S_MAX && s <= SLICE_CRT_BASE) return;
  const double* a = A + row * lda + c0;
  uint64_t vb[8];
  const int cnt = static_cast<int>((k - c0) < 8 ? (k - c0) : 8);
#pragma unroll
  for (int u = 0; u < 8; ++u) vb[u] = (u < cnt && Ei != EXP_NONFINITE) ? dbits(__ldg(a + u)) : 0ull;
  if constexpr (MODE == 3)
    slice8_auto_store(vb, Ei, s, bits, slices + row * kp + c0, static_cast<size_t>(plane_rows) * kp, cnt);
  else
    slice8_store<MODE>(vb, Ei, s, slices + row * kp + c0, static_cast<size_t>(plane_rows) * kp, cnt);
}

// Slices of the 64 (k) x 32 (n) block of B at (k0, n0), transposed through
// shared memory into [S][n][kp]. Needs 256 threads; contains __syncthreads.
template <int MODE>
__device__ __forceinline__ void slice_cols_body(const double* __restrict__ B, int64_t k, int64_t n, int64_t ldb,
                                                const uint64_t* __restrict__ colmax, int s, int64_t kp,
                                                typename SliceElem<MODE>::T* __restrict__ slices,
                                                int32_t* __restrict__ F,
                                                uint32_t* __restrict__ err, int64_t k0, int64_t n0,
                                                int bits = 0) {
  __shared__ uint64_t tile[64][33];
  __shared__ int32_t fexp[32];
  const int t = threadIdx.x;
  if (t < 32) {
    const int64_t j = n0 + t;
    int32_t Fj = 0;
    if (j < n) {
      Fj = exponent_from_max(colmax[j], exp_offset(MODE));
      if (k0 == 0) {
        F[j] = Fj;
        if (Fj == EXP_NONFINITE) atomicOr(err, MM_DEV_ERR_NONFINITE);
      }
    }
    fexp[t] = Fj;
  }
  if (MODE != 1 && MODE != 3 && s > SLICE_S_MAX) return;   // plain FP64 fallback: F only (uniform over the block)
  if (MODE == 3 && s > SLICE_S_MAX && s <= SLICE_CRT_BASE) return;
  {
    // load 64 x 32 doubles: thread -> row t/4, columns (t%4)*8 .. +8
    const int r = t >> 2, cb = (t & 3) * 8;
    const int64_t gr = k0 + r;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t gc = n0 + cb + u;
      tile[r][cb + u] = (gr < k && gc < n) ? dbits(__ldg(B + gr * ldb + gc)) : 0ull;
    }
  }
  __syncthreads();
  // compute: thread -> column t/8, k sub-range (t%8)*8 .. +8
  const int jl = t >> 3, kb = (t & 7) * 8;
  const int64_t j = n0 + jl, c0 = k0 + kb;
  if (j < n && c0 < k) {
    const int32_t Fj = fexp[jl];
    const int cnt = static_cast<int>((k - c0) < 8 ? (k - c0) : 8);
    uint64_t vb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) vb[u] = (Fj == EXP_NONFINITE || u >= cnt) ? 0ull : tile[kb + u][jl];
    if constexpr (MODE == 3)
      slice8_auto_store(vb, Fj, s, bits, slices + j * kp + c0, static_cast<size_t>(n) * kp, cnt);
    else
      slice8_store<MODE>(vb, Fj, s, slices + j * kp + c0, static_cast<size_t>(n) * kp, cnt);
  }
  __syncthreads();  // the tile is reused by the next block of a persistent loop
}

// -------------------------------------------------- single-product kernels
// SPREAD: also the rows' spreads, merged into *amin.
template <bool SPREAD>
__global__ void __launch_bounds__(256) row_absmax_kernel(const double* __restrict__ A, int64_t m, int64_t k,
                                                         int64_t lda, uint64_t* __restrict__ rowmax,
                                                         uint32_t* __restrict__ amin) {
  const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row < m) {
    const float al = row_absmax_body<SPREAD>(A, k, lda, row, rowmax);
    if constexpr (SPREAD) warp_min_to(al, amin);
  }
}

template <bool SPREAD>
__global__ void col_absmax_kernel(const double* __restrict__ B, int64_t k, int64_t n, int64_t ldb,
                                  int64_t rows_per_block, unsigned long long* __restrict__ colmax,
                                  uint2* __restrict__ colpart) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rows_per_block;
  col_absmax_body<SPREAD>(B, ldb, j, r0, min(k, r0 + rows_per_block), colmax,
                          SPREAD ? colpart + static_cast<int64_t>(blockIdx.y) * n + j : nullptr);
}

// Both maxima in one launch: blocks [0, row_blocks) take 8 rows of A each (a
// warp per row), the rest 256 columns x rows_per_block rows of B each, so the
// two read streams overlap and the launch's ramp and tail are paid once.
// SPREAD: rows' spreads into *amin, columns' partial sums into colpart
// (record p * n + j for rows [p rows_per_block, (p+1) rows_per_block)).
template <bool SPREAD>
__global__ void __launch_bounds__(256) absmax_both_kernel(const double* __restrict__ A, int64_t m, int64_t k,
                                                          int64_t lda, uint64_t* __restrict__ rowmax,
                                                          const double* __restrict__ B, int64_t n, int64_t ldb,
                                                          int64_t rows_per_block, unsigned long long* __restrict__ colmax,
                                                          int row_blocks, int col_bx, uint32_t* __restrict__ amin,
                                                          uint2* __restrict__ colpart) {
  const int b = static_cast<int>(blockIdx.x);
  if (b < row_blocks) {
    const int64_t row = static_cast<int64_t>(b) * 8 + (threadIdx.x >> 5);
    if (row < m) {
      const float al = row_absmax_body<SPREAD>(A, k, lda, row, rowmax);
      if constexpr (SPREAD) warp_min_to(al, amin);
    }
    return;
  }
  const int cb = b - row_blocks;
  const int64_t j = static_cast<int64_t>(cb % col_bx) * 256 + threadIdx.x;
  if (j >= n) return;
  const int64_t p = cb / col_bx, r0 = p * rows_per_block;
  col_absmax_body<SPREAD>(B, ldb, j, r0, min(k, r0 + rows_per_block), colmax, SPREAD ? colpart + p * n + j : nullptr);
}

// The columns' spreads from their partial sums, merged into *bmin.
__global__ void __launch_bounds__(256) col_spread_kernel(const uint64_t* __restrict__ colmax,
                                                         const uint2* __restrict__ colpart, int64_t n, int64_t k,
                                                         int64_t parts, uint32_t* __restrict__ bmin) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const float be = (j < n) ? col_spread_body(colmax, colpart, n, k, parts, j) : __uint_as_float(0x7F800000u);
  block_min_to(be, bmin);
}

template <int MODE>
__global__ void slice_rows_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t lda,
                                  const uint64_t* __restrict__ rowmax, int s, int64_t kp, void* __restrict__ slices,
                                  int32_t* __restrict__ E, uint32_t* __restrict__ err, int64_t plane_rows,
                                  SliceDecision* dec) {
  const int64_t row = blockIdx.x;
  const int64_t c0 = (static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x) * 8;
  int bits = 0;
  const int se = (MODE == 3) ? decided_fp64(dec, &bits)
                             : decided_slices(dec, s, k, blockIdx.x == 0 && blockIdx.y == 0, MODE == 2 ? 0.5f : 1.0f);
  if (row < m && c0 < k)
    slice_rows_body<MODE>(A, plane_rows, k, lda, rowmax, se, kp, static_cast<typename SliceElem<MODE>::T*>(slices), E,
                          err, row, c0, bits);
}

template <int MODE>
__global__ void __launch_bounds__(256) slice_cols_kernel(const double* __restrict__ B, int64_t k, int64_t n,
                                                         int64_t ldb, const uint64_t* __restrict__ colmax, int s,
                                                         int64_t kp, void* __restrict__ slices,
                                                         int32_t* __restrict__ F, uint32_t* __restrict__ err,
                                                         SliceDecision* dec) {
  int bits = 0;
  const int se = (MODE == 3) ? decided_fp64(dec, &bits) : decided_slices(dec, s, k, false, MODE == 2 ? 0.5f : 1.0f);
  slice_cols_body<MODE>(B, k, n, ldb, colmax, se, kp, static_cast<typename SliceElem<MODE>::T*>(slices), F, err,
                        static_cast<int64_t>(blockIdx.y) * 64, static_cast<int64_t>(blockIdx.x) * 32, bits);
}

// --------------------------------------------------------- grouped kernels
// Problem of virtual block vb: the last p with off[p] <= vb (binary search).
__device__ __forceinline__ int find_problem(const int64_t* __restrict__ off, int count, int64_t vb) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= vb) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// A block's copy of two kinds' block offsets in shared memory, so the search
// for each virtual block costs shared loads, not a chain of dependent global
// ones. Groups of more than GS_MAXC problems search the global arrays.
constexpr int GS_MAXC = 1024;
struct OffCache {
  int64_t v[2][GS_MAXC + 1];
};

__device__ __forceinline__ void load_offsets(OffCache& oc, const GroupedSplitArgs& a, int k0, int k1, int count) {
  if (count <= GS_MAXC) {
    for (int i = threadIdx.x; i <= count; i += blockDim.x) {
      oc.v[0][i] = __ldg(a.off[k0] + i);
      oc.v[1][i] = __ldg(a.off[k1] + i);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ const int64_t* offsets(const OffCache& oc, const GroupedSplitArgs& a, int which, int kind,
                                                  int count) {
  return count <= GS_MAXC ? oc.v[which] : a.off[kind];
}

// Phase 1: row maxima (8 rows per block) then column maxima (256 columns x
// 256 rows per block) of every problem.
__global__ void __launch_bounds__(256) grouped_absmax_kernel(const GroupedSplitArgs a) {
  __shared__ int pref[8][32];
  __shared__ float psum[8][32];
  __shared__ OffCache oc;
  const int count = *a.count_dev;
  load_offsets(oc, a, 0, 1, count);
  const int64_t* off0 = offsets(oc, a, 0, 0, count);
  const int64_t* off1 = offsets(oc, a, 1, 1, count);
  const int64_t t0 = off0[count], t1 = off1[count];
  for (int64_t vb = blockIdx.x; vb < t0 + t1; vb += gridDim.x) {
    if (vb < t0) {
      const int p = find_problem(off0, count, vb);
      const GroupedSplit& g = a.probs[p];
      const int64_t row = (vb - off0[p]) * 8 + (threadIdx.x >> 5);
      if (g.dec != nullptr) {
        if (row < g.m) warp_min_to(row_absmax_body<true>(g.A, g.k, g.lda, row, g.rowmax), &g.dec->amin_room);
      } else if (row < g.m) {
        row_absmax_body<false>(g.A, g.k, g.lda, row, g.rowmax);
      }
    } else {
      const int64_t v = vb - t0;
      const int p = find_problem(off1, count, v);
      const GroupedSplit& g = a.probs[p];
      const int64_t lb = v - off1[p];
      // 32 columns x 256 rows per block: warp w takes rows r0 + w, r0 + w + 8, ...
      const int64_t ncb = (g.n + 31) / 32;
      const int lane = static_cast<int>(threadIdx.x & 31), w = static_cast<int>(threadIdx.x >> 5);
      const int64_t j = (lb % ncb) * 32 + lane, r0 = (lb / ncb) * 256 + w;
      uint64_t mx = 0;
      SpreadAcc acc;
      if (j < g.n) {
        const int64_t r1 = min(g.k, (lb / ncb) * 256 + 256);
        int64_t r = r0;
        // four rows in flight per thread, then the rest
        for (; r + 24 < r1; r += 32) {
          uint64_t b[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) b[u] = dbits(__ldg(g.B + (r + 8 * u) * g.ldb + j)) & ABS_MASK;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            mx = max(mx, b[u]);
            spread_add<true>(acc, b[u]);
          }
        }
        for (; r < r1; r += 8) {
          const uint64_t b = dbits(__ldg(g.B + r * g.ldb + j)) & ABS_MASK;
          mx = max(mx, b);
          spread_add<true>(acc, b);
        }
        if (mx) atomicMax(reinterpret_cast<unsigned long long*>(g.colmax) + j, static_cast<unsigned long long>(mx));
      }
      if (g.dec != nullptr) {
        // the 8 warps' sums of each column, merged in warp order
        pref[w][lane] = acc.ref;
        psum[w][lane] = acc.sum;
        __syncthreads();
        if (w == 0 && j < g.n) {
          SpreadAcc t;
          for (int i = 0; i < 8; ++i) {
            SpreadAcc o;
            o.ref = pref[i][lane];
            o.sum = psum[i][lane];
            t = spread_merge(t, o);
          }
          g.colpart[(lb / ncb) * g.n + j] = make_uint2(static_cast<uint32_t>(t.ref), __float_as_uint(t.sum));
        }
        __syncthreads();
      }
    }
  }
}

// Phase 1b (automatic slice count): every column's spread from its partial
// sums, 256 columns per block.
__global__ void __launch_bounds__(256) grouped_spread_kernel(const GroupedSplitArgs a) {
  __shared__ OffCache oc;
  const int count = *a.count_dev;
  load_offsets(oc, a, 4, 4, count);
  const int64_t* off4 = offsets(oc, a, 0, 4, count);
  const int64_t t4 = off4[count];
  for (int64_t vb = blockIdx.x; vb < t4; vb += gridDim.x) {
    const int p = find_problem(off4, count, vb);
    const GroupedSplit& g = a.probs[p];
    if (g.dec == nullptr) continue;   // uniform over the block
    const int64_t j = (vb - off4[p]) * 256 + threadIdx.x;
    const float be = (j < g.n) ? col_spread_body(g.colmax, g.colpart, g.n, g.k, (g.k + 255) / 256, j)
                               : __uint_as_float(0x7F800000u);
    block_min_to(be, &g.dec->bmin_room);
  }
}

// Between the phases, with the modular form allowed for some problem: one
// thread per problem records its decision (fp64_decision on its spreads, the
// modular form only where the problem allows it).
__global__ void __launch_bounds__(256) grouped_decide_kernel(const GroupedSplitArgs a) {
  const int count = *a.count_dev;
  for (int p = static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x); p < count;
       p += static_cast<int>(gridDim.x * blockDim.x)) {
    SliceDecision* d = a.probs[p].dec;
    if (d == nullptr) continue;
    int b = 0;
    const int code = fp64_decision(a.probs[p].k, spread_from_room(d->amin_room), spread_from_room(d->bmin_room),
                                   a.probs[p].crt != 0, &b);
    d->s = code;
    d->bits = b;
  }
}

// Phase 2: slices of A, 256 runs of 8 entries per block taken row after row
// (so short rows share a block), then of every 64 x 32 block of B.
template <int MODE>
__global__ void __launch_bounds__(256) grouped_slice_kernel(const GroupedSplitArgs a) {
  __shared__ OffCache oc;
  const int count = *a.count_dev;
  load_offsets(oc, a, 2, 3, count);
  const int64_t* off2 = offsets(oc, a, 0, 2, count);
  const int64_t* off3 = offsets(oc, a, 1, 3, count);
  const int64_t t2 = off2[count], t3 = off3[count];
  for (int64_t vb = blockIdx.x; vb < t2 + t3; vb += gridDim.x) {
    if (vb < t2) {
      const int p = find_problem(off2, count, vb);
      const GroupedSplit& g = a.probs[p];
      const int64_t lb = vb - off2[p];
      const int64_t runs = (g.k + 7) / 8;   // runs of 8 entries per row
      const int64_t u = lb * 256 + threadIdx.x;
      const int64_t row = u / runs, c0 = (u - row * runs) * 8;
      int bits = 0;
      const int se = (MODE == 3) ? decided_fp64(g.dec, &bits) : decided_slices(g.dec, g.s, g.k, lb == 0);
      if (row < g.m)
        slice_rows_body<MODE>(g.A, g.m, g.k, g.lda, g.rowmax, se, g.kp, g.slA, g.E, g.perr ? g.perr : a.err, row, c0,
                              bits);
    } else {
      const int64_t v = vb - t2;
      const int p = find_problem(off3, count, v);
      const GroupedSplit& g = a.probs[p];
      const int64_t lb = v - off3[p];
      const int64_t nnb = (g.n + 31) / 32;
      int bits = 0;
      const int se = (MODE == 3) ? decided_fp64(g.dec, &bits) : decided_slices(g.dec, g.s, g.k, false);
      slice_cols_body<MODE>(g.B, g.k, g.n, g.ldb, g.colmax, se, g.kp, g.slB, g.F, g.perr ? g.perr : a.err, (lb / nnb) * 64,
                            (lb % nnb) * 32, bits);
    }
  }
}

// --------------------------------------------------------- seeded inputs
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ double unit_draw(uint64_t base, uint64_t i) {
  uint64_t w = splitmix_mix(base + (i + 1ull) * GOLDEN);
  return static_cast<double>(w >> 11) * 0x1.0p-53;
}

__global__ void fill_uniform_kernel(double* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                                    uint64_t base, int scale_mode, uint64_t exp_base) {
  int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t total = rows * cols;
  for (; idx < total; idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t r = idx / cols, c = idx - r * cols;
    double v = 2.0 * unit_draw(base, static_cast<uint64_t>(idx)) - 1.0;
    if (scale_mode) {
      uint64_t ei = (scale_mode == 1) ? static_cast<uint64_t>(r) : static_cast<uint64_t>(c);
      double u = unit_draw(exp_base, ei);
      int e = -20 + static_cast<int>(floor(u * 41.0));
      // exact power-of-two scaling through the exponent field (|v| < 1, e in [-20, 20])
      uint64_t b = dbits(v);
      if ((b & ABS_MASK) != 0) b += static_cast<uint64_t>(static_cast<int64_t>(e)) << 52;
      v = __longlong_as_double(static_cast<long long>(b));
    }
    X[r * ld + c] = v;
  }
}

}  // namespace mmdev

// --------------------------------------------------------------- launchers
using namespace mmdev;

int64_t launch_absmax_parts(int64_t k) { return (k + 255) / 256; }

cudaError_t launch_absmax(const double* A, int64_t m, int64_t k, int64_t lda, const double* B, int64_t n,
                          int64_t ldb, uint64_t* rowmax, uint64_t* colmax, cudaStream_t st, int* nlaunch,
                          SliceDecision* dec, uint2* colpart) {
  if (nlaunch) *nlaunch = 0;
  const bool spread = dec != nullptr;
  uint32_t* amin = spread ? &dec->amin_room : nullptr;
  const int64_t rpb = 256;   // rows of B per column block: one partial record each
  bool cols_done = false;
  if (m > 0 && n > 0 && k > 0) {
    cudaError_t e = cudaMemsetAsync(colmax, 0, sizeof(uint64_t) * n, st);
    if (e != cudaSuccess) return e;
    const int64_t row_blocks = (m + 7) / 8, col_bx = (n + 255) / 256, col_by = (k + rpb - 1) / rpb;
    const int64_t blocks = row_blocks + col_bx * col_by;
    if (blocks <= 0x7fffffff) {
      if (spread)
        absmax_both_kernel<true><<<static_cast<unsigned>(blocks), 256, 0, st>>>(
            A, m, k, lda, rowmax, B, n, ldb, rpb, reinterpret_cast<unsigned long long*>(colmax),
            static_cast<int>(row_blocks), static_cast<int>(col_bx), amin, colpart);
      else
        absmax_both_kernel<false><<<static_cast<unsigned>(blocks), 256, 0, st>>>(
            A, m, k, lda, rowmax, B, n, ldb, rpb, reinterpret_cast<unsigned long long*>(colmax),
            static_cast<int>(row_blocks), static_cast<int>(col_bx), nullptr, nullptr);
      if (nlaunch) *nlaunch = 1;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      m = 0;   // both done
      cols_done = true;
    }
  }
  if (m > 0) {
    dim3 blk(256), grd(static_cast<unsigned>((m + 7) / 8));
    if (spread)
      row_absmax_kernel<true><<<grd, blk, 0, st>>>(A, m, k, lda, rowmax, amin);
    else
      row_absmax_kernel<false><<<grd, blk, 0, st>>>(A, m, k, lda, rowmax, nullptr);
    if (nlaunch) ++*nlaunch;
  }
  if (n > 0 && !cols_done) {
    cudaError_t e = cudaMemsetAsync(colmax, 0, sizeof(uint64_t) * n, st);
    if (e != cudaSuccess) return e;
    dim3 blk(128), grd(static_cast<unsigned>((n + 127) / 128), static_cast<unsigned>((k + rpb - 1) / rpb));
    if (k > 0) {
      if (spread)
        col_absmax_kernel<true><<<grd, blk, 0, st>>>(B, k, n, ldb, rpb, reinterpret_cast<unsigned long long*>(colmax),
                                                     colpart);
      else
        col_absmax_kernel<false><<<grd, blk, 0, st>>>(B, k, n, ldb, rpb, reinterpret_cast<unsigned long long*>(colmax),
                                                      nullptr);
      if (nlaunch) ++*nlaunch;
    }
  }
  if (spread && n > 0 && k > 0) {
    col_spread_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(colmax, colpart, n, k,
                                                                               launch_absmax_parts(k), &dec->bmin_room);
    if (nlaunch) ++*nlaunch;
  }
  return cudaGetLastError();
}

cudaError_t launch_slice_rows(int mode, const double* A, int64_t m, int64_t k, int64_t lda, const uint64_t* rowmax,
                              int s, int64_t kp, void* slices, int32_t* E, uint32_t* err, cudaStream_t st,
                              int64_t plane_rows, SliceDecision* dec) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  if (plane_rows < m) plane_rows = m;
  dim3 blk(128), grd(static_cast<unsigned>(m), static_cast<unsigned>((k + 1023) / 1024));
  if (mode == 0)
    slice_rows_kernel<0><<<grd, blk, 0, st>>>(A, m, k, lda, rowmax, s, kp, slices, E, err, plane_rows, dec);
  else if (mode == 3)
    slice_rows_kernel<3><<<grd, blk, 0, st>>>(A, m, k, lda, rowmax, s, kp, slices, E, err, plane_rows, dec);
  else if (mode == 2)
    slice_rows_kernel<2><<<grd, blk, 0, st>>>(A, m, k, lda, rowmax, s, kp, slices, E, err, plane_rows, dec);
  else
    slice_rows_kernel<1><<<grd, blk, 0, st>>>(A, m, k, lda, rowmax, s, kp, slices, E, err, plane_rows, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_slice_cols(int mode, const double* B, int64_t k, int64_t n, int64_t ldb, const uint64_t* colmax,
                              int s, int64_t kp, void* slices, int32_t* F, uint32_t* err, cudaStream_t st,
                              SliceDecision* dec) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  dim3 blk(256), grd(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((k + 63) / 64));
  if (mode == 0)
    slice_cols_kernel<0><<<grd, blk, 0, st>>>(B, k, n, ldb, colmax, s, kp, slices, F, err, dec);
  else if (mode == 3)
    slice_cols_kernel<3><<<grd, blk, 0, st>>>(B, k, n, ldb, colmax, s, kp, slices, F, err, dec);
  else if (mode == 2)
    slice_cols_kernel<2><<<grd, blk, 0, st>>>(B, k, n, ldb, colmax, s, kp, slices, F, err, dec);
  else
    slice_cols_kernel<1><<<grd, blk, 0, st>>>(B, k, n, ldb, colmax, s, kp, slices, F, err, nullptr);
  return cudaGetLastError();
}

namespace mmdev {
__global__ void crt_residues_out_kernel(const uint8_t* __restrict__ res, int64_t rplane, int64_t blk, int N,
                                        int64_t m, int64_t n, uint8_t* __restrict__ out) {
  const int64_t total = static_cast<int64_t>(N) * m * n;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t l = i / (m * n), r = (i / n) % m, c = i % n;
    out[i] = res[l * rplane + (c >> 3) * blk + r * 8 + (c & 7)];
  }
}
}  // namespace mmdev

cudaError_t launch_crt_residues_out(const uint8_t* res, int64_t rplane, int64_t blk, int N, int64_t m, int64_t n,
                                   uint8_t* out, cudaStream_t st) {
  crt_residues_out_kernel<<<1024, 256, 0, st>>>(res, rplane, blk, N, m, n, out);
  return cudaGetLastError();
}

cudaError_t launch_decide_fp64(SliceDecision* dec, int64_t k, cudaStream_t st) {
  decide_fp64_kernel<<<1, 32, 0, st>>>(dec, k);
  return cudaGetLastError();
}

cudaError_t launch_grouped_split(int mode01, const GroupedSplitArgs& a, int grid, cudaStream_t st) {
  grouped_absmax_kernel<<<grid, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (mode01 == 0 || mode01 == 3) {
    grouped_spread_kernel<<<grid, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (mode01 == 3) {
    grouped_decide_kernel<<<4, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    grouped_slice_kernel<3><<<grid, 256, 0, st>>>(a);
  } else if (mode01 == 0) {
    grouped_slice_kernel<0><<<grid, 256, 0, st>>>(a);
  } else {
    grouped_slice_kernel<1><<<grid, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_fill_uniform(double* X, int64_t rows, int64_t cols, int64_t ld, uint64_t seed, uint64_t stream_id,
                                int scale_mode, uint64_t exp_stream_id, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  uint64_t base = splitmix_mix_host(seed + stream_id * 0x9E3779B97F4A7C15ull);
  uint64_t ebase = splitmix_mix_host(seed + exp_stream_id * 0x9E3779B97F4A7C15ull);
  int64_t total = rows * cols;
  unsigned blocks = static_cast<unsigned>((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
  fill_uniform_kernel<<<blocks, 256, 0, st>>>(X, rows, cols, ld, base, scale_mode, ebase);
  return cudaGetLastError();
}

// ------------------------------------------------------------ wait probe
namespace mmdev {

// One thread waits, with the kernels' bounded wait, on an mbarrier that no
// thread ever arrives at: the wait gives up at the deadline, sets the timeout
// bit of the error word and the kernel returns normally.
__global__ void wait_probe_kernel(uint32_t* err, uint64_t timeout_ns, int* gave_up) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile uint32_t abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0u;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    WaitCtl wc;
    wc.abort = &abort_flag;
    wc.err = err;
    wc.deadline_ns = globaltimer_ns() + timeout_ns;
    *gave_up = mbar_wait(&bar, 0u, wc) ? 0 : 1;
  }
}

}  // namespace mmdev

cudaError_t launch_wait_probe(uint32_t* err, uint64_t timeout_ns, int* gave_up, cudaStream_t st) {
  mmdev::wait_probe_kernel<<<1, 32, 0, st>>>(err, timeout_ns, gave_up);
  return cudaGetLastError();
}

