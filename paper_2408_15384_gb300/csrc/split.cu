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

// FP64-accuracy digits of one entry: out[p] for p = 0..s-1, most significant
// first, as bfloat16 bit patterns.
__device__ __forceinline__ void fp64_digits(uint64_t bits, int sh, int s, uint16_t* out) {
  int64_t R = scaled_rne(bits, sh);
  for (int p = s - 1; p >= 1; --p) {
    int64_t d = ((R + 128) & 255) - 128;
    out[p] = bf16_of_small_int(static_cast<int32_t>(d));
    R = (R - d) >> 8;
  }
  out[0] = bf16_of_small_int(static_cast<int32_t>(R));
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
      q = a >> sh;
      uint64_t rem = a & ((1ull << sh) - 1ull);
      uint64_t half = 1ull << (sh - 1);
      if (rem > half || (rem == half && (q & 1ull))) ++q;
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
  while (q < 128 && L > -133) {
    q <<= 1;
    --L;
  }
  if (q < 128) return static_cast<uint16_t>(sgn | q);  // subnormal bfloat16, L == -133
  int biased = L + 7 + 127;
  return static_cast<uint16_t>(sgn | (static_cast<uint32_t>(biased) << 7) | static_cast<uint32_t>(q - 128));
}

__device__ __forceinline__ void fp32_slices3(uint64_t bits, int E, uint16_t* out) {
  uint64_t ab = bits & ABS_MASK;
  if (ab == 0) {
    out[0] = out[1] = out[2] = 0;
    return;
  }
  uint64_t mant;
  int e;
  decompose(ab, mant, e);
  int64_t M = (bits >> 63) ? -static_cast<int64_t>(mant) : static_cast<int64_t>(mant);
  e -= E;
  out[0] = bf16_rne_take(M, e);
  out[1] = bf16_rne_take(M, e);
  out[2] = bf16_rne_take(M, e);
}

// -------------------------------------------------------------- scan kernels
// One warp per row: maximum of |a| bits over the row.
__global__ void row_absmax_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t lda,
                                  uint64_t* __restrict__ rowmax) {
  int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= m) return;
  const double* a = A + row * lda;
  uint64_t mx = 0;
  uint32_t lane = threadIdx.x & 31u;
  int64_t c = lane;
  for (; c + 96 < k; c += 128) {
    uint64_t v0 = dbits(__ldg(a + c)) & ABS_MASK, v1 = dbits(__ldg(a + c + 32)) & ABS_MASK;
    uint64_t v2 = dbits(__ldg(a + c + 64)) & ABS_MASK, v3 = dbits(__ldg(a + c + 96)) & ABS_MASK;
    mx = max(mx, max(max(v0, v1), max(v2, v3)));
  }
  for (; c < k; c += 32) mx = max(mx, dbits(__ldg(a + c)) & ABS_MASK);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, static_cast<uint64_t>(__shfl_xor_sync(0xffffffffu, static_cast<unsigned long long>(mx), o)));
  if (lane == 0) rowmax[row] = mx;
}

// Column maxima of B (k x n): thread per column over a range of rows, merged
// with atomicMax (colmax must be zeroed first).
__global__ void col_absmax_kernel(const double* __restrict__ B, int64_t k, int64_t n, int64_t ldb,
                                  int64_t rows_per_block, unsigned long long* __restrict__ colmax) {
  int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int64_t r0 = static_cast<int64_t>(blockIdx.y) * rows_per_block;
  int64_t r1 = min(k, r0 + rows_per_block);
  uint64_t mx = 0;
  for (int64_t r = r0; r < r1; ++r) mx = max(mx, dbits(__ldg(B + r * ldb + j)) & ABS_MASK);
  if (mx) atomicMax(colmax + j, static_cast<unsigned long long>(mx));
}

// ------------------------------------------------------------ slice kernels
// A (m x k, rows scaled): thread handles 8 consecutive entries of one row.
// Writes slices [S][m][kp] (bf16 bits), E[m]; raises NONFINITE in err.
template <int MODE>  // 0: FP64-accuracy digits, 1: FP32-accuracy bf16 slices
__global__ void slice_rows_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t lda,
                                  const uint64_t* __restrict__ rowmax, int s, int64_t kp,
                                  uint16_t* __restrict__ slices, int32_t* __restrict__ E,
                                  uint32_t* __restrict__ err) {
  int64_t row = blockIdx.x;
  int64_t c0 = (static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x) * 8;
  if (row >= m || c0 >= k) return;
  uint64_t mx = rowmax[row];
  int32_t Ei = exponent_from_max(mx, MODE == 0 ? 2 : 1);
  if (c0 == 0) {
    E[row] = Ei;
    if (Ei == EXP_NONFINITE) atomicOr(err, MM_DEV_ERR_NONFINITE);
  }
  const double* a = A + row * lda + c0;
  uint64_t vb[8];
  int cnt = static_cast<int>((k - c0) < 8 ? (k - c0) : 8);
#pragma unroll
  for (int u = 0; u < 8; ++u) vb[u] = (u < cnt) ? dbits(__ldg(a + u)) : 0ull;
  if (Ei == EXP_NONFINITE) {
#pragma unroll
    for (int u = 0; u < 8; ++u) vb[u] = 0ull;
  }
  const int S = (MODE == 0) ? s : 3;
  const size_t plane = static_cast<size_t>(m) * kp;
  uint16_t dig[8][8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (MODE == 0)
      fp64_digits(vb[u], 8 * s - Ei, s, dig[u]);
    else
      fp32_slices3(vb[u], Ei, dig[u]);
  }
  uint16_t* dst = slices + row * kp + c0;
  bool vec = (cnt == 8) && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0);
  for (int p = 0; p < S; ++p) {
    uint16_t* d = dst + p * plane;
    if (vec) {
      uint4 w;
      w.x = dig[0][p] | (static_cast<uint32_t>(dig[1][p]) << 16);
      w.y = dig[2][p] | (static_cast<uint32_t>(dig[3][p]) << 16);
      w.z = dig[4][p] | (static_cast<uint32_t>(dig[5][p]) << 16);
      w.w = dig[6][p] | (static_cast<uint32_t>(dig[7][p]) << 16);
      *reinterpret_cast<uint4*>(d) = w;
    } else {
      for (int u = 0; u < cnt; ++u) d[u] = dig[u][p];
    }
  }
}

// B (k x n, columns scaled) -> slices [S][n][kp], transposed through shared
// memory: a block covers 64 rows (k) x 32 columns (n) of B.
template <int MODE>
__global__ void __launch_bounds__(256) slice_cols_kernel(const double* __restrict__ B, int64_t k, int64_t n,
                                                         int64_t ldb, const uint64_t* __restrict__ colmax, int s,
                                                         int64_t kp, uint16_t* __restrict__ slices,
                                                         int32_t* __restrict__ F, uint32_t* __restrict__ err) {
  __shared__ uint64_t tile[64][33];
  __shared__ int32_t fexp[32];
  int64_t k0 = static_cast<int64_t>(blockIdx.y) * 64;
  int64_t n0 = static_cast<int64_t>(blockIdx.x) * 32;
  int t = threadIdx.x;
  if (t < 32) {
    int64_t j = n0 + t;
    int32_t Fj = 0;
    if (j < n) {
      Fj = exponent_from_max(colmax[j], MODE == 0 ? 2 : 1);
      if (k0 == 0) {
        F[j] = Fj;
        if (Fj == EXP_NONFINITE) atomicOr(err, MM_DEV_ERR_NONFINITE);
      }
    }
    fexp[t] = Fj;
  }
  // load 64 x 32 doubles: thread -> row t/4, columns (t%4)*8 .. +8
  {
    int r = t >> 2, cb = (t & 3) * 8;
    int64_t gr = k0 + r;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      int64_t gc = n0 + cb + u;
      tile[r][cb + u] = (gr < k && gc < n) ? dbits(__ldg(B + gr * ldb + gc)) : 0ull;
    }
  }
  __syncthreads();
  // compute: thread -> column t/8, k sub-range (t%8)*8 .. +8
  int jl = t >> 3, kb = (t & 7) * 8;
  int64_t j = n0 + jl, c0 = k0 + kb;
  if (j >= n || c0 >= k) return;
  int32_t Fj = fexp[jl];
  int cnt = static_cast<int>((k - c0) < 8 ? (k - c0) : 8);
  const int S = (MODE == 0) ? s : 3;
  uint16_t dig[8][8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    uint64_t b = (Fj == EXP_NONFINITE) ? 0ull : tile[kb + u][jl];
    if (MODE == 0)
      fp64_digits(b, 8 * s - Fj, s, dig[u]);
    else
      fp32_slices3(b, Fj, dig[u]);
  }
  const size_t plane = static_cast<size_t>(n) * kp;
  uint16_t* dst = slices + j * kp + c0;
  bool vec = (cnt == 8) && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0);
  for (int p = 0; p < S; ++p) {
    uint16_t* d = dst + p * plane;
    if (vec) {
      uint4 w;
      w.x = dig[0][p] | (static_cast<uint32_t>(dig[1][p]) << 16);
      w.y = dig[2][p] | (static_cast<uint32_t>(dig[3][p]) << 16);
      w.z = dig[4][p] | (static_cast<uint32_t>(dig[5][p]) << 16);
      w.w = dig[6][p] | (static_cast<uint32_t>(dig[7][p]) << 16);
      *reinterpret_cast<uint4*>(d) = w;
    } else {
      for (int u = 0; u < cnt; ++u) d[u] = dig[u][p];
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

cudaError_t launch_absmax(const double* A, int64_t m, int64_t k, int64_t lda, const double* B, int64_t n,
                          int64_t ldb, uint64_t* rowmax, uint64_t* colmax, cudaStream_t st) {
  if (m > 0) {
    dim3 blk(256), grd(static_cast<unsigned>((m + 7) / 8));
    row_absmax_kernel<<<grd, blk, 0, st>>>(A, m, k, lda, rowmax);
  }
  if (n > 0) {
    cudaError_t e = cudaMemsetAsync(colmax, 0, sizeof(uint64_t) * n, st);
    if (e != cudaSuccess) return e;
    int64_t rpb = 256;
    dim3 blk(128), grd(static_cast<unsigned>((n + 127) / 128), static_cast<unsigned>((k + rpb - 1) / rpb));
    if (k > 0) col_absmax_kernel<<<grd, blk, 0, st>>>(B, k, n, ldb, rpb, reinterpret_cast<unsigned long long*>(colmax));
  }
  return cudaGetLastError();
}

cudaError_t launch_slice_rows(int mode, const double* A, int64_t m, int64_t k, int64_t lda, const uint64_t* rowmax,
                              int s, int64_t kp, uint16_t* slices, int32_t* E, uint32_t* err, cudaStream_t st) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  dim3 blk(128), grd(static_cast<unsigned>(m), static_cast<unsigned>((k + 1023) / 1024));
  if (mode == 0)
    slice_rows_kernel<0><<<grd, blk, 0, st>>>(A, m, k, lda, rowmax, s, kp, slices, E, err);
  else
    slice_rows_kernel<1><<<grd, blk, 0, st>>>(A, m, k, lda, rowmax, s, kp, slices, E, err);
  return cudaGetLastError();
}

cudaError_t launch_slice_cols(int mode, const double* B, int64_t k, int64_t n, int64_t ldb, const uint64_t* colmax,
                              int s, int64_t kp, uint16_t* slices, int32_t* F, uint32_t* err, cudaStream_t st) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  dim3 blk(256), grd(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((k + 63) / 64));
  if (mode == 0)
    slice_cols_kernel<0><<<grd, blk, 0, st>>>(B, k, n, ldb, colmax, s, kp, slices, F, err);
  else
    slice_cols_kernel<1><<<grd, blk, 0, st>>>(B, k, n, ldb, colmax, s, kp, slices, F, err);
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
