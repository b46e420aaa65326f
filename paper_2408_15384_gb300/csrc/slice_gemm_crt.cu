// slice_gemm_crt.cu -- instances of the slice GEMM for the modular form of the
// FP64-accuracy product (SLICE_CRT: one residue product a modulus, the
// Chinese-remainder rebuild in the epilogue or as a pass of its own) and the
// rebuild constants.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "slice_gemm_kernel.cuh"

namespace mmdev {

namespace {

using u128 = unsigned __int128;

// x^-1 mod m for x coprime to m (m <= 256): the one y in [1, m) with x y = 1.
uint32_t inverse_mod(uint32_t x, uint32_t m) {
  x %= m;
  for (uint32_t y = 1; y < m; ++y)
    if ((x * y) % m == 1u) return y;
  return 0u;
}

// The rebuild constants for every modulus count: M_N, M_N / 2, 1/M_N and
// W_l = (M/m_l) ((M/m_l)^-1 mod m_l) mod M (congruent to 1 modulo m_l and to
// 0 modulo every other modulus).
CrtTab make_tab() {
  CrtTab t;
  memset(&t, 0, sizeof(t));
  for (int l = 0; l < CRT_N_MAX; ++l) {
    const uint32_t m = static_cast<uint32_t>(crt_modulus(l));
    t.magic[l] = static_cast<uint32_t>((1ull << 32) / m + 1ull);
    t.c16[l] = (1u << 16) % m;
    t.c31[l] = static_cast<int32_t>((1u << 31) % m);
  }
  for (int N = 1; N <= CRT_N_MAX; ++N) {
    u128 M = 1;
    for (int l = 0; l < N; ++l) M *= static_cast<uint32_t>(crt_modulus(l));
    for (int i = 0; i < 4; ++i) t.M[N][i] = static_cast<uint32_t>(M >> (32 * i));
    t.H[N][0] = static_cast<uint64_t>(M >> 1);
    t.H[N][1] = static_cast<uint64_t>(M >> 65);
    int bits = 0;
    for (u128 x = M; x != 0; x >>= 1) ++bits;
    t.wsh[N] = bits > 20 ? bits - 20 : 0;
    t.qscale[N] = static_cast<float>(std::ldexp(1.0, t.wsh[N]) / static_cast<double>(M));
    for (int l = 0; l < N; ++l) {
      const uint32_t m = static_cast<uint32_t>(crt_modulus(l));
      const u128 Ml = M / m;
      const uint32_t y = inverse_mod(static_cast<uint32_t>(Ml % m), m);
      const u128 W = (Ml * y) % M;
      for (int i = 0; i < 4; ++i) t.W[N][l][i] = static_cast<uint32_t>(W >> (32 * i));
    }
  }
  return t;
}

template <int BN, int CG>
cudaError_t launch_bn(const CUtensorMap* tmA, const CUtensorMap* tmB, const SliceGemmArgs& a, int grid,
                      cudaStream_t st) {
  return launch_t<BN, SLICE_CRT, CG>(tmA, tmB, a, grid, st);
}

// The rebuild as a pass of its own, after a slice GEMM launched with
// crt_defer. A block takes 32 rows x 64 columns of C: warp w the 8 columns
// 8w .. 8w+7 (one 8-byte residue record a modulus), lane r row r, so each
// residue load of a warp is 256 contiguous bytes. The outputs go through
// shared memory and leave as whole 256-byte row segments. N is a template
// parameter: the W_l and M words are compile-time constant-bank operands, and
// the words M_N does not need fold away.
constexpr int RB_ROWS = 32, RB_COLS = 64, RB_PITCH = RB_COLS + 1;   // doubles; odd pitch: 2-way stores at most

// M_N and its bit length, at compile time.
__host__ __device__ constexpr u128 modulus_product(int N) {
  u128 M = 1;
  for (int l = 0; l < N; ++l) M *= static_cast<unsigned>(crt_modulus(l));
  return M;
}
__host__ __device__ constexpr int bit_length(u128 x) {
  int b = 0;
  for (; x != 0; x >>= 1) ++b;
  return b;
}

// Compile-time constants of N <= 12 moduli (M_N < 2^95): M_N and M_N / 2 as
// 32-bit words, and the quotient window: S < 2^12 M_N, so S >> SH (SH = bit
// length of M_N minus 11) is below 2^23 and QS = 2^SH / M_N scales it to S / M_N
// within 2^-10.
template <int N>
struct Crt96 {
  static constexpr u128 M = modulus_product(N);
  static constexpr int BITS = bit_length(M);
  static constexpr uint32_t m0 = static_cast<uint32_t>(M), m1 = static_cast<uint32_t>(M >> 32),
                            m2 = static_cast<uint32_t>(M >> 64);
  static constexpr uint64_t Mlo = static_cast<uint64_t>(M), Hlo = static_cast<uint64_t>(M >> 1);
  static constexpr uint32_t Mhi = static_cast<uint32_t>(M >> 64), Hhi = static_cast<uint32_t>(M >> 65);
  static constexpr int SH = BITS > 11 ? BITS - 11 : 0;
  static constexpr float QS = static_cast<float>(static_cast<double>(u128(1) << SH) / static_cast<double>(M));
};

// One output of a product with N <= 12 moduli from the column sums T0..T2 of
// S = sum_l c_l W_l (the same value as crt_output, specialised): Y = S - q M
// is kept modulo 2^96 (|Y| < M_N < 2^95 before the one correction step), and a
// result in the normal range is rounded from the 96-bit magnitude directly;
// the rest (subnormal or overflowing results) take rn_double_bits.
template <int N>
__device__ __forceinline__ uint64_t crt_output96(uint64_t T0, uint64_t T1, uint64_t T2, int e) {
  using K = Crt96<N>;
  // S = hi 2^64 + a
  const uint64_t t1s = T1 << 32;
  const uint64_t a = T0 + t1s;
  const uint64_t hi = T2 + (T1 >> 32) + (a < t1s ? 1ull : 0ull);
  // q = round(S / M) from the top 23 bits of S
  uint32_t win;
  if constexpr (K::SH >= 64)
    win = static_cast<uint32_t>(hi >> (K::SH - 64));
  else if constexpr (K::SH > 0)
    win = static_cast<uint32_t>((a >> K::SH) | (hi << (64 - K::SH)));
  else
    win = static_cast<uint32_t>(a);
  const float wf = __uint_as_float(0x4B000000u | win) - 8388608.0f;   // exact: win < 2^23
  const uint32_t q = __float_as_uint(fmaf(wf, K::QS, 8388608.0f)) - 0x4B000000u;
  // Y = S - q M modulo 2^96: (yh, yl), yh the top 32 bits as signed
  const uint64_t p0 = static_cast<uint64_t>(q) * K::m0;
  const uint64_t p1 = static_cast<uint64_t>(q) * K::m1 + (p0 >> 32);
  const uint32_t p2 = q * K::m2 + static_cast<uint32_t>(p1 >> 32);
  const uint64_t qml = (p1 << 32) | (p0 & 0xFFFFFFFFull);
  uint64_t yl = a - qml;
  int32_t yh = static_cast<int32_t>(static_cast<uint32_t>(hi) - p2 - (a < qml ? 1u : 0u));
  // Y >= M/2: Y - M; Y < -M/2: Y + M (u = Y + M/2 outside [0, M))
  {
    const uint64_t ul = yl + K::Hlo;
    const int32_t uh = yh + static_cast<int32_t>(K::Hhi) + (ul < yl ? 1 : 0);
    if (uh < 0) {
      const uint64_t nl = yl + K::Mlo;
      yh = yh + static_cast<int32_t>(K::Mhi) + (nl < yl ? 1 : 0);
      yl = nl;
    } else if (static_cast<uint32_t>(uh) > K::Mhi || (static_cast<uint32_t>(uh) == K::Mhi && ul >= K::Mlo)) {
      const uint64_t nl = yl - K::Mlo;
      yh = yh - static_cast<int32_t>(K::Mhi) - (yl < K::Mlo ? 1 : 0);
      yl = nl;
    }
  }
  const bool neg = yh < 0;
  uint32_t u2 = static_cast<uint32_t>(yh);
  if (neg) {
    yl = ~yl + 1ull;
    u2 = ~u2 + (yl == 0ull ? 1u : 0u);
  }
  // |Y| = u2 2^64 + yl < 2^95: its leading 64 bits t (bit 63 set), the
  // exponent L of its leading bit, and whether any bit below t is set
  uint64_t t;
  int L;
  bool below;
  if (u2 != 0u) {
    const int sft = __clz(static_cast<int>(u2));   // 1 .. 31
    t = (static_cast<uint64_t>(u2) << (32 + sft)) | (yl >> (32 - sft));
    below = (static_cast<uint32_t>(yl) << sft) != 0u;
    L = 95 - sft;
  } else {
    if (yl == 0ull) return 0ull;
    const int sft = __clzll(static_cast<long long>(yl));
    t = yl << sft;
    below = false;
    L = 63 - sft;
  }
  const int E = L + e;
  if (E < -1021 || E > 1022)   // subnormal, overflowing, or rounding up to the edge: the general path
    return rn_double_bits(static_cast<uint64_t>(u2), yl, e, neg);
  uint64_t mant = t >> 11;                                       // 53 bits, leading bit set
  const bool rbit = (t >> 10) & 1ull;
  const bool sticky = below || (t & 0x3FFull) != 0ull;
  mant += (rbit && (sticky || (mant & 1ull))) ? 1ull : 0ull;
  const int Ef = E + static_cast<int>(mant >> 53);               // a carry out of the 53 bits
  return (neg ? (1ull << 63) : 0ull) | (static_cast<uint64_t>(Ef + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
}

template <int N>
__device__ __forceinline__ void rebuild_tile(const SliceProblem& P, int bits, int64_t r0, int64_t c0,
                                             double (*tile)[RB_PITCH]) {
  constexpr int NW = N <= 4 ? 1 : N <= 8 ? 2 : N <= 12 ? 3 : 4;   // 32-bit words of M_N
  const int r = static_cast<int>(threadIdx.x & 31), w = static_cast<int>(threadIdx.x >> 5);
  const int64_t row = r0 + r, cb = c0 + 8 * w;
  if (row < P.m && cb < P.n) {
    const uint8_t* const rb = P.res + row * 8 + (cb >> 3) * P.ldr;
    uint2 rec[N];
#pragma unroll
    for (int l = 0; l < N; ++l) rec[l] = *reinterpret_cast<const uint2*>(rb + static_cast<int64_t>(l) * P.rplane);
    const int32_t Ei = P.E[row];
    const int ebase = Ei - 2 * bits;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint64_t T0 = 0ull, T1 = 0ull, T2 = 0ull, T3 = 0ull;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const uint32_t cl = ((j < 4 ? rec[l].x : rec[l].y) >> (8 * (j & 3))) & 255u;
        T0 += static_cast<uint64_t>(cl) * c_crt.W[N][l][0];
        if (NW > 1) T1 += static_cast<uint64_t>(cl) * c_crt.W[N][l][1];
        if (NW > 2) T2 += static_cast<uint64_t>(cl) * c_crt.W[N][l][2];
        if (NW > 3) T3 += static_cast<uint64_t>(cl) * c_crt.W[N][l][3];
      }
      const int32_t Fj = cb + j < P.n ? __ldg(P.F + cb + j) : 0;
      uint64_t o;
      if (Ei == EXP_NONFINITE || Fj == EXP_NONFINITE)
        o = 0x7FF8000000000000ull;
      else if constexpr (N <= 12)
        o = crt_output96<N>(T0, T1, T2, ebase + Fj);
      else
        o = crt_output<4>(T0, T1, T2, T3, crt_k<4>(N), ebase + Fj);
      tile[r][8 * w + j] = __longlong_as_double(static_cast<long long>(o));
    }
  }
  __syncthreads();
  // warp w writes rows w, w + 8, w + 16, w + 24: lanes on consecutive columns
#pragma unroll
  for (int i = 0; i < RB_ROWS / 8; ++i) {
    const int rr = w + 8 * i;
    const int64_t orow = r0 + rr;
    if (orow < P.m) {
      double* const crow = P.C + orow * P.ldc + c0;
      if (c0 + r < P.n) crow[r] = tile[rr][r];
      if (c0 + 32 + r < P.n) crow[32 + r] = tile[rr][32 + r];
    }
  }
  __syncthreads();
}

template <int N>
__device__ __forceinline__ void rebuild_all(const SliceProblem& P, int bits, double (*tile)[RB_PITCH]) {
  const int64_t rblocks = (P.m + RB_ROWS - 1) / RB_ROWS, cblocks = (P.n + RB_COLS - 1) / RB_COLS;
  for (int64_t cbk = blockIdx.y; cbk < cblocks; cbk += gridDim.y)
    for (int64_t rbk = blockIdx.x; rbk < rblocks; rbk += gridDim.x)
      rebuild_tile<N>(P, bits, rbk * RB_ROWS, cbk * RB_COLS, tile);
}

// A product the digit form took (decision code at most SLICE_CRT_BASE)
// returns at once. Consecutive blocks take consecutive row blocks of the same
// columns, so each residue plane streams in order.
__global__ void __launch_bounds__(256, 3) crt_rebuild_kernel(const SliceProblem P) {
  __shared__ double tile[RB_ROWS][RB_PITCH];
  int N, bits;
  if (P.s_dev != nullptr) {
    const int code = *P.s_dev;
    if (code <= SLICE_CRT_BASE || code > SLICE_CRT_BASE + CRT_N_MAX) return;
    N = code - SLICE_CRT_BASE;
    bits = P.s_dev[1];
  } else {
    N = P.s;
    bits = P.fix_shift;
  }
  switch (N) {
    case 1: rebuild_all<1>(P, bits, tile); break;
    case 2: rebuild_all<2>(P, bits, tile); break;
    case 3: rebuild_all<3>(P, bits, tile); break;
    case 4: rebuild_all<4>(P, bits, tile); break;
    case 5: rebuild_all<5>(P, bits, tile); break;
    case 6: rebuild_all<6>(P, bits, tile); break;
    case 7: rebuild_all<7>(P, bits, tile); break;
    case 8: rebuild_all<8>(P, bits, tile); break;
    case 9: rebuild_all<9>(P, bits, tile); break;
    case 10: rebuild_all<10>(P, bits, tile); break;
    case 11: rebuild_all<11>(P, bits, tile); break;
    case 12: rebuild_all<12>(P, bits, tile); break;
    case 13: rebuild_all<13>(P, bits, tile); break;
    default: rebuild_all<14>(P, bits, tile); break;
  }
}

}  // namespace

cudaError_t slice_launch_crt(int bn, int cg, const CUtensorMap* tmA, const CUtensorMap* tmB, const SliceGemmArgs& a,
                             int grid, cudaStream_t st) {
  switch (bn * 4 + cg) {
    case 128 * 4 + 1: return launch_bn<128, 1>(tmA, tmB, a, grid, st);
    case 128 * 4 + 2: return launch_bn<128, 2>(tmA, tmB, a, grid, st);
    case 256 * 4 + 1: return launch_bn<256, 1>(tmA, tmB, a, grid, st);
    case 256 * 4 + 2: return launch_bn<256, 2>(tmA, tmB, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t slice_prepare_crt() {
  cudaError_t e;
  if ((e = set_smem_attr<128, SLICE_CRT, 1>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<128, SLICE_CRT, 2>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<256, SLICE_CRT, 1>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<256, SLICE_CRT, 2>()) != cudaSuccess) return e;
  static const CrtTab tab = make_tab();
  return cudaMemcpyToSymbol(c_crt, &tab, sizeof(tab));
}

int slice_max_pairs_crt() { return max_pairs_t<256, SLICE_CRT>(); }

}  // namespace mmdev

cudaError_t slice_rebuild_crt(const SliceProblem& P, int sm_count, cudaStream_t st) {
  const int64_t rblocks = (P.m + mmdev::RB_ROWS - 1) / mmdev::RB_ROWS;
  const int64_t cblocks = (P.n + mmdev::RB_COLS - 1) / mmdev::RB_COLS;
  if (rblocks <= 0 || cblocks <= 0) return cudaSuccess;
  // one block a tile (the grid strides only past the launch limits)
  (void)sm_count;
  const int64_t gy = std::min<int64_t>(cblocks, 65535);
  const int64_t gx = std::min<int64_t>(rblocks, 0x7FFFFFFF);
  mmdev::crt_rebuild_kernel<<<dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy)), 256, 0, st>>>(P);
  return cudaGetLastError();
}
