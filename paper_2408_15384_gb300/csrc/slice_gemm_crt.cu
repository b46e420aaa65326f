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

// Compile-time constants of N <= 12 moduli (M_N < 2^95) as 32-bit words:
// M_N, H = M_N / 2, NM = 2^96 - M_N (so S - q M = S + q NM modulo 2^96), H2
// = the top word of H, and the quotient window: S < 2^12 M_N, so S >> SH (SH
// = bit length of M_N minus 11) is below 2^23 and QS = 2^SH / M_N scales it to
// S / M_N within 2^-10.
template <int N>
struct Crt96 {
  static constexpr u128 M = modulus_product(N);
  static constexpr u128 H = M >> 1;
  static constexpr u128 NM = ((u128(1) << 96) - M) & ((u128(1) << 96) - 1);
  static constexpr int BITS = bit_length(M);
  static constexpr uint32_t m0 = static_cast<uint32_t>(M), m1 = static_cast<uint32_t>(M >> 32),
                            m2 = static_cast<uint32_t>(M >> 64);
  static constexpr uint32_t h0 = static_cast<uint32_t>(H), h1 = static_cast<uint32_t>(H >> 32),
                            h2 = static_cast<uint32_t>(H >> 64);
  static constexpr uint32_t n0 = static_cast<uint32_t>(NM), n1 = static_cast<uint32_t>(NM >> 32),
                            n2 = static_cast<uint32_t>(NM >> 64);
  static constexpr int SH = BITS > 11 ? BITS - 11 : 0;
  static constexpr float QS = static_cast<float>(static_cast<double>(u128(1) << SH) / static_cast<double>(M));
};

// 96-bit two's-complement words (least significant first) with the carry flag.
__device__ __forceinline__ void add96(uint32_t& a0, uint32_t& a1, uint32_t& a2, uint32_t b0, uint32_t b1,
                                      uint32_t b2) {
  asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
      : "+r"(a0), "+r"(a1), "+r"(a2)
      : "r"(b0), "r"(b1), "r"(b2));
}
__device__ __forceinline__ void sub96(uint32_t& a0, uint32_t& a1, uint32_t& a2, uint32_t b0, uint32_t b1,
                                      uint32_t b2) {
  asm("sub.cc.u32 %0, %0, %3;\n\tsubc.cc.u32 %1, %1, %4;\n\tsubc.u32 %2, %2, %5;"
      : "+r"(a0), "+r"(a1), "+r"(a2)
      : "r"(b0), "r"(b1), "r"(b2));
}

// One output of a product with N <= 12 moduli from the column sums T0..T2 of
// S = sum_l c_l W_l (the same value as crt_output, specialised): Y = S - q M
// is kept modulo 2^96 (|Y| <= 0.501 M_N < 2^94 before the correction), and a
// result in the normal range is rounded from the 96-bit magnitude directly;
// the rest (subnormal or overflowing results) take rn_double_bits.
template <int N>
__device__ __forceinline__ uint64_t crt_output96(uint64_t T0, uint64_t T1, uint64_t T2, int e) {
  using K = Crt96<N>;
  // S = T0 + T1 2^32 + T2 2^64 as words s0..s3 (s3 < 2^12)
  const uint32_t s0 = static_cast<uint32_t>(T0);
  uint32_t s1, s2, s3;
  asm("add.cc.u32 %0, %3, %4;\n\taddc.cc.u32 %1, %5, %6;\n\taddc.u32 %2, %7, 0;"
      : "=r"(s1), "=r"(s2), "=r"(s3)
      : "r"(static_cast<uint32_t>(T0 >> 32)), "r"(static_cast<uint32_t>(T1)), "r"(static_cast<uint32_t>(T1 >> 32)),
        "r"(static_cast<uint32_t>(T2)), "r"(static_cast<uint32_t>(T2 >> 32)));
  // q = round(S / M) from the 23 bits of S from bit SH up
  uint32_t win;
  {
    constexpr int w = K::SH / 32, r = K::SH % 32;
    const uint32_t wd[5] = {s0, s1, s2, s3, 0u};
    win = r == 0 ? wd[w] : __funnelshift_r(wd[w], wd[w + 1], r);
  }
  const float wf = __uint_as_float(0x4B000000u | win) - 8388608.0f;   // exact: win < 2^23
  const uint32_t q = __float_as_uint(fmaf(wf, K::QS, 8388608.0f)) - 0x4B000000u;
  // Y = S + q (2^96 - M) modulo 2^96
  uint32_t y0, y1, y2;
  asm("mad.lo.cc.u32 %0, %3, %4, %7;\n\t"
      "madc.hi.cc.u32 %1, %3, %4, %8;\n\t"
      "madc.hi.u32 %2, %3, %5, %9;\n\t"
      "mad.lo.cc.u32 %1, %3, %5, %1;\n\t"
      "madc.lo.u32 %2, %3, %6, %2;"
      : "=r"(y0), "=r"(y1), "=r"(y2)
      : "r"(q), "r"(K::n0), "r"(K::n1), "r"(K::n2), "r"(s0), "r"(s1), "r"(s2));
  // Y in [-M/2, M/2) for sure when its top word lies in [-h2, h2); else the
  // exact correction (Y + H outside [0, M): Y + M or Y - M)
  if (!(K::h2 > 0u && static_cast<uint32_t>(y2 + K::h2) < 2u * K::h2)) {
    uint32_t u0 = y0, u1 = y1, u2 = y2;
    add96(u0, u1, u2, K::h0, K::h1, K::h2);
    if (static_cast<int32_t>(u2) < 0) {
      add96(y0, y1, y2, K::m0, K::m1, K::m2);
    } else {
      sub96(u0, u1, u2, K::m0, K::m1, K::m2);
      if (static_cast<int32_t>(u2) >= 0) sub96(y0, y1, y2, K::m0, K::m1, K::m2);
    }
  }
  // |Y| and its sign
  const uint32_t sg = static_cast<uint32_t>(static_cast<int32_t>(y2) >> 31);
  y0 ^= sg;
  y1 ^= sg;
  y2 ^= sg;
  add96(y0, y1, y2, sg & 1u, 0u, 0u);
  const bool neg = sg != 0u;
  // the leading 64 bits th:tl of |Y| (bit 63 set), the exponent L of its
  // leading bit, and the bits below them (rest)
  uint32_t th, tl, rest;
  int L;
  if (y2 != 0u) {
    const int sft = __clz(static_cast<int>(y2));
    th = __funnelshift_l(y1, y2, sft);
    tl = __funnelshift_l(y0, y1, sft);
    rest = y0 << sft;
    L = 95 - sft;
  } else if (y1 != 0u) {
    const int sft = __clz(static_cast<int>(y1));
    th = __funnelshift_l(y0, y1, sft);
    tl = y0 << sft;
    rest = 0u;
    L = 63 - sft;
  } else {
    if (y0 == 0u) return 0ull;
    const int sft = __clz(static_cast<int>(y0));
    th = y0 << sft;
    tl = 0u;
    rest = 0u;
    L = 31 - sft;
  }
  const int E = L + e;
  if (E < -1022 || E > 1022)   // subnormal, underflowing or overflowing: the general path
    return rn_double_bits(y2, (static_cast<uint64_t>(y1) << 32) | y0, e, neg);
  // 53 bits mh:ml (leading bit at bit 20 of mh), rounded to nearest even
  uint32_t mh = th >> 11, ml = __funnelshift_r(tl, th, 11);
  const uint32_t rbit = (tl >> 10) & 1u;
  const uint32_t sticky = ((tl & 0x3FFu) | rest) != 0u ? 1u : 0u;
  const uint32_t inc = rbit & (sticky | (ml & 1u));
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+r"(ml), "+r"(mh) : "r"(inc));
  // the leading bit (and a carry out of the 53 bits) adds to the exponent field
  const uint32_t hw = (static_cast<uint32_t>(E + 1022) << 20) + mh + (neg ? 0x80000000u : 0u);
  return (static_cast<uint64_t>(hw) << 32) | ml;
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
    int32_t Fv[8];
    if (cb + 7 < P.n && (reinterpret_cast<uintptr_t>(P.F + cb) & 15u) == 0) {
      const int4 f0 = __ldg(reinterpret_cast<const int4*>(P.F + cb)), f1 = __ldg(reinterpret_cast<const int4*>(P.F + cb) + 1);
      Fv[0] = f0.x; Fv[1] = f0.y; Fv[2] = f0.z; Fv[3] = f0.w;
      Fv[4] = f1.x; Fv[5] = f1.y; Fv[6] = f1.z; Fv[7] = f1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) Fv[j] = cb + j < P.n ? __ldg(P.F + cb + j) : 0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint64_t T0 = 0ull, T1 = 0ull, T2 = 0ull, T3 = 0ull;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const uint32_t cl = __byte_perm(j < 4 ? rec[l].x : rec[l].y, 0u, 0x4440u | static_cast<uint32_t>(j & 3));
        T0 += static_cast<uint64_t>(cl) * c_crt.W[N][l][0];
        if (NW > 1) T1 += static_cast<uint64_t>(cl) * c_crt.W[N][l][1];
        if (NW > 2) T2 += static_cast<uint64_t>(cl) * c_crt.W[N][l][2];
        if (NW > 3) T3 += static_cast<uint64_t>(cl) * c_crt.W[N][l][3];
      }
      const int32_t Fj = Fv[j];
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
// columns, so each residue plane streams in order. Four blocks an SM (64
// registers, a few spills on 12 moduli) ran faster than three without spills.
__global__ void __launch_bounds__(256, 4) crt_rebuild_kernel(const SliceProblem P) {
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
