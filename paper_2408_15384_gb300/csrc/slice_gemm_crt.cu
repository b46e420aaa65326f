// slice_gemm_crt.cu -- instances of the slice GEMM for the modular form of the
// FP64-accuracy product (SLICE_CRT: one residue product a modulus, the
// Chinese-remainder rebuild in the epilogue) and the rebuild constants.
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
