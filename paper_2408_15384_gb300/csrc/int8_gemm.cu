// int8_gemm.cu -- FP64-accuracy slice products on the legacy integer tensor
// path (mma.sync m16n8k32, signed bytes, int32 accumulation), the INT8 form
// of the integer-slice method (Ootomo, Ozaki, Yokota 2024).
//
// The digits come from the splitting kernels' INT8 form: scale exponent
// E = floor(log2 max) + 3, digits in [-128, 127] as signed bytes, planes
// [s][rows][kp] (B transposed, K contiguous). Each block computes a 128 x 64
// tile of C with 8 warps (4 along M x 2 along N, 32 x 32 outputs a warp):
// the levels d = s+1 .. 2 one after the other, every K block of 32 and every
// pair (p, d-p) of the level a pipeline step that brings the two 128 x 32 and
// 64 x 32 byte tiles into shared memory with cp.async (bytes past k or past
// the last row/column arrive as zeros), then 8 mma.sync per warp into int32
// level sums. Products of two digits are at most 2^14 in magnitude, so an
// int32 sum is exact for up to 2^17 products; a level is folded into the
// int64 total every SEG_KB K blocks and at its end, with the same fixed point
// and rounding as the tcgen05 path (levels below 2^shift summed exactly and
// rounded once, half up). After level 2 each output is converted to double
// once and scaled by 2^(E_i + F_j - 8(s+1) + shift).
//
// On GB300 the 8-bit integer tensor rate is far below the bfloat16 tcgen05
// rate: this path exists to measure that against the default bfloat16 slices
// (mm_set_option MM_OPT_INT8_SLICES) and for its bit-exact level products.
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "slice_gemm_kernel.cuh"   // scale_pow2

namespace mmdev {

namespace {

constexpr int I8_BM = 128, I8_BN = 64, I8_BK = 32, I8_THREADS = 256, I8_STAGES = 4;
constexpr int I8_LD = 48;        // bytes per tile row in shared memory: 32 data + 16 pad
                                 // (rows 12 banks apart: conflict-free 32-bit fragment loads)
constexpr int SEG_KB = 512;      // K blocks per int32 segment: 512 * 32 * 7 pairs * 2^14 < 2^31

struct I8Smem {
  uint8_t a[I8_STAGES][I8_BM * I8_LD];
  uint8_t b[I8_STAGES][I8_BN * I8_LD];
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mma_s8(int32_t (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Position in the step sequence: level d, K block kb, pair index pi (pair
// p = p_lo(d) + pi).
struct StepPos {
  int d, kb, pi;
};

__device__ __forceinline__ int pair_lo(int d, int s) { return d - s > 1 ? d - s : 1; }
__device__ __forceinline__ int pair_count(int d, int s) {
  const int hi = d - 1 < s ? d - 1 : s;
  return hi - pair_lo(d, s) + 1;
}

__device__ __forceinline__ void advance(StepPos& p, int s, int nkb) {
  if (++p.pi < pair_count(p.d, s)) return;
  p.pi = 0;
  if (++p.kb < nkb) return;
  p.kb = 0;
  --p.d;
}

// One step's byte tiles into stage `stage`: A plane p-1 rows [row0, row0+128),
// B plane d-p-1 rows (columns of B) [col0, col0+64), K bytes [32 kb, 32 kb + 32).
__device__ __forceinline__ void load_step(I8Smem& sm, int stage, const Int8GemmArgs& a, int s, const StepPos& p,
                                          int64_t row0, int64_t col0) {
  const int pa = pair_lo(p.d, s) + p.pi;
  const int pb = p.d - pa;
  const int64_t k0 = static_cast<int64_t>(p.kb) * I8_BK;
  const int t = static_cast<int>(threadIdx.x);
  {
    const int r = t >> 1, half = t & 1;
    const int64_t gr = row0 + r, gk = k0 + 16 * half;
    const int8_t* src = a.A + static_cast<int64_t>(pa - 1) * a.plane_a;
    int bytes = 0;
    if (gr < a.m && gk < a.k) {
      src += gr * a.kp + gk;
      bytes = static_cast<int>(a.k - gk < 16 ? a.k - gk : 16);
    }
    cp_async16(&sm.a[stage][r * I8_LD + 16 * half], src, bytes);
  }
  if (t < 2 * I8_BN) {
    const int r = t >> 1, half = t & 1;
    const int64_t gc = col0 + r, gk = k0 + 16 * half;
    const int8_t* src = a.B + static_cast<int64_t>(pb - 1) * a.plane_b;
    int bytes = 0;
    if (gc < a.n && gk < a.k) {
      src += gc * a.kp + gk;
      bytes = static_cast<int>(a.k - gk < 16 ? a.k - gk : 16);
    }
    cp_async16(&sm.b[stage][r * I8_LD + 16 * half], src, bytes);
  }
}

__global__ void __launch_bounds__(I8_THREADS) int8_slice_gemm_kernel(const Int8GemmArgs a) {
  const int s = a.s_dev != nullptr ? *a.s_dev : a.s;
  if (s < SLICE_S_MIN || s > SLICE_S_MAX) return;   // the plain FP64 fallback handles it
  int fix = a.fix_shift;
  if (a.s_dev != nullptr) {
#pragma unroll
    for (int c = SLICE_S_MIN; c <= SLICE_S_MAX; ++c)
      if (c == s) fix = a.fix_tab[c];   // constant indices: the parameter block stays in place
  }
  __shared__ __align__(16) I8Smem sm;
  const int64_t row0 = static_cast<int64_t>(blockIdx.y) * I8_BM, col0 = static_cast<int64_t>(blockIdx.x) * I8_BN;
  const int warp = static_cast<int>(threadIdx.x >> 5), lane = static_cast<int>(threadIdx.x & 31);
  const int wm = warp & 3, wn = warp >> 2;
  const int g = lane >> 2, t4 = lane & 3;
  const int nkb = static_cast<int>((a.k + I8_BK - 1) / I8_BK);
  int total = 0;
  for (int d = s + 1; d >= 2; --d) total += pair_count(d, s) * nkb;

  int32_t acc[2][4][4];
  int64_t X[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        acc[i][j][v] = 0;
        X[i][j][v] = 0;
      }

  // the first STAGES-1 steps in flight
  StepPos ld{s + 1, 0, 0};
  for (int i = 0; i < I8_STAGES - 1; ++i) {
    if (i < total) {
      load_step(sm, i, a, s, ld, row0, col0);
      advance(ld, s, nkb);
    }
    cp_async_commit();
  }
  StepPos cur{s + 1, 0, 0};
  int seg_kb = 0;   // K blocks summed into acc since its last fold
  for (int it = 0; it < total; ++it) {
    cp_async_wait<I8_STAGES - 2>();
    __syncthreads();
    // refill the stage used one step ago
    if (it + I8_STAGES - 1 < total) {
      load_step(sm, (it + I8_STAGES - 1) % I8_STAGES, a, s, ld, row0, col0);
      advance(ld, s, nkb);
    }
    cp_async_commit();
    const uint8_t* sa = sm.a[it % I8_STAGES];
    const uint8_t* sb = sm.b[it % I8_STAGES];
    uint32_t af[2][4], bf[4][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = wm * 32 + i * 16 + g;
      af[i][0] = *reinterpret_cast<const uint32_t*>(sa + r * I8_LD + 4 * t4);
      af[i][1] = *reinterpret_cast<const uint32_t*>(sa + (r + 8) * I8_LD + 4 * t4);
      af[i][2] = *reinterpret_cast<const uint32_t*>(sa + r * I8_LD + 16 + 4 * t4);
      af[i][3] = *reinterpret_cast<const uint32_t*>(sa + (r + 8) * I8_LD + 16 + 4 * t4);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = wn * 32 + j * 8 + g;
      bf[j][0] = *reinterpret_cast<const uint32_t*>(sb + c * I8_LD + 4 * t4);
      bf[j][1] = *reinterpret_cast<const uint32_t*>(sb + c * I8_LD + 16 + 4 * t4);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) mma_s8(acc[i][j], af[i], bf[j]);

    // end of a K block's pairs: count it; fold at a segment's or the level's end
    const bool kb_end = cur.pi == pair_count(cur.d, s) - 1;
    const bool level_end = kb_end && cur.kb == nkb - 1;
    if (kb_end) ++seg_kb;
    if (level_end || (kb_end && seg_kb == SEG_KB)) {
      const int d = cur.d;
      const int w = 8 * (s + 1 - d);
      const bool raw = w < fix;
      const int lsh = a.levels != nullptr ? 0 : (raw ? w : w - fix);
      const bool rnd = a.levels == nullptr && level_end && raw && (d == 2 || w + 8 >= fix);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            if (a.levels != nullptr) {
              const int64_t r = row0 + wm * 32 + i * 16 + g + ((v & 2) ? 8 : 0);
              const int64_t c = col0 + wn * 32 + j * 8 + 2 * t4 + (v & 1);
              if (r < a.m && c < a.n)
                a.levels[(static_cast<int64_t>(d - 2) * a.m + r) * a.n + c] += static_cast<int64_t>(acc[i][j][v]);
            } else {
              int64_t x = X[i][j][v] + (static_cast<int64_t>(acc[i][j][v]) << lsh);
              if (rnd) x = (x + (1ll << (fix - 1))) >> fix;
              X[i][j][v] = x;
            }
            acc[i][j][v] = 0;
          }
      seg_kb = 0;
    }
    advance(cur, s, nkb);
  }
  cp_async_wait<0>();
  if (a.levels != nullptr) return;

  // C = X * 2^(E_i + F_j - 8(s+1) + shift), one conversion and scaling per output
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int v2 = 0; v2 < 2; ++v2) {
      const int64_t r = row0 + wm * 32 + i * 16 + g + 8 * v2;
      if (r >= a.m) continue;
      const int32_t Ei = a.E[r];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int v1 = 0; v1 < 2; ++v1) {
          const int64_t c = col0 + wn * 32 + j * 8 + 2 * t4 + v1;
          if (c >= a.n) continue;
          const int32_t Fj = __ldg(a.F + c);
          double o;
          if (Ei == EXP_NONFINITE || Fj == EXP_NONFINITE)
            o = __longlong_as_double(0x7FF8000000000000ll);
          else
            o = scale_pow2(__ll2double_rn(X[i][j][2 * v2 + v1]), Ei + Fj - 8 * (s + 1) + fix);
          a.C[r * a.ldc + c] = o;
        }
    }
}

}  // namespace

}  // namespace mmdev

cudaError_t launch_int8_slice_gemm(const Int8GemmArgs& a, cudaStream_t st) {
  if (a.m <= 0 || a.n <= 0) return cudaSuccess;
  const int64_t gx = (a.n + mmdev::I8_BN - 1) / mmdev::I8_BN, gy = (a.m + mmdev::I8_BM - 1) / mmdev::I8_BM;
  if (gx > 0x7fffffff || gy > 65535) return cudaErrorInvalidValue;
  mmdev::int8_slice_gemm_kernel<<<dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy)), mmdev::I8_THREADS, 0,
                                  st>>>(a);
  return cudaGetLastError();
}
