// fp64_gemm.cu -- plain FP64 product C = A*B on the FP64 pipe (the paper's
// computation, Sec. III definition, run on the GPU instead of the Sec. V CPU
// triple loop), plus FP64 peak microbenchmarks.
//
// Block tile 128 x 128, K step 16, 256 threads. A and B tiles are staged in
// shared memory (A transposed to K-major so both operands are read along K),
// double-buffered: the next tile's global loads are in registers while the
// current tile is multiplied.
//   kind 1 (DFMA): each thread owns an 8 x 8 block of C and issues 64 DFMA per k.
//   kind 2 (DMMA): each warp owns a 64 x 32 block of C as 8 x 4 tiles of the
//                  mma.sync.aligned.m8n8k4 f64 shape.
// Global loads are coalesced along the contiguous dimension; 16-byte vectors
// when the operand's leading dimension and base allow it.
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace mmdev {

static constexpr int FT = 128;   // tile M = N
static constexpr int FK = 16;    // tile K
static constexpr int FTHREADS = 256;

struct Fp64Smem {
  double As[2][FK][FT + 2];   // As[k][m]
  double Bs[2][FK][FT + 2];   // Bs[k][n]
};

// Each thread loads 8 A values and 8 B values per K tile.
// A tile 128 x 16: thread -> row t/2, k (t%2)*8 .. +8 (contiguous in A).
// B tile 16 x 128: thread -> k t/16, n (t%16)*8 .. +8 (contiguous in B).
__device__ __forceinline__ void load_tiles(const Fp64GemmArgs& a, int64_t m0, int64_t n0, int64_t k0, bool vecA,
                                           bool vecB, double (&ra)[8], double (&rb)[8]) {
  const int t = threadIdx.x;
  {
    const int r = t >> 1, kc = (t & 1) * 8;
    const int64_t gr = m0 + r, gk = k0 + kc;
    const double* p = a.A + gr * a.lda + gk;
    if (gr < a.m && vecA && gk + 8 <= a.k) {
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        double2 v = __ldg(reinterpret_cast<const double2*>(p + u));
        ra[u] = v.x;
        ra[u + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) ra[u] = (gr < a.m && gk + u < a.k) ? __ldg(p + u) : 0.0;
    }
  }
  {
    const int kr = t >> 4, nc = (t & 15) * 8;
    const int64_t gk = k0 + kr, gn = n0 + nc;
    const double* p = a.B + gk * a.ldb + gn;
    if (gk < a.k && vecB && gn + 8 <= a.n) {
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        double2 v = __ldg(reinterpret_cast<const double2*>(p + u));
        rb[u] = v.x;
        rb[u + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) rb[u] = (gk < a.k && gn + u < a.n) ? __ldg(p + u) : 0.0;
    }
  }
}

__device__ __forceinline__ void store_tiles(Fp64Smem& sm, int buf, const double (&ra)[8], const double (&rb)[8]) {
  const int t = threadIdx.x;
  {
    const int r = t >> 1, kc = (t & 1) * 8;
#pragma unroll
    for (int u = 0; u < 8; ++u) sm.As[buf][kc + u][r] = ra[u];
  }
  {
    const int kr = t >> 4, nc = (t & 15) * 8;
#pragma unroll
    for (int u = 0; u < 8; ++u) sm.Bs[buf][kr][nc + u] = rb[u];
  }
}

// One 128 x 128 tile of C = A*B with its top-left corner at (m0, n0).
template <int KIND>
__device__ __forceinline__ void fp64_tile(const Fp64GemmArgs& a, int64_t m0, int64_t n0, Fp64Smem& sm) {
  const bool vecA = ((a.lda & 1) == 0) && ((reinterpret_cast<uintptr_t>(a.A) & 15u) == 0);
  const bool vecB = ((a.ldb & 1) == 0) && ((reinterpret_cast<uintptr_t>(a.B) & 15u) == 0);
  const int t = threadIdx.x;
  const int nkt = static_cast<int>((a.k + FK - 1) / FK);

  double ra[8], rb[8];
  load_tiles(a, m0, n0, 0, vecA, vecB, ra, rb);
  store_tiles(sm, 0, ra, rb);
  __syncthreads();

  if (KIND == 1) {
    // thread -> rows ty*4 + {0..3} and 64 + ty*4 + {0..3}; cols tx*4 + {0..3} and 64 + tx*4 + {0..3}
    const int tx = t & 15, ty = t >> 4;
    double acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
    for (int kt = 0; kt < nkt; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nkt) load_tiles(a, m0, n0, static_cast<int64_t>(kt + 1) * FK, vecA, vecB, ra, rb);
#pragma unroll
      for (int kk = 0; kk < FK; ++kk) {
        double av[8], bv[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          av[u] = sm.As[buf][kk][ty * 4 + u];
          av[4 + u] = sm.As[buf][kk][64 + ty * 4 + u];
          bv[u] = sm.Bs[buf][kk][tx * 4 + u];
          bv[4 + u] = sm.Bs[buf][kk][64 + tx * 4 + u];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
      if (kt + 1 < nkt) {
        store_tiles(sm, buf ^ 1, ra, rb);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t r = m0 + ((i < 4) ? (ty * 4 + i) : (64 + ty * 4 + i - 4));
      if (r >= a.m) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t c = n0 + ((j < 4) ? (tx * 4 + j) : (64 + tx * 4 + j - 4));
        if (c < a.n) a.C[r * a.ldc + c] = acc[i][j];
      }
    }
  } else {
    // DMMA: warp w -> rows (w & 1) * 64 .. +64, cols (w >> 1) * 32 .. +32
    const int w = t >> 5, lane = t & 31;
    const int wm = (w & 1) * 64, wn = (w >> 1) * 32;
    const int g = lane >> 2, q = lane & 3;
    double acc[8][4][2];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
    for (int kt = 0; kt < nkt; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nkt) load_tiles(a, m0, n0, static_cast<int64_t>(kt + 1) * FK, vecA, vecB, ra, rb);
#pragma unroll
      for (int k4 = 0; k4 < FK; k4 += 4) {
        double af[8], bf[4];
        // A fragment (8 x 4, row): thread holds A[g][q]; B fragment (4 x 8, col): B[q][g]
#pragma unroll
        for (int i = 0; i < 8; ++i) af[i] = sm.As[buf][k4 + q][wm + i * 8 + g];
#pragma unroll
        for (int j = 0; j < 4; ++j) bf[j] = sm.Bs[buf][k4 + q][wn + j * 8 + g];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(acc[i][j][0]), "+d"(acc[i][j][1])
                         : "d"(af[i]), "d"(bf[j]));
      }
      if (kt + 1 < nkt) store_tiles(sm, buf ^ 1, ra, rb);
      __syncthreads();
    }
    // C fragment (8 x 8): thread holds C[g][2q], C[g][2q+1]
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t r = m0 + wm + i * 8 + g;
      if (r >= a.m) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t c = n0 + wn + j * 8 + 2 * q;
        if (c < a.n) a.C[r * a.ldc + c] = acc[i][j][0];
        if (c + 1 < a.n) a.C[r * a.ldc + c + 1] = acc[i][j][1];
      }
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(FTHREADS) fp64_gemm_kernel(const Fp64GemmArgs a) {
  extern __shared__ __align__(16) uint8_t fsm_raw[];
  Fp64Smem& sm = *reinterpret_cast<Fp64Smem*>(fsm_raw);
  fp64_tile<KIND>(a, static_cast<int64_t>(blockIdx.y) * FT, static_cast<int64_t>(blockIdx.x) * FT, sm);
}

// The fallback of an emulated product: a persistent grid over the tiles that
// does nothing unless the product's recorded slice count asks for it, so the
// usual case costs one small grid that returns at once.
template <int KIND>
__global__ void __launch_bounds__(FTHREADS) fp64_fallback_kernel(const Fp64GemmArgs a, int tiles_n, int tiles) {
  if (*a.only_if_plain != SLICE_S_PLAIN) return;
  extern __shared__ __align__(16) uint8_t fsm_raw[];
  Fp64Smem& sm = *reinterpret_cast<Fp64Smem*>(fsm_raw);
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    fp64_tile<KIND>(a, static_cast<int64_t>(t / tiles_n) * FT, static_cast<int64_t>(t % tiles_n) * FT, sm);
    __syncthreads();
  }
}

// Grouped: a persistent grid walks the tile list of many products; the tile
// count is read from device memory so a captured graph can be replayed with
// new work.
// With count_dev set, the problems carry fallback guards: a block first looks
// at every problem's guard and returns at once when no problem asks for the
// plain kernel (the usual case), else runs the tiles of those that do.
template <int KIND>
__global__ void __launch_bounds__(FTHREADS) fp64_grouped_kernel(const Fp64GemmArgs* __restrict__ probs,
                                                                const TileRef* __restrict__ tiles,
                                                                const int* __restrict__ ntiles_dev,
                                                                const int* __restrict__ count_dev) {
  extern __shared__ __align__(16) uint8_t fsm_raw[];
  Fp64Smem& sm = *reinterpret_cast<Fp64Smem*>(fsm_raw);
  if (count_dev != nullptr) {
    const int count = *count_dev;
    int any = 0;
    for (int p = threadIdx.x; p < count; p += blockDim.x) {
      const int32_t* g = probs[p].only_if_plain;
      any |= (g != nullptr && *g == SLICE_S_PLAIN) ? 1 : 0;
    }
    if (!__syncthreads_or(any)) return;
  }
  const int nt = *ntiles_dev;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const TileRef r = tiles[t];
    const Fp64GemmArgs a = probs[r.prob];
    if (a.only_if_plain != nullptr && *a.only_if_plain != SLICE_S_PLAIN) continue;   // uniform over the block
    fp64_tile<KIND>(a, static_cast<int64_t>(r.tm) * FT, static_cast<int64_t>(r.tn) * FT, sm);
    __syncthreads();
  }
}

__global__ void zero_c_kernel(double* C, int64_t m, int64_t n, int64_t ldc) {
  int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t total = m * n;
  for (; idx < total; idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t r = idx / n;
    C[r * ldc + (idx - r * n)] = 0.0;
  }
}

// ------------------------------------------------------------------- peaks
// DFMA: 8 independent FMA chains per thread.
__global__ void peak_dfma_kernel(double* sink, int iters) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-9 + i;
  const double a = 0.999999, b = 1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 12345.678) sink[threadIdx.x] = s;
}

// DMMA: 4 independent m8n8k4 accumulators per warp.
__global__ void peak_dmma_kernel(double* sink, int iters) {
  double c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i][0] = c[i][1] = 0.0;
  const double av = 1e-3 * (threadIdx.x & 31), bv = 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[i][0]), "+d"(c[i][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
  if (s == 12345.678) sink[threadIdx.x] = s;
}

}  // namespace mmdev

using namespace mmdev;

cudaError_t fp64_gemm_prepare() {
  const int smem = static_cast<int>(sizeof(Fp64Smem));
  cudaError_t e = cudaFuncSetAttribute(fp64_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fp64_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fp64_grouped_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fp64_grouped_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fp64_fallback_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fp64_fallback_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

int fp64_tile_size() { return FT; }

cudaError_t launch_fp64_grouped(int kind, const Fp64GemmArgs* probs, const TileRef* tiles, const int* ntiles_dev,
                                int grid, cudaStream_t st, const int* count_dev) {
  const int smem = static_cast<int>(sizeof(Fp64Smem));
  if (kind == 1)
    fp64_grouped_kernel<1><<<grid, FTHREADS, smem, st>>>(probs, tiles, ntiles_dev, count_dev);
  else
    fp64_grouped_kernel<2><<<grid, FTHREADS, smem, st>>>(probs, tiles, ntiles_dev, count_dev);
  return cudaGetLastError();
}

cudaError_t launch_fp64_gemm(int kind, const Fp64GemmArgs& a, cudaStream_t st) {
  if (a.m <= 0 || a.n <= 0) return cudaSuccess;
  if (a.k <= 0) return launch_zero_c(a.C, a.m, a.n, a.ldc, st);
  const int smem = static_cast<int>(sizeof(Fp64Smem));
  if (a.only_if_plain != nullptr) {
    const int64_t tn = (a.n + FT - 1) / FT, tiles = tn * ((a.m + FT - 1) / FT);
    if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorInvalidValue;
    const unsigned grid = static_cast<unsigned>(tiles < 2 * sms ? tiles : 2 * sms);
    if (kind == 1)
      fp64_fallback_kernel<1><<<grid, FTHREADS, smem, st>>>(a, static_cast<int>(tn), static_cast<int>(tiles));
    else
      fp64_fallback_kernel<2><<<grid, FTHREADS, smem, st>>>(a, static_cast<int>(tn), static_cast<int>(tiles));
    return cudaGetLastError();
  }
  dim3 grid(static_cast<unsigned>((a.n + FT - 1) / FT), static_cast<unsigned>((a.m + FT - 1) / FT));
  if (kind == 1)
    fp64_gemm_kernel<1><<<grid, FTHREADS, smem, st>>>(a);
  else
    fp64_gemm_kernel<2><<<grid, FTHREADS, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_zero_c(double* C, int64_t m, int64_t n, int64_t ldc, cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  int64_t total = m * n;
  unsigned blocks = static_cast<unsigned>(total / 256 + 1 < 152 * 16 ? total / 256 + 1 : 152 * 16);
  zero_c_kernel<<<blocks, 256, 0, st>>>(C, m, n, ldc);
  return cudaGetLastError();
}

cudaError_t launch_peak_fp64(int kind, double* sink, int iters, int blocks, cudaStream_t st) {
  if (kind == 1)
    peak_dfma_kernel<<<blocks, 256, 0, st>>>(sink, iters);
  else
    peak_dmma_kernel<<<blocks, 256, 0, st>>>(sink, iters);
  return cudaGetLastError();
}
