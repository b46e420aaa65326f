// noalloc.cu -- mm_gemm_emu_static: the emulated product without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: code that runs where a device allocation is not allowed or not
// acceptable -- inside a host callback or a custom allocator's own hooks, in a
// latency-critical loop that must never hit cudaMalloc's implicit device-wide
// synchronisation, or in a process that reserved all of its device memory up
// front and forbids further allocation. mm_gemm takes its workspace from the
// handle's memory pool; this entry point needs no handle and instead uses one
// fixed scratch array that the library image carries.
//
// The scratch is a file-scope __device__ array of NOALLOC_SCRATCH_BYTES
// (32 MiB). Every GPU that loads this part of the library holds it until the
// process exits. Host code cannot use the array's name as a device address, so
// the first call on each device (with that device current) looks the address
// up once with cudaGetSymbolAddress and keeps it; do that first call before
// any stream capture. All calls on a device share the one array: calls whose
// GPU work overlaps (different streams, or different host threads without
// ordering) race on it and give wrong results. Each call clears what must
// start at zero (the column maxima and the status word) itself.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
constexpr int MAX_DEVICES = 64;

// The scratch of every call (layout: status word, then the split workspace).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

struct NoAllocDevice {
  std::once_flag once;
  int status = MM_ERR_CUDA;
  unsigned char* scratch = nullptr;   // device address of g_noalloc_scratch
  int sm_count = 0;
  EncodeTiledFn encode = nullptr;
};

NoAllocDevice g_dev[MAX_DEVICES];

void setup_device(NoAllocDevice& d) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    d.status = MM_ERR_CUDA;
    return;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    d.status = MM_ERR_CUDA;
    return;
  }
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    d.status = MM_ERR_CUDA;
    return;
  }
  if (slice_gemm_prepare() != cudaSuccess || fp64_gemm_prepare() != cudaSuccess) {
    d.status = MM_ERR_CUDA;
    return;
  }
  d.scratch = static_cast<unsigned char*>(p);
  d.sm_count = sms;
  d.encode = reinterpret_cast<EncodeTiledFn>(fn);
  d.status = MM_OK;
}

}  // namespace

using namespace mmhost;

int mm_gemm_emu_static(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                       double* C, int64_t ldc, int precision, void* stream) {
  if (precision != MM_FP64_EMU && precision != MM_FP32_EMU) return MM_ERR_INVALID_ARG;
  int rc = validate_problem(m, n, k, A, lda, B, ldb, C, ldc, precision);
  if (rc != MM_OK) return rc;
  if (m == 0 || n == 0) return MM_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MM_ERR_CUDA;
  NoAllocDevice& d = g_dev[dev];
  std::call_once(d.once, setup_device, std::ref(d));
  if (d.status != MM_OK) return d.status;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* err = reinterpret_cast<uint32_t*>(d.scratch);

  if (k == 0 || (precision == MM_FP64_EMU && k <= 4)) {
    // the status word covers this call too (nothing below sets it)
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return cuda_status(e, "status word");
    if (k == 0) return cuda_status(launch_zero_c(C, m, n, ldc, st), "zero C");
    // same rule as mm_gemm: short sums go to the FP64 kernel (no scratch)
    Fp64GemmArgs a{m, n, k, A, lda, B, ldb, C, ldc};
    return cuda_status(launch_fp64_gemm(2, a, st), "fp64 gemm");
  }
  const bool fp64 = precision == MM_FP64_EMU;
  // FP64-accuracy: the automatic slice count, as mm_gemm's default; FP32-accuracy: 3 or 2 slices by k
  const int s = fp64 ? 0 : fp32_slice_count(k);
  SplitLayout L;
  L.plan(m, n, k, s);
  const size_t status_bytes = 256;
  if (status_bytes + L.bytes > NOALLOC_SCRATCH_BYTES) return MM_ERR_BUDGET;   // larger than the fixed scratch

  char* ws = reinterpret_cast<char*>(d.scratch + status_bytes);
  SliceDecision* dec = L.dec(ws);
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess && dec) e = cudaMemsetAsync(dec, 0, sizeof(SliceDecision), st);
  if (e != cudaSuccess) return cuda_status(e, "clear status");
  uint64_t* rowmax = reinterpret_cast<uint64_t*>(ws + L.off_rowmax);
  uint64_t* colmax = reinterpret_cast<uint64_t*>(ws + L.off_colmax);   // zeroed by launch_absmax
  e = launch_absmax(A, m, k, lda, B, n, ldb, rowmax, colmax, st, nullptr, dec, L.part(ws));
  if (e == cudaSuccess)
    e = launch_slice_rows(fp64 ? 0 : 1, A, m, k, lda, rowmax, L.S, L.kp, reinterpret_cast<uint16_t*>(ws + L.off_sa),
                          reinterpret_cast<int32_t*>(ws + L.off_E), err, st, 0, dec);
  if (e == cudaSuccess)
    e = launch_slice_cols(fp64 ? 0 : 1, B, k, n, ldb, colmax, L.S, L.kp, reinterpret_cast<uint16_t*>(ws + L.off_sb),
                          reinterpret_cast<int32_t*>(ws + L.off_F), err, st, dec);
  if (e != cudaSuccess) return cuda_status(e, "split");
  const int bn = 128;   // 128-wide tiles in both modes: one kernel takes every slice count
  CUtensorMap tmA, tmB;
  if (!encode_slices_tmap_with(d.encode, &tmA, ws + L.off_sa, k, m, L.S, L.kp, 128) ||
      !encode_slices_tmap_with(d.encode, &tmB, ws + L.off_sb, k, n, L.S, L.kp, bn))
    return MM_ERR_CUDA;
  SliceGemmArgs a;
  memset(&a, 0, sizeof(a));
  SliceProblem& P = a.single;
  P.m = m; P.n = n; P.k = k;
  P.nkb = static_cast<int>((k + 63) / 64);
  P.s = L.S;
  P.fix_shift = fp64 ? fixed_shift(L.S, k) : 0;
  if (dec) {
    P.s_dev = &dec->s;
    for (int c = SLICE_S_MIN; c <= SLICE_S_MAX; ++c) P.fix_tab[c] = static_cast<int8_t>(fixed_shift(c, k));
    a.s_lo = SLICE_S_MIN;
    a.s_hi = SLICE_S_MAX;
  }
  P.tiles_m = static_cast<int>((m + 127) / 128);
  P.tiles_n = static_cast<int>((n + bn - 1) / bn);
  P.E = reinterpret_cast<const int32_t*>(ws + L.off_E);
  P.F = reinterpret_cast<const int32_t*>(ws + L.off_F);
  P.C = C;
  P.ldc = ldc;
  a.err = err;
  a.timeout_ns = 2000ull * 1000000ull;
  const int grid = std::min(P.tiles_m * P.tiles_n, d.sm_count);
  e = launch_slice_gemm(fp64 ? SLICE_FP64EMU : SLICE_FP32EMU, bn, 1, &tmA, &tmB, a, grid, st);
  if (e == cudaSuccess && dec) {
    // the plain FP64 kernel where the count came out as SLICE_S_PLAIN (no scratch)
    Fp64GemmArgs f{m, n, k, A, lda, B, ldb, C, ldc, &dec->s};
    e = launch_fp64_gemm(2, f, st);
  }
  return cuda_status(e, "slice gemm");
}

int mm_gemm_emu_static_status(void* stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MM_ERR_CUDA;
  NoAllocDevice& d = g_dev[dev];
  std::call_once(d.once, setup_device, std::ref(d));
  if (d.status != MM_OK) return d.status;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* err = reinterpret_cast<uint32_t*>(d.scratch);
  uint32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, err, sizeof(v), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && v != 0u) e = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_status(e, "static status word");
  if (v & MM_DEV_ERR_TIMEOUT_H) return MM_ERR_TIMEOUT;
  if (v & MM_DEV_ERR_NONFINITE_H) return MM_ERR_NONFINITE;
  return MM_OK;
}
