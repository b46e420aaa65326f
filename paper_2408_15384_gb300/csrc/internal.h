// internal.h -- the handle and host helpers shared by the C ABI files.
#pragma once
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/mm.h"
#include "kernels.cuh"

// host copies of the device error bits (ptx.cuh)
#define MM_DEV_ERR_TIMEOUT_H 1u
#define MM_DEV_ERR_NONFINITE_H 2u

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

namespace mmhost {
struct GroupedCache;
struct ServeEngine;
struct TuneTable;

// Launch configuration of a product: 0 in a field means "automatic".
struct TileCfg {
  int bn = 0;     // emulated modes: output tile width (128, 192, 240, 256)
  int cg = 0;     // emulated modes: CTAs per tile (1, or 2 = CTA pair)
  int kern = 0;   // plain FP64: 1 = DFMA tiles, 2 = DMMA tiles
};
}

struct mm_handle_s {
  int device = 0;
  size_t budget = 0;
  int sm_count = 148;
  std::chrono::steady_clock::time_point t0;
  EncodeTiledFn encode = nullptr;
  cudaMemPool_t pool = nullptr;
  // device error words (MM_DEV_ERR_* bits), one per stream the handle has
  // seen (err_word); slot 0 is shared by streams beyond the table's size
  uint32_t* d_err = nullptr;
  std::mutex err_mu;
  std::unordered_map<cudaStream_t, int> err_slot;
  int err_next = 1;
  std::atomic<size_t> ws_in_use{0};          // workspace bytes held (budget accounting)
  std::atomic<uint64_t> launches{0};         // kernels launched by the library

  // options
  int opt_slices = 0;        // 0: automatic slice count (decided on the device from the operands)
  int64_t opt_timeout_ms = 2000;
  bool opt_autotune = false;
  int opt_serve_max_batch = 32;
  int opt_serve_streams = 4;
  int opt_fp64_kernel = 0;
  int opt_fp32_bn = 0;
  bool opt_profile = false;
  int opt_cta_pair = 0;
  int opt_tile_n = 0;        // FP64-accuracy tile width (0 = automatic, 128, 192, 240, 256)
  bool opt_int8 = false;     // FP64-accuracy single products on INT8-form digits (mma.sync s8)
  int opt_fp64_scheme = 0;   // 0: modular form for products of m n k >= CRT_MIN_WORK where it fits; 1: digits
                             // only; 2: modular form wherever it fits
  int max_pairs_fp32 = 0, max_pairs_fp64 = 0, max_pairs_crt = 0;   // co-resident CTA pairs of the pair kernels
  int max_clusters4_fp32 = 0, max_clusters4_fp64 = 0;   // co-resident clusters of two pairs (cg = 4)

  // profiling: (start, end) event pairs per kernel class, drained by mm_profile_read
  std::mutex prof_mu;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending[4];
  double prof_ms[4] = {0, 0, 0, 0};
  uint64_t prof_count[4] = {0, 0, 0, 0};

  std::mutex grouped_mu;
  mmhost::GroupedCache* grouped = nullptr;
  std::mutex serve_mu;
  mmhost::ServeEngine* serve = nullptr;
  mmhost::TuneTable* tune = nullptr;         // autotuned launch configurations (tune.cu)
};

namespace mmhost {

void logf(int level, const char* fmt, ...);
double now_us(const mm_handle_s* h);
int cuda_status(cudaError_t e, const char* what);
size_t align_up(size_t x, size_t a);
int ws_alloc(mm_handle_s* h, size_t bytes, cudaStream_t st, void** out);
void ws_free(mm_handle_s* h, void* p, size_t bytes, cudaStream_t st);
int validate_problem(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                     const double* C, int64_t ldc, int precision);
// error words: MM_ERR_SLOTS per handle
constexpr int MM_ERR_SLOTS = 256;
uint32_t* err_word(mm_handle_s* h, cudaStream_t st);
int fixed_shift(int s, int64_t k);
// 3-D map (k, rows, slice) over bfloat16 slices; planes of plane_rows rows
// (0: rows), so a panel of a larger matrix's slices can be mapped.
bool encode_slices_tmap(mm_handle_s* h, CUtensorMap* tm, const void* base, int64_t k, int64_t rows, int S, int64_t kp,
                        int box_rows, int64_t plane_rows = 0);
// the same with an explicit encoder (callers without a handle)
bool encode_slices_tmap_with(EncodeTiledFn encode, CUtensorMap* tm, const void* base, int64_t k, int64_t rows, int S,
                             int64_t kp, int box_rows, int64_t plane_rows = 0);
void count_launch(mm_handle_s* h, uint64_t n);
int fp64_kind(mm_handle_s* h);
int gemm_device(mm_handle_s* h, int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                int64_t ldb, double* C, int64_t ldc, int precision, cudaStream_t st);
struct SplitLayout;
// The slice count of an emulated product: 3 (FP32-accuracy), the override or
// the handle's fixed count, else 0 = automatic (decided on the device).
int emu_slices(mm_handle_s* h, int precision, int64_t k, int s_override);
// Slice planes a workspace holds for slice count s (0: automatic -> 7).
inline int emu_planes(int s) { return s > 0 ? s : SLICE_S_MAX; }
int emu_gemm_rows(mm_handle_s* h, int precision, const SplitLayout& L, char* ws, int s, int64_t r0, int64_t mr,
                  double* C, int64_t ldc, int64_t* levels, const TileCfg& cfg, cudaStream_t st);
// one product with an explicit launch configuration (no tuning)
int gemm_with_cfg(mm_handle_s* h, int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                  int64_t ldb, double* C, int64_t ldc, int precision, const TileCfg& cfg, cudaStream_t st);
// Reads and clears the error word of stream st (synchronous copy).
int read_and_clear_err(mm_handle_s* h, cudaStream_t st);

// Brackets one launch with events when profiling is on.
struct ProfScope {
  mm_handle_s* h;
  int kernel;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ProfScope(mm_handle_s* h_, int kernel_, cudaStream_t st_);
  ~ProfScope();
};

struct DeviceGuard {
  int prev = 0, target = 0;
  explicit DeviceGuard(int dev);
  ~DeviceGuard();
};

// Workspace layout of one emulated product. s = 0: automatic slice count
// (7 planes, plus the decision record and the column partial sums); crt: the
// modular form allowed (CRT_N_MAX planes, and the products' residue bytes,
// CRT_N_MAX planes of m rows of ldr bytes).
struct SplitLayout {
  int64_t m = 0, n = 0, k = 0, kp = 0, ldr = 0;
  int S = 0;
  bool autos = false, crt = false;
  size_t off_rowmax = 0, off_colmax = 0, off_E = 0, off_F = 0, off_sa = 0, off_sb = 0, off_dec = 0, off_part = 0,
         off_res = 0, bytes = 0;
  int elem = 2;   // bytes per slice entry: 2 (bfloat16), 1 (INT8-form digits)
  void plan(int64_t m_, int64_t n_, int64_t k_, int s, int elem_bytes = 2, bool crt_ = false);
  SliceDecision* dec(char* ws) const { return autos ? reinterpret_cast<SliceDecision*>(ws + off_dec) : nullptr; }
  uint2* part(char* ws) const { return autos ? reinterpret_cast<uint2*>(ws + off_part) : nullptr; }
};

// mode: a launch_slice_rows mode (3 for a layout with crt)
int run_split(mm_handle_s* h, int mode, const SplitLayout& L, char* ws, const double* A, int64_t lda,
              const double* B, int64_t ldb, cudaStream_t st);
// Whether an FP64-accuracy product of m x k by k x n may take the modular form
// (automatic slice count; the scheme option; below CRT_MIN_WORK the digit
// form is faster: the modular form's longer split and its rebuild, which a
// product with few tiles a CTA cannot overlap with tensor-core work, cost more
// than its fewer products save).
constexpr double CRT_MIN_WORK = 8589934592.0;   // m n k >= 2^33 (2048^3)
bool crt_allowed(const mm_handle_s* h, int precision, int s, int64_t m, int64_t n, int64_t k);

// tune.cu: the autotuner. Keys are shape buckets (ceil(log2) of the single
// product's m, n, k; of a group's problem count and mean dimension).
enum { TUNE_SINGLE = 0, TUNE_GROUPED = 1 };
bool tile_options_set(const mm_handle_s* h);
TileCfg default_cfg(const mm_handle_s* h, int precision, int64_t m, int64_t n, int s);
TileCfg grouped_default_cfg(const mm_handle_s* h, int precision, int count, const mm_problem* probs);
void tune_key_single(int precision, int64_t m, int64_t n, int64_t k, int key[5]);
void tune_key_grouped(int precision, int count, const mm_problem* probs, int key[5]);
bool tune_lookup(mm_handle_s* h, const int key[5], TileCfg* out);
std::vector<TileCfg> tune_candidates(const mm_handle_s* h, int kind, int precision, int64_t m, int64_t n);
// Times every candidate (one warm-up and two timed runs of run(cfg) on st,
// CUDA events), stores the fastest under key and returns it in *best. The
// runs write the caller's outputs; the caller runs the chosen configuration
// once more afterwards. Returns MM_OK, or the first CUDA error.
int tune_pick(mm_handle_s* h, const int key[5], const std::vector<TileCfg>& cands, cudaStream_t st,
              int (*run)(void* ctx, const TileCfg& cfg), void* ctx, TileCfg* best);
bool stream_capturing(cudaStream_t st);
void tune_init(mm_handle_s* h);
void tune_release(mm_handle_s* h);

// grouped.cu / serve.cu
void grouped_release(mm_handle_s* h);
int grouped_run(mm_handle_s* h, int count, const mm_problem* probs, int precision, cudaStream_t st);
// direct (graph-free) grouped launch with the pool's workspace, as the
// serving engine issues it; cfg as from grouped_cfg
TileCfg grouped_cfg(mm_handle_s* h, int count, const mm_problem* probs, int precision);
size_t grouped_direct_bytes(mm_handle_s* h, int count, const mm_problem* probs, int precision, const TileCfg& cfg,
                            size_t* host_bytes);
// Per-problem error reporting of a direct grouped launch: the launch's word
// (header word 3: timeouts) and one word per emulated problem (non-finite
// input, at off_perr) are copied back into the host blob's first `bytes`
// bytes on the stream after the launch; main_idx[i] is the problem of word i.
struct GroupedErrReport {
  size_t bytes = 0, off_perr = 0;
  std::vector<int> main_idx;
};
int grouped_direct(mm_handle_s* h, int count, const mm_problem* probs, int precision, const TileCfg& cfg,
                   void* host_blob, size_t host_cap, cudaStream_t st, GroupedErrReport* rep = nullptr);
void serve_shutdown(mm_handle_s* h);

}  // namespace mmhost
