// grouped.cu -- mm_gemm_grouped: many independent products in one persistent
// launch per stage, replayed from a CUDA graph.
//
// A call writes a descriptor blob (problem records, per-problem block offsets
// of the grouped split kernels, tensor maps, a cost-sorted tile list) into a
// pinned staging buffer and launches a graph made of: one memcpy of the blob
// to the device, one memset of the column-maximum region, the grouped split
// kernels and the grouped slice GEMM (emulated modes), or the grouped FP64
// kernel (plain mode). Kernel arguments point into the device blob and read
// the tile count from it, so the graph is captured once per
// (count, precision, stream) and replayed with new descriptors; it is captured
// again only when a call needs more descriptor or workspace room than the
// captured one. Two graph slots alternate so the host can stage a call while
// the previous one still runs; each slot's staging buffer is reused only after
// its last launch finished (event).
//
// Problems the emulated kernels do not take (k == 0, or k <= 4 in
// FP64-accuracy) run through the single-product path, so every problem's
// result equals mm_gemm on it.
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"

namespace mmhost {

struct GroupedSlot {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* stage = nullptr;       // pinned host staging of the blob
  void* dblob = nullptr;       // device blob
  size_t blob_cap = 0;
  void* ws = nullptr;          // device workspace (emulated modes)
  size_t ws_cap = 0;
  size_t colmax_cap = 0;       // bytes of the column-maximum region at ws + 0
  int tiles_cap = 0;
  cudaEvent_t done = nullptr;
  bool launched = false;
};

struct GroupedKey {
  int count, precision;
  cudaStream_t stream;
  bool operator<(const GroupedKey& o) const {
    return std::tie(count, precision, stream) < std::tie(o.count, o.precision, o.stream);
  }
};

struct GroupedEntry {
  GroupedSlot slot[2];
  int next = 0;
};

struct GroupedCache {
  std::map<GroupedKey, GroupedEntry> entries;
};

static void release_slot(mm_handle_s* h, GroupedSlot& s) {
  if (s.done) cudaEventSynchronize(s.done);
  if (s.exec) cudaGraphExecDestroy(s.exec);
  if (s.graph) cudaGraphDestroy(s.graph);
  if (s.stage) cudaFreeHost(s.stage);
  if (s.dblob) { cudaFree(s.dblob); h->ws_in_use.fetch_sub(s.blob_cap); }
  if (s.ws) { cudaFree(s.ws); h->ws_in_use.fetch_sub(s.ws_cap); }
  if (s.done) cudaEventDestroy(s.done);
  s = GroupedSlot();
}

void grouped_release(mm_handle_s* h) {
  std::lock_guard<std::mutex> lk(h->grouped_mu);
  if (!h->grouped) return;
  for (auto& kv : h->grouped->entries)
    for (auto& s : kv.second.slot) release_slot(h, s);
  delete h->grouped;
  h->grouped = nullptr;
}

static int reserve(mm_handle_s* h, size_t bytes, void** p) {
  *p = nullptr;
  if (bytes == 0) return MM_OK;
  if (h->ws_in_use.fetch_add(bytes) + bytes > h->budget) {
    h->ws_in_use.fetch_sub(bytes);
    return MM_ERR_BUDGET;
  }
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->ws_in_use.fetch_sub(bytes);
    return MM_ERR_BUDGET;
  }
  return MM_OK;
}

// ------------------------------------------------------------ blob layouts
struct EmuLayout {
  size_t off_hdr = 0, off_split = 0, off_off = 0, off_sp = 0, off_tmap = 0, off_tiles = 0, bytes = 0;
  void plan(int count, int tiles) {
    size_t o = 0;
    off_hdr = o; o = align_up(o + 64, 64);
    off_split = o; o = align_up(o + sizeof(GroupedSplit) * count, 64);
    off_off = o; o = align_up(o + sizeof(int64_t) * 4 * (count + 1), 64);
    off_sp = o; o = align_up(o + sizeof(SliceProblem) * count, 64);
    off_tmap = o; o = align_up(o + sizeof(CUtensorMap) * 2 * count, 64);
    off_tiles = o; o = align_up(o + sizeof(TileRef) * std::max(tiles, 1), 64);
    bytes = o;
  }
};

struct Fp64Layout {
  size_t off_hdr = 0, off_args = 0, off_tiles = 0, bytes = 0;
  void plan(int count, int tiles) {
    size_t o = 0;
    off_hdr = o; o = align_up(o + 64, 64);
    off_args = o; o = align_up(o + sizeof(Fp64GemmArgs) * count, 64);
    off_tiles = o; o = align_up(o + sizeof(TileRef) * std::max(tiles, 1), 64);
    bytes = o;
  }
};

// Per-problem workspace of the emulated modes inside the group workspace.
struct ProbWs {
  size_t rowmax, colmax, E, F, sa, sb;
};

struct TileCost {
  int64_t cost;
  int prob, idx;
  TileRef ref;
};

static void sort_tiles(std::vector<TileCost>& v) {
  std::stable_sort(v.begin(), v.end(), [](const TileCost& a, const TileCost& b) {
    if (a.cost != b.cost) return a.cost > b.cost;
    if (a.prob != b.prob) return a.prob < b.prob;
    return a.idx < b.idx;
  });
}

// ------------------------------------------------------------- emulated
static int grouped_emulated(mm_handle_s* h, GroupedEntry& ent, const std::vector<int>& idx, const mm_problem* probs,
                            int precision, cudaStream_t st) {
  const bool fp64 = precision == MM_FP64_EMU;
  const int count = static_cast<int>(idx.size());
  const int bn = 128;
  // ---- workspace plan and tile list
  std::vector<ProbWs> pw(count);
  std::vector<int> S(count), sl(count);
  std::vector<int64_t> kp(count);
  size_t colmax_bytes = 0;
  for (int i = 0; i < count; ++i) colmax_bytes += align_up(8 * static_cast<size_t>(probs[idx[i]].n), 256);
  size_t o = 0;   // per-problem regions follow the column-maximum region (offset colmax_cap)
  std::vector<TileCost> tiles;
  size_t cm = 0;
  for (int i = 0; i < count; ++i) {
    const mm_problem& p = probs[idx[i]];
    sl[i] = fp64 ? (h->opt_slices > 0 ? h->opt_slices : slices_for_k(p.k)) : 3;
    S[i] = sl[i];
    kp[i] = static_cast<int64_t>(align_up(static_cast<size_t>(p.k), 8));
    pw[i].colmax = cm; cm += align_up(8 * static_cast<size_t>(p.n), 256);
    pw[i].rowmax = o; o = align_up(o + 8 * static_cast<size_t>(p.m), 256);
    pw[i].E = o; o = align_up(o + 4 * static_cast<size_t>(p.m), 256);
    pw[i].F = o; o = align_up(o + 4 * static_cast<size_t>(p.n), 256);
    pw[i].sa = o; o = align_up(o + 2 * static_cast<size_t>(S[i]) * p.m * kp[i], 1024);
    pw[i].sb = o; o = align_up(o + 2 * static_cast<size_t>(S[i]) * p.n * kp[i], 1024);
    const int tm = static_cast<int>((p.m + 127) / 128), tn = static_cast<int>((p.n + bn - 1) / bn);
    const int64_t nkb = (p.k + 63) / 64;
    const int64_t pairs = fp64 ? static_cast<int64_t>(sl[i]) * (sl[i] + 1) / 2 : 6;
    for (int a = 0; a < tm; ++a)
      for (int b = 0; b < tn; ++b)
        tiles.push_back({nkb * pairs, i, a * tn + b, TileRef{i, static_cast<int16_t>(a), static_cast<int16_t>(b)}});
  }
  const size_t ws_bytes = o;
  sort_tiles(tiles);
  const int ntiles = static_cast<int>(tiles.size());
  EmuLayout L;
  GroupedSlot& slot = ent.slot[ent.next];
  // ---- (re)capture when the slot is too small
  const bool fits = slot.exec && slot.ws_cap - slot.colmax_cap >= ws_bytes && slot.colmax_cap >= colmax_bytes &&
                    slot.tiles_cap >= ntiles;
  if (slot.launched) cudaEventSynchronize(slot.done);
  if (!fits) {
    release_slot(h, slot);
    const int tiles_cap = std::max(ntiles, 1) * 5 / 4 + 64;
    L.plan(count, tiles_cap);
    slot.blob_cap = L.bytes;
    slot.tiles_cap = tiles_cap;
    slot.ws_cap = ws_bytes + ws_bytes / 4 + (1 << 20);
    slot.colmax_cap = align_up(colmax_bytes + colmax_bytes / 4 + 4096, 1024);
    int rc;
    if ((rc = reserve(h, slot.blob_cap, &slot.dblob)) != MM_OK) { slot = GroupedSlot(); return rc; }
    if ((rc = reserve(h, slot.ws_cap + slot.colmax_cap, &slot.ws)) != MM_OK) {
      cudaFree(slot.dblob); h->ws_in_use.fetch_sub(slot.blob_cap); slot = GroupedSlot(); return rc;
    }
    slot.ws_cap += slot.colmax_cap;
    if (cudaMallocHost(&slot.stage, slot.blob_cap) != cudaSuccess || cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming) != cudaSuccess) {
      release_slot(h, slot);
      return MM_ERR_CUDA;
    }
    // capture on a private stream
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { release_slot(h, slot); return MM_ERR_CUDA; }
    char* db = static_cast<char*>(slot.dblob);
    GroupedSplitArgs ga;
    ga.probs = reinterpret_cast<const GroupedSplit*>(db + L.off_split);
    for (int q = 0; q < 4; ++q) ga.off[q] = reinterpret_cast<const int64_t*>(db + L.off_off) + q * (count + 1);
    ga.count_dev = reinterpret_cast<const int*>(db + L.off_hdr);
    ga.err = h->d_err;
    SliceGemmArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.probs = reinterpret_cast<const SliceProblem*>(db + L.off_sp);
    sa.tmaps = reinterpret_cast<const CUtensorMap*>(db + L.off_tmap);
    sa.tiles = reinterpret_cast<const TileRef*>(db + L.off_tiles);
    sa.ntiles_dev = reinterpret_cast<const int*>(db + L.off_hdr) + 1;
    sa.err = h->d_err;
    sa.timeout_ns = static_cast<uint64_t>(h->opt_timeout_ms) * 1000000ull;
    CUtensorMap dummy;
    memset(&dummy, 0, sizeof(dummy));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(slot.dblob, slot.stage, slot.blob_cap, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(slot.ws, 0, slot.colmax_cap, cs);
    if (e == cudaSuccess) e = launch_grouped_split(fp64 ? 0 : 1, ga, h->sm_count * 8, cs);
    if (e == cudaSuccess)
      e = launch_slice_gemm(fp64 ? SLICE_FP64EMU : SLICE_FP32EMU, bn, &dummy, &dummy, sa, h->sm_count, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&slot.exec, g, 0);
    slot.graph = g;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      release_slot(h, slot);
      return cuda_status(e, "grouped capture");
    }
  }
  L.plan(count, slot.tiles_cap);
  // ---- fill the staging blob
  char* hb = static_cast<char*>(slot.stage);
  char* ws = static_cast<char*>(slot.ws);
  const size_t cmo = 0, wso = slot.colmax_cap;   // column maxima first, then per-problem regions
  int* hdr = reinterpret_cast<int*>(hb + L.off_hdr);
  hdr[0] = count;
  hdr[1] = ntiles;
  GroupedSplit* gs = reinterpret_cast<GroupedSplit*>(hb + L.off_split);
  int64_t* off = reinterpret_cast<int64_t*>(hb + L.off_off);
  SliceProblem* sp = reinterpret_cast<SliceProblem*>(hb + L.off_sp);
  CUtensorMap* tm = reinterpret_cast<CUtensorMap*>(hb + L.off_tmap);
  TileRef* tr = reinterpret_cast<TileRef*>(hb + L.off_tiles);
  int64_t acc[4] = {0, 0, 0, 0};
  for (int i = 0; i < count; ++i) {
    const mm_problem& p = probs[idx[i]];
    GroupedSplit& g = gs[i];
    g.m = p.m; g.n = p.n; g.k = p.k; g.lda = p.lda; g.ldb = p.ldb; g.kp = kp[i];
    g.A = p.A; g.B = p.B; g.s = S[i]; g.pad = 0;
    g.rowmax = reinterpret_cast<uint64_t*>(ws + wso + pw[i].rowmax);
    g.colmax = reinterpret_cast<uint64_t*>(ws + cmo + pw[i].colmax);
    g.E = reinterpret_cast<int32_t*>(ws + wso + pw[i].E);
    g.F = reinterpret_cast<int32_t*>(ws + wso + pw[i].F);
    g.slA = reinterpret_cast<uint16_t*>(ws + wso + pw[i].sa);
    g.slB = reinterpret_cast<uint16_t*>(ws + wso + pw[i].sb);
    off[0 * (count + 1) + i] = acc[0]; acc[0] += (p.m + 7) / 8;
    off[1 * (count + 1) + i] = acc[1]; acc[1] += ((p.n + 255) / 256) * ((p.k + 255) / 256);
    off[2 * (count + 1) + i] = acc[2]; acc[2] += p.m * ((p.k + 2047) / 2048);
    off[3 * (count + 1) + i] = acc[3]; acc[3] += ((p.n + 31) / 32) * ((p.k + 63) / 64);
    SliceProblem& P = sp[i];
    memset(&P, 0, sizeof(P));
    P.m = p.m; P.n = p.n; P.k = p.k;
    P.nkb = static_cast<int>((p.k + 63) / 64);
    P.s = sl[i];
    P.fix_shift = fp64 ? fixed_shift(sl[i], p.k) : 0;
    P.tiles_m = static_cast<int>((p.m + 127) / 128);
    P.tiles_n = static_cast<int>((p.n + bn - 1) / bn);
    P.E = g.E; P.F = g.F; P.C = p.C; P.ldc = p.ldc; P.levels = nullptr;
    if (!encode_slices_tmap(h, &tm[2 * i], g.slA, p.k, p.m, S[i], kp[i], 128) ||
        !encode_slices_tmap(h, &tm[2 * i + 1], g.slB, p.k, p.n, S[i], kp[i], bn))
      return MM_ERR_CUDA;
  }
  for (int q = 0; q < 4; ++q) off[q * (count + 1) + count] = acc[q];
  for (int t = 0; t < ntiles; ++t) tr[t] = tiles[t].ref;
  {
    ProfScope ps(h, MM_KERNEL_SLICE_GEMM, st);
    cudaError_t e = cudaGraphLaunch(slot.exec, st);
    if (e != cudaSuccess) return cuda_status(e, "grouped graph launch");
  }
  cudaEventRecord(slot.done, st);
  slot.launched = true;
  ent.next ^= 1;
  count_launch(h, 3);
  return MM_OK;
}

// ------------------------------------------------------------------ FP64
static int grouped_fp64(mm_handle_s* h, GroupedEntry& ent, const std::vector<int>& idx, const mm_problem* probs,
                        cudaStream_t st) {
  const int count = static_cast<int>(idx.size());
  const int T = fp64_tile_size();
  std::vector<TileCost> tiles;
  for (int i = 0; i < count; ++i) {
    const mm_problem& p = probs[idx[i]];
    const int tm = static_cast<int>((p.m + T - 1) / T), tn = static_cast<int>((p.n + T - 1) / T);
    for (int a = 0; a < tm; ++a)
      for (int b = 0; b < tn; ++b)
        tiles.push_back({std::max<int64_t>(p.k, 1), i, a * tn + b, TileRef{i, static_cast<int16_t>(a), static_cast<int16_t>(b)}});
  }
  sort_tiles(tiles);
  const int ntiles = static_cast<int>(tiles.size());
  GroupedSlot& slot = ent.slot[ent.next];
  if (slot.launched) cudaEventSynchronize(slot.done);
  Fp64Layout L;
  if (!(slot.exec && slot.tiles_cap >= ntiles)) {
    release_slot(h, slot);
    const int tiles_cap = std::max(ntiles, 1) * 5 / 4 + 64;
    L.plan(count, tiles_cap);
    slot.blob_cap = L.bytes;
    slot.tiles_cap = tiles_cap;
    int rc;
    if ((rc = reserve(h, slot.blob_cap, &slot.dblob)) != MM_OK) { slot = GroupedSlot(); return rc; }
    if (cudaMallocHost(&slot.stage, slot.blob_cap) != cudaSuccess ||
        cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming) != cudaSuccess) {
      release_slot(h, slot);
      return MM_ERR_CUDA;
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { release_slot(h, slot); return MM_ERR_CUDA; }
    char* db = static_cast<char*>(slot.dblob);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(slot.dblob, slot.stage, slot.blob_cap, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
      e = launch_fp64_grouped(fp64_kind(h), reinterpret_cast<const Fp64GemmArgs*>(db + L.off_args),
                              reinterpret_cast<const TileRef*>(db + L.off_tiles),
                              reinterpret_cast<const int*>(db + L.off_hdr) + 1, h->sm_count * 2, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&slot.exec, g, 0);
    slot.graph = g;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      release_slot(h, slot);
      return cuda_status(e, "grouped capture");
    }
  }
  L.plan(count, slot.tiles_cap);
  char* hb = static_cast<char*>(slot.stage);
  int* hdr = reinterpret_cast<int*>(hb + L.off_hdr);
  hdr[0] = count;
  hdr[1] = ntiles;
  Fp64GemmArgs* args = reinterpret_cast<Fp64GemmArgs*>(hb + L.off_args);
  for (int i = 0; i < count; ++i) {
    const mm_problem& p = probs[idx[i]];
    args[i] = Fp64GemmArgs{p.m, p.n, p.k, p.A, p.lda, p.B, p.ldb, p.C, p.ldc};
  }
  TileRef* tr = reinterpret_cast<TileRef*>(hb + L.off_tiles);
  for (int t = 0; t < ntiles; ++t) tr[t] = tiles[t].ref;
  {
    ProfScope ps(h, MM_KERNEL_FP64_GEMM, st);
    cudaError_t e = cudaGraphLaunch(slot.exec, st);
    if (e != cudaSuccess) return cuda_status(e, "grouped graph launch");
  }
  cudaEventRecord(slot.done, st);
  slot.launched = true;
  ent.next ^= 1;
  count_launch(h, 1);
  return MM_OK;
}

int grouped_run(mm_handle_s* h, int count, const mm_problem* probs, int precision, cudaStream_t st) {
  // problems the grouped kernels take, the rest go through the single path
  std::vector<int> main_idx, side_idx;
  for (int i = 0; i < count; ++i) {
    const mm_problem& p = probs[i];
    if (p.m == 0 || p.n == 0) continue;
    const bool side = (precision != MM_FP64) && (p.k == 0 || (precision == MM_FP64_EMU && p.k <= 4));
    (side ? side_idx : main_idx).push_back(i);
  }
  for (int i : side_idx) {
    const mm_problem& p = probs[i];
    int rc = gemm_device(h, p.m, p.n, p.k, p.A, p.lda, p.B, p.ldb, p.C, p.ldc, precision, st);
    if (rc != MM_OK) return rc;
  }
  if (main_idx.empty()) return MM_OK;
  std::lock_guard<std::mutex> lk(h->grouped_mu);
  if (!h->grouped) h->grouped = new GroupedCache();
  GroupedEntry& ent = h->grouped->entries[GroupedKey{static_cast<int>(main_idx.size()), precision, st}];
  if (precision == MM_FP64) return grouped_fp64(h, ent, main_idx, probs, st);
  return grouped_emulated(h, ent, main_idx, probs, precision, st);
}

}  // namespace mmhost

using namespace mmhost;

int mm_gemm_grouped(mm_handle h, int count, const mm_problem* probs, int precision, void* stream) {
  if (!h || count < 0 || (count > 0 && !probs)) return MM_ERR_INVALID_ARG;
  if (precision != MM_FP64 && precision != MM_FP64_EMU && precision != MM_FP32_EMU) return MM_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const mm_problem& p = probs[i];
    int rc = validate_problem(p.m, p.n, p.k, p.A, p.lda, p.B, p.ldb, p.C, p.ldc, precision);
    if (rc != MM_OK) return rc;
    if ((p.m + 127) / 128 > 32767 || (p.n + 127) / 128 > 32767) return MM_ERR_INVALID_ARG;
  }
  if (count == 0) return MM_OK;
  DeviceGuard g(h->device);
  return grouped_run(h, count, probs, precision, static_cast<cudaStream_t>(stream));
}
