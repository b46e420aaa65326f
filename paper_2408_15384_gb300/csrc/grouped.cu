// grouped.cu -- many independent products in one persistent launch per stage.
//
// A group is described by a descriptor blob (problem records, per-problem
// block offsets of the grouped split kernels, tensor maps, a cost-sorted tile
// list, and a header with the problem and tile counts). The kernels read all
// of it, counts included, from device memory, so the same launches serve any
// group that fits the blob's capacities.
//
// mm_gemm_grouped replays a CUDA graph made of: one memcpy of the blob from a
// pinned staging buffer to the device, one memset of the column-maximum
// region, the grouped split kernels and the grouped slice GEMM (emulated
// modes), or the grouped FP64 kernel (plain mode). The graph is captured once
// per (precision, stream) and again only when a call needs more problems,
// tiles or workspace than the captured capacities. Two graph slots alternate
// so the host can stage a call while the previous one still runs; a slot's
// staging buffer is rewritten only after its last launch finished (event).
//
// The serving engine uses the direct path: the same blob and launches, with
// the blob and workspace taken from the handle's stream-ordered pool per batch.
//
// Problems the emulated kernels do not take (k == 0, or k <= 4 in
// FP64-accuracy) run through the single-product path, so every problem's
// result equals mm_gemm on it (bit for bit in FP64 and FP64-accuracy: same
// kernels, slice counts and exact recombination).
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"

namespace mmhost {

// ------------------------------------------------------------ blob layouts
// Header words: [0] problems, [1] slice-GEMM tiles, [2] plain-fallback tiles.
// The per-problem error words follow the header (serving reads them back).
struct EmuLayout {
  size_t off_hdr = 0, off_perr = 0, off_split = 0, off_off = 0, off_sp = 0, off_tmap = 0, off_tiles = 0,
         off_fargs = 0, off_ftiles = 0, bytes = 0;
  int count_cap = 0;
  void plan(int count, int tiles, int ftiles) {
    count_cap = count;
    size_t o = 0;
    off_hdr = o; o = align_up(o + 64, 64);
    off_perr = o; o = align_up(o + sizeof(uint32_t) * count, 64);
    off_split = o; o = align_up(o + sizeof(GroupedSplit) * count, 64);
    off_off = o; o = align_up(o + sizeof(int64_t) * 5 * (count + 1), 64);
    off_sp = o; o = align_up(o + sizeof(SliceProblem) * count, 64);
    off_tmap = o; o = align_up(o + sizeof(CUtensorMap) * 2 * count, 64);
    off_tiles = o; o = align_up(o + sizeof(TileRef) * std::max(tiles, 1), 64);
    off_fargs = o; o = align_up(o + sizeof(Fp64GemmArgs) * count, 64);
    off_ftiles = o; o = align_up(o + sizeof(TileRef) * std::max(ftiles, 1), 64);
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

// Work plan of an emulated group: per-problem slice counts (0: automatic,
// decided on the device) and workspace offsets (column maxima in their own
// region first, then per-problem regions), the cost-sorted tile list, and for
// automatic counts the plain-FP64 fallback's tile list.
struct EmuPlan {
  struct Prob {
    int s;          // slice count, 0 = automatic
    int s_floor;    // smallest count the automatic rule can give for this k
    int64_t kp, ldr;
    size_t colmax, rowmax, E, F, dec, part, sa, sb, res;
    bool crt;       // the modular form allowed for this problem
  };
  std::vector<Prob> p;
  std::vector<TileCost> tiles;
  std::vector<TileRef> ftiles;
  size_t colmax_bytes = 0, ws_bytes = 0;
  int bn = 128;   // output tile width of the group's slice GEMM (one CTA per 128 x bn tile)
  bool any_auto = false;
  bool crt = false;               // some problem may take the modular form
  int auto_floor = SLICE_S_MAX;   // smallest s_floor over the automatic problems
  void build(mm_handle_s* h, const std::vector<int>& idx, const mm_problem* probs, bool fp64, int bn_) {
    bn = bn_;
    const int count = static_cast<int>(idx.size());
    p.resize(count);
    tiles.clear();
    ftiles.clear();
    any_auto = false;
    auto_floor = SLICE_S_MAX;
    const int FT = fp64_tile_size();
    size_t cm = 0, o = 0;
    for (int i = 0; i < count; ++i) {
      const mm_problem& q = probs[idx[i]];
      Prob& r = p[i];
      r.s = emu_slices(h, fp64 ? MM_FP64_EMU : MM_FP32_EMU, q.k, 0);
      r.s_floor = r.s > 0 ? r.s : std::max(SLICE_S_MIN, slice_count_floor(q.k));
      r.crt = fp64 && crt_allowed(h, MM_FP64_EMU, r.s, q.m, q.n, q.k);
      crt = crt || r.crt;
      const int planes = r.crt ? std::max(CRT_N_MAX, SLICE_S_MAX) : emu_planes(r.s);
      r.kp = static_cast<int64_t>(align_up(static_cast<size_t>(q.k), 8));
      r.ldr = static_cast<int64_t>(align_up(static_cast<size_t>(std::max<int64_t>(q.n, 1)), 16));
      // column maxima and decision records in the region zeroed before each launch
      r.colmax = cm; cm += align_up(8 * static_cast<size_t>(q.n), 256);
      r.dec = cm; cm += (r.s == 0 ? 256 : 0);
      r.rowmax = o; o = align_up(o + 8 * static_cast<size_t>(q.m), 256);
      r.E = o; o = align_up(o + 4 * static_cast<size_t>(q.m), 256);
      r.F = o; o = align_up(o + 4 * static_cast<size_t>(q.n), 256);
      r.part = o; o = align_up(o + (r.s == 0 ? 8 * static_cast<size_t>(launch_absmax_parts(q.k)) * q.n : 0), 256);
      r.sa = o; o = align_up(o + 2 * static_cast<size_t>(planes) * q.m * r.kp, 1024);
      r.sb = o; o = align_up(o + 2 * static_cast<size_t>(planes) * q.n * r.kp, 1024);
      r.res = o; o = align_up(o + (r.crt ? static_cast<size_t>(CRT_N_MAX) * q.m * r.ldr : 0), 256);
      const int tm = static_cast<int>((q.m + 127) / 128), tn = static_cast<int>((q.n + bn - 1) / bn);
      const int64_t nkb = (q.k + 63) / 64;
      // products a tile runs (for the cost order): the modular form's typical
      // 12 moduli, the digit form's pairs at its smallest count
      const int64_t pairs = r.crt ? 12 : fp64 ? static_cast<int64_t>(r.s_floor) * (r.s_floor + 1) / 2 : (r.s == 2 ? 3 : 6);
      for (int a = 0; a < tm; ++a)
        for (int b = 0; b < tn; ++b)
          tiles.push_back({nkb * pairs, i, a * tn + b, TileRef{i, static_cast<int16_t>(a), static_cast<int16_t>(b)}});
      if (r.s == 0) {
        any_auto = true;
        auto_floor = std::min(auto_floor, r.s_floor);
        const int fm = static_cast<int>((q.m + FT - 1) / FT), fn = static_cast<int>((q.n + FT - 1) / FT);
        for (int a = 0; a < fm; ++a)
          for (int b = 0; b < fn; ++b) ftiles.push_back(TileRef{i, static_cast<int16_t>(a), static_cast<int16_t>(b)});
      }
    }
    colmax_bytes = align_up(cm, 1024);
    ws_bytes = o;
    sort_tiles(tiles);
  }
};

// Fill the host copy of an emulated blob. ws points at the device workspace:
// column maxima at ws, per-problem regions at ws + colmax_cap. With perr the
// splitting kernels report non-finite input in per-problem words of the blob
// (they start at zero: the host copy is zeroed here).
static int fill_emu_blob(mm_handle_s* h, const EmuPlan& plan, const EmuLayout& L, const std::vector<int>& idx,
                         const mm_problem* probs, bool fp64, char* hb, char* ws, size_t colmax_cap, char* db,
                         bool perr) {
  const int count = static_cast<int>(idx.size());
  const int cap = L.count_cap;
  memset(hb, 0, L.off_split);   // header and per-problem error words
  int* hdr = reinterpret_cast<int*>(hb + L.off_hdr);
  hdr[0] = count;
  hdr[1] = static_cast<int>(plan.tiles.size());
  hdr[2] = static_cast<int>(plan.ftiles.size());
  GroupedSplit* gs = reinterpret_cast<GroupedSplit*>(hb + L.off_split);
  int64_t* off = reinterpret_cast<int64_t*>(hb + L.off_off);
  SliceProblem* sp = reinterpret_cast<SliceProblem*>(hb + L.off_sp);
  CUtensorMap* tm = reinterpret_cast<CUtensorMap*>(hb + L.off_tmap);
  TileRef* tr = reinterpret_cast<TileRef*>(hb + L.off_tiles);
  Fp64GemmArgs* fa = reinterpret_cast<Fp64GemmArgs*>(hb + L.off_fargs);
  TileRef* ftr = reinterpret_cast<TileRef*>(hb + L.off_ftiles);
  uint32_t* dperr = reinterpret_cast<uint32_t*>(db + L.off_perr);
  char* wsp = ws + colmax_cap;
  int64_t acc[5] = {0, 0, 0, 0, 0};
  for (int i = 0; i < count; ++i) {
    const mm_problem& q = probs[idx[i]];
    const EmuPlan::Prob& r = plan.p[i];
    const int planes = r.crt ? std::max(CRT_N_MAX, SLICE_S_MAX) : emu_planes(r.s);
    GroupedSplit& g = gs[i];
    g.m = q.m; g.n = q.n; g.k = q.k; g.lda = q.lda; g.ldb = q.ldb; g.kp = r.kp;
    g.A = q.A; g.B = q.B; g.s = r.s > 0 ? r.s : SLICE_S_MAX; g.crt = r.crt ? 1 : 0;
    g.rowmax = reinterpret_cast<uint64_t*>(wsp + r.rowmax);
    g.colmax = reinterpret_cast<uint64_t*>(ws + r.colmax);
    g.E = reinterpret_cast<int32_t*>(wsp + r.E);
    g.F = reinterpret_cast<int32_t*>(wsp + r.F);
    g.slA = reinterpret_cast<uint16_t*>(wsp + r.sa);
    g.slB = reinterpret_cast<uint16_t*>(wsp + r.sb);
    g.dec = r.s == 0 ? reinterpret_cast<SliceDecision*>(ws + r.dec) : nullptr;
    g.colpart = r.s == 0 ? reinterpret_cast<uint2*>(wsp + r.part) : nullptr;
    g.perr = perr ? dperr + i : nullptr;
    off[0 * (cap + 1) + i] = acc[0]; acc[0] += (q.m + 7) / 8;
    off[1 * (cap + 1) + i] = acc[1]; acc[1] += ((q.n + 31) / 32) * ((q.k + 255) / 256);
    off[2 * (cap + 1) + i] = acc[2]; acc[2] += (q.m * ((q.k + 7) / 8) + 255) / 256;
    off[3 * (cap + 1) + i] = acc[3]; acc[3] += ((q.n + 31) / 32) * ((q.k + 63) / 64);
    off[4 * (cap + 1) + i] = acc[4]; acc[4] += r.s == 0 ? (q.n + 255) / 256 : 0;
    SliceProblem& P = sp[i];
    memset(&P, 0, sizeof(P));
    P.m = q.m; P.n = q.n; P.k = q.k;
    P.nkb = static_cast<int>((q.k + 63) / 64);
    P.s = r.s > 0 ? r.s : SLICE_S_MAX;
    P.fix_shift = fp64 ? fixed_shift(P.s, q.k) : 0;
    if (r.s == 0) {
      P.s_dev = &g.dec->s;
      for (int c = SLICE_S_MIN; c <= SLICE_S_MAX; ++c) P.fix_tab[c] = static_cast<int8_t>(fixed_shift(c, q.k));
    }
    P.tiles_m = static_cast<int>((q.m + 127) / 128);
    P.tiles_n = static_cast<int>((q.n + plan.bn - 1) / plan.bn);
    P.E = g.E; P.F = g.F; P.C = q.C; P.ldc = q.ldc; P.levels = nullptr;
    if (r.crt) {
      P.res = reinterpret_cast<uint8_t*>(wsp + r.res);
      P.ldr = q.m * 8;
      P.rplane = q.m * r.ldr;
    }
    fa[i] = Fp64GemmArgs{q.m, q.n, q.k, q.A, q.lda, q.B, q.ldb, q.C, q.ldc, r.s == 0 ? &g.dec->s : nullptr};
    if (!encode_slices_tmap(h, &tm[2 * i], g.slA, q.k, q.m, planes, r.kp, 128) ||
        !encode_slices_tmap(h, &tm[2 * i + 1], g.slB, q.k, q.n, planes, r.kp, plan.bn))
      return MM_ERR_CUDA;
  }
  // the offsets of problems past `count` repeat the totals
  for (int q5 = 0; q5 < 5; ++q5)
    for (int i = count; i <= cap; ++i) off[q5 * (cap + 1) + i] = acc[q5];
  for (size_t t = 0; t < plan.tiles.size(); ++t) tr[t] = plan.tiles[t].ref;
  for (size_t t = 0; t < plan.ftiles.size(); ++t) ftr[t] = plan.ftiles[t];
  return MM_OK;
}

// The slice GEMM launches of an emulated group: (mode, s_lo, s_hi) each, and
// whether the plain-FP64 fallback runs. Fixed counts: one launch, the mode all
// problems allow. Automatic counts: on 128-wide tiles one launch for s = 3..7;
// on wider tiles the byte-carry kernel for s <= 5 (when some problem's k
// allows s <= 5) and the s = 6, 7 kernel; each skips the other's problems;
// then the plain-FP64 fallback for problems whose count came out as 8.
// With the modular form allowed, one more launch for it (SLICE_CRT over the
// decision codes above SLICE_CRT_BASE); the digit launches then take the
// problems whose decision fell back to the digit form.
struct GroupLaunches {
  int n = 0;
  int mode[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  bool fallback = false, crt = false;
  int sig() const {
    return (crt ? 1 << 16 : 0) | (n << 12) | (mode[0] << 8) | (mode[1] << 4) | (lo[0] << 1) | (fallback ? 1 : 0);
  }
};

static GroupLaunches group_launches(const mm_handle_s* h, const EmuPlan& plan, const std::vector<int>& idx,
                                    const mm_problem* probs, int precision, int bn) {
  GroupLaunches g;
  g.n = 1;
  if (precision != MM_FP64_EMU) {
    g.mode[0] = SLICE_FP32EMU;
    return g;
  }
  if (!plan.any_auto) {
    // fixed counts: the byte-carry recombination when every problem allows it
    int mode = bn == 128 ? SLICE_FP64EMU : -1;
    int max_s = 0;
    for (size_t i = 0; i < idx.size() && mode < 0; ++i) {
      const mm_problem& q = probs[idx[i]];
      const int s = plan.p[i].s;
      if (!slice_fp64_carry_ok(s, q.k, fixed_shift(s, q.k))) mode = SLICE_FP64EMU;
      max_s = std::max(max_s, s);
    }
    g.mode[0] = mode >= 0 ? mode : (max_s >= 6 ? SLICE_FP64EMU_CARRY7 : SLICE_FP64EMU_CARRY);
    (void)h;
    return g;
  }
  g.fallback = true;
  g.crt = plan.crt;
  if (bn == 128) {
    g.mode[0] = SLICE_FP64EMU;
    g.lo[0] = SLICE_S_MIN;
    g.hi[0] = SLICE_S_MAX;
    if (g.crt) {
      g.mode[1] = SLICE_CRT;
      g.lo[1] = SLICE_CRT_BASE + 1;
      g.hi[1] = SLICE_CRT_BASE + CRT_N_MAX;
      g.n = 2;
    }
    return g;
  }
  g.n = 0;
  if (plan.auto_floor <= 5) {
    g.mode[g.n] = SLICE_FP64EMU_CARRY;
    g.lo[g.n] = SLICE_S_MIN;
    g.hi[g.n] = 5;
    ++g.n;
  }
  g.mode[g.n] = SLICE_FP64EMU_CARRY7;
  g.lo[g.n] = 6;
  g.hi[g.n] = SLICE_S_MAX;
  ++g.n;
  if (g.crt) {
    g.mode[g.n] = SLICE_CRT;
    g.lo[g.n] = SLICE_CRT_BASE + 1;
    g.hi[g.n] = SLICE_CRT_BASE + CRT_N_MAX;
    ++g.n;
  }
  return g;
}

// The launches of an emulated group whose blob is at db (device). err: the
// word kernels report timeouts (and, without per-problem words, non-finite
// input) to.
static cudaError_t launch_emu_group(mm_handle_s* h, bool fp64, const GroupLaunches& gl, int bn, const EmuLayout& L,
                                    char* db, char* ws, size_t colmax_cap, uint32_t* err, cudaStream_t st) {
  GroupedSplitArgs ga;
  ga.probs = reinterpret_cast<const GroupedSplit*>(db + L.off_split);
  for (int q = 0; q < 5; ++q) ga.off[q] = reinterpret_cast<const int64_t*>(db + L.off_off) + q * (L.count_cap + 1);
  ga.count_dev = reinterpret_cast<const int*>(db + L.off_hdr);
  ga.err = err;
  SliceGemmArgs sa;
  memset(&sa, 0, sizeof(sa));
  sa.probs = reinterpret_cast<const SliceProblem*>(db + L.off_sp);
  sa.tmaps = reinterpret_cast<const CUtensorMap*>(db + L.off_tmap);
  sa.tiles = reinterpret_cast<const TileRef*>(db + L.off_tiles);
  sa.ntiles_dev = reinterpret_cast<const int*>(db + L.off_hdr) + 1;
  sa.err = err;
  sa.timeout_ns = static_cast<uint64_t>(h->opt_timeout_ms) * 1000000ull;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  // column maxima and decision records start at zero
  cudaError_t e = cudaMemsetAsync(ws, 0, colmax_cap, st);
  if (e == cudaSuccess) e = launch_grouped_split(fp64 ? (gl.crt ? 3 : 0) : 1, ga, h->sm_count * 8, st);
  for (int i = 0; i < gl.n && e == cudaSuccess; ++i) {
    sa.s_lo = gl.lo[i];
    sa.s_hi = gl.hi[i];
    e = launch_slice_gemm(gl.mode[i], bn, 1, &dummy, &dummy, sa, h->sm_count, st);
  }
  if (e == cudaSuccess && gl.fallback)
    e = launch_fp64_grouped(fp64_kind(h), reinterpret_cast<const Fp64GemmArgs*>(db + L.off_fargs),
                            reinterpret_cast<const TileRef*>(db + L.off_ftiles),
                            reinterpret_cast<const int*>(db + L.off_hdr) + 2, h->sm_count * 2, st,
                            reinterpret_cast<const int*>(db + L.off_hdr));
  return e;
}

struct Fp64Plan {
  std::vector<TileCost> tiles;
  void build(const std::vector<int>& idx, const mm_problem* probs) {
    const int T = fp64_tile_size();
    tiles.clear();
    for (size_t i = 0; i < idx.size(); ++i) {
      const mm_problem& p = probs[idx[i]];
      const int tm = static_cast<int>((p.m + T - 1) / T), tn = static_cast<int>((p.n + T - 1) / T);
      for (int a = 0; a < tm; ++a)
        for (int b = 0; b < tn; ++b)
          tiles.push_back({std::max<int64_t>(p.k, 1), static_cast<int>(i), a * tn + b,
                           TileRef{static_cast<int32_t>(i), static_cast<int16_t>(a), static_cast<int16_t>(b)}});
    }
    sort_tiles(tiles);
  }
};

static void fill_fp64_blob(const Fp64Plan& plan, const Fp64Layout& L, const std::vector<int>& idx,
                           const mm_problem* probs, char* hb) {
  int* hdr = reinterpret_cast<int*>(hb + L.off_hdr);
  hdr[0] = static_cast<int>(idx.size());
  hdr[1] = static_cast<int>(plan.tiles.size());
  Fp64GemmArgs* args = reinterpret_cast<Fp64GemmArgs*>(hb + L.off_args);
  for (size_t i = 0; i < idx.size(); ++i) {
    const mm_problem& p = probs[idx[i]];
    args[i] = Fp64GemmArgs{p.m, p.n, p.k, p.A, p.lda, p.B, p.ldb, p.C, p.ldc};
  }
  TileRef* tr = reinterpret_cast<TileRef*>(hb + L.off_tiles);
  for (size_t t = 0; t < plan.tiles.size(); ++t) tr[t] = plan.tiles[t].ref;
}

static cudaError_t launch_fp64_group(mm_handle_s* h, int kern, const Fp64Layout& L, char* db, cudaStream_t st) {
  return launch_fp64_grouped((kern == 1 || kern == 2) ? kern : fp64_kind(h),
                             reinterpret_cast<const Fp64GemmArgs*>(db + L.off_args),
                             reinterpret_cast<const TileRef*>(db + L.off_tiles),
                             reinterpret_cast<const int*>(db + L.off_hdr) + 1, h->sm_count * 2, st);
}

// Split a group into the problems the grouped kernels take and the rest.
static void partition(int count, const mm_problem* probs, int precision, std::vector<int>& main_idx,
                      std::vector<int>& side_idx) {
  for (int i = 0; i < count; ++i) {
    const mm_problem& p = probs[i];
    if (p.m == 0 || p.n == 0) continue;
    const bool side = (precision != MM_FP64) && (p.k == 0 || (precision == MM_FP64_EMU && p.k <= 4));
    (side ? side_idx : main_idx).push_back(i);
  }
}

// --------------------------------------------------------------- graph path
struct GroupedSlot {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* stage = nullptr;       // pinned host staging of the blob
  void* dblob = nullptr;       // device blob
  size_t blob_cap = 0;
  void* ws = nullptr;          // device workspace (emulated modes): column maxima, then per-problem regions
  size_t ws_cap = 0, colmax_cap = 0;
  int count_cap = 0, tiles_cap = 0, ftiles_cap = 0;
  cudaEvent_t done = nullptr;
  bool launched = false;
};

struct GroupedKey {
  int precision;
  cudaStream_t stream;
  int bn, kern, mode;   // launch configuration captured in the graph
  bool operator<(const GroupedKey& o) const {
    return std::tie(precision, stream, bn, kern, mode) < std::tie(o.precision, o.stream, o.bn, o.kern, o.mode);
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

// Capture [blob memcpy, launches] into the slot's graph.
template <typename LaunchFn>
static int capture_slot(GroupedSlot& slot, LaunchFn&& launches) {
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MM_ERR_CUDA;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaMemcpyAsync(slot.dblob, slot.stage, slot.blob_cap, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = launches(cs);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&slot.exec, g, 0);
  slot.graph = g;
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e, "grouped capture");
  }
  return MM_OK;
}

static int alloc_slot(mm_handle_s* h, GroupedSlot& slot, size_t blob_bytes, size_t ws_bytes) {
  int rc;
  slot.blob_cap = blob_bytes;
  if ((rc = reserve(h, slot.blob_cap, &slot.dblob)) != MM_OK) { slot = GroupedSlot(); return rc; }
  if (ws_bytes) {
    slot.ws_cap = ws_bytes;
    if ((rc = reserve(h, slot.ws_cap, &slot.ws)) != MM_OK) {
      slot.ws_cap = 0;
      release_slot(h, slot);
      return rc;
    }
  }
  if (cudaMallocHost(&slot.stage, slot.blob_cap) != cudaSuccess ||
      cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming) != cudaSuccess) {
    release_slot(h, slot);
    return MM_ERR_CUDA;
  }
  return MM_OK;
}

static int graph_emulated(mm_handle_s* h, GroupedEntry& ent, const EmuPlan& plan, const GroupLaunches& gl,
                          const std::vector<int>& idx, const mm_problem* probs, int precision, int bn,
                          cudaStream_t st) {
  const bool fp64 = precision == MM_FP64_EMU;
  const int count = static_cast<int>(idx.size());
  const int ntiles = static_cast<int>(plan.tiles.size()), nftiles = static_cast<int>(plan.ftiles.size());
  GroupedSlot& slot = ent.slot[ent.next];
  if (slot.launched) cudaEventSynchronize(slot.done);
  const bool fits = slot.exec && slot.count_cap >= count && slot.tiles_cap >= ntiles && slot.ftiles_cap >= nftiles &&
                    slot.colmax_cap >= plan.colmax_bytes && slot.ws_cap - slot.colmax_cap >= plan.ws_bytes;
  EmuLayout L;
  uint32_t* err = err_word(h, st);
  if (!fits) {
    release_slot(h, slot);
    const int cc = std::max(count, 64), tc = std::max(ntiles, 1) * 5 / 4 + 64;
    const int fc = nftiles > 0 ? std::max(nftiles, 1) * 5 / 4 + 64 : 0;
    L.plan(cc, tc, fc);
    const size_t colmax_cap = align_up(plan.colmax_bytes + plan.colmax_bytes / 4 + 4096, 1024);
    const size_t ws_total = colmax_cap + plan.ws_bytes + plan.ws_bytes / 4 + (size_t(1) << 20);
    int rc = alloc_slot(h, slot, L.bytes, ws_total);
    if (rc != MM_OK) return rc;
    slot.count_cap = cc;
    slot.tiles_cap = tc;
    slot.ftiles_cap = fc;
    slot.colmax_cap = colmax_cap;
    char* db = static_cast<char*>(slot.dblob);
    char* ws = static_cast<char*>(slot.ws);
    rc = capture_slot(
        slot, [&](cudaStream_t cs) { return launch_emu_group(h, fp64, gl, bn, L, db, ws, colmax_cap, err, cs); });
    if (rc != MM_OK) {
      release_slot(h, slot);
      return rc;
    }
  }
  L.plan(slot.count_cap, slot.tiles_cap, slot.ftiles_cap);
  int rc = fill_emu_blob(h, plan, L, idx, probs, fp64, static_cast<char*>(slot.stage), static_cast<char*>(slot.ws),
                         slot.colmax_cap, static_cast<char*>(slot.dblob), false);
  if (rc != MM_OK) return rc;
  {
    ProfScope ps(h, MM_KERNEL_SLICE_GEMM, st);
    cudaError_t e = cudaGraphLaunch(slot.exec, st);
    if (e != cudaSuccess) return cuda_status(e, "grouped graph launch");
  }
  cudaEventRecord(slot.done, st);
  slot.launched = true;
  ent.next ^= 1;
  count_launch(h, 2 + static_cast<uint64_t>(fp64) + (gl.crt ? 1 : 0) + static_cast<uint64_t>(gl.n) +
                     (gl.fallback ? 1 : 0));
  return MM_OK;
}

static int graph_fp64(mm_handle_s* h, GroupedEntry& ent, const std::vector<int>& idx, const mm_problem* probs,
                      int kern, cudaStream_t st) {
  const int count = static_cast<int>(idx.size());
  Fp64Plan plan;
  plan.build(idx, probs);
  const int ntiles = static_cast<int>(plan.tiles.size());
  GroupedSlot& slot = ent.slot[ent.next];
  if (slot.launched) cudaEventSynchronize(slot.done);
  Fp64Layout L;
  if (!(slot.exec && slot.count_cap >= count && slot.tiles_cap >= ntiles)) {
    release_slot(h, slot);
    const int cc = std::max(count, 64), tc = std::max(ntiles, 1) * 5 / 4 + 64;
    L.plan(cc, tc);
    int rc = alloc_slot(h, slot, L.bytes, 0);
    if (rc != MM_OK) return rc;
    slot.count_cap = cc;
    slot.tiles_cap = tc;
    char* db = static_cast<char*>(slot.dblob);
    rc = capture_slot(slot, [&](cudaStream_t cs) { return launch_fp64_group(h, kern, L, db, cs); });
    if (rc != MM_OK) {
      release_slot(h, slot);
      return rc;
    }
  }
  L.plan(slot.count_cap, slot.tiles_cap);
  fill_fp64_blob(plan, L, idx, probs, static_cast<char*>(slot.stage));
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

static int run_side(mm_handle_s* h, const std::vector<int>& side_idx, const mm_problem* probs, int precision,
                    cudaStream_t st) {
  for (int i : side_idx) {
    const mm_problem& p = probs[i];
    int rc = gemm_device(h, p.m, p.n, p.k, p.A, p.lda, p.B, p.ldb, p.C, p.ldc, precision, st);
    if (rc != MM_OK) return rc;
  }
  return MM_OK;
}

namespace {
struct GroupedRun {
  mm_handle_s* h;
  int count;
  const mm_problem* probs;
  int precision;
  cudaStream_t st;
  std::vector<char> host;
};
int grouped_tune_run(void* ctx, const TileCfg& c) {
  GroupedRun* r = static_cast<GroupedRun*>(ctx);
  size_t hb = 0;
  grouped_direct_bytes(r->h, r->count, r->probs, r->precision, c, &hb);
  if (r->host.size() < hb) r->host.resize(hb);
  // the staging buffer is reused by the next run: wait for this one's copy
  int rc = grouped_direct(r->h, r->count, r->probs, r->precision, c, r->host.data(), r->host.size(), r->st);
  if (rc == MM_OK && cudaStreamSynchronize(r->st) != cudaSuccess) rc = MM_ERR_CUDA;
  return rc;
}
}  // namespace

TileCfg grouped_cfg(mm_handle_s* h, int count, const mm_problem* probs, int precision) {
  TileCfg c = grouped_default_cfg(h, precision, count, probs);
  if (tile_options_set(h)) return c;
  int key[5];
  tune_key_grouped(precision, count, probs, key);
  TileCfg t;
  if (tune_lookup(h, key, &t)) c = t;
  return c;
}

int grouped_run(mm_handle_s* h, int count, const mm_problem* probs, int precision, cudaStream_t st) {
  std::vector<int> main_idx, side_idx;
  partition(count, probs, precision, main_idx, side_idx);
  int rc = run_side(h, side_idx, probs, precision, st);
  if (rc != MM_OK || main_idx.empty()) return rc;
  TileCfg cfg = grouped_default_cfg(h, precision, count, probs);
  if (!tile_options_set(h)) {
    int key[5];
    tune_key_grouped(precision, count, probs, key);
    if (!tune_lookup(h, key, &cfg) && h->opt_autotune && !stream_capturing(st)) {
      // the tuning runs go through the direct path (same kernels); the chosen
      // configuration then runs once more below, through the graph
      GroupedRun r{h, count, probs, precision, st, {}};
      rc = tune_pick(h, key, tune_candidates(h, TUNE_GROUPED, precision, 0, 0), st, grouped_tune_run, &r, &cfg);
      if (rc == MM_ERR_BUDGET) cfg = grouped_default_cfg(h, precision, count, probs);
      else if (rc != MM_OK) return rc;
    }
  }
  std::lock_guard<std::mutex> lk(h->grouped_mu);
  if (!h->grouped) h->grouped = new GroupedCache();
  if (precision == MM_FP64) {
    GroupedEntry& ent = h->grouped->entries[GroupedKey{precision, st, 0, cfg.kern, 0}];
    return graph_fp64(h, ent, main_idx, probs, cfg.kern, st);
  }
  EmuPlan plan;
  plan.build(h, main_idx, probs, precision == MM_FP64_EMU, cfg.bn);
  const GroupLaunches gl = group_launches(h, plan, main_idx, probs, precision, cfg.bn);
  GroupedEntry& ent = h->grouped->entries[GroupedKey{precision, st, cfg.bn, 0, gl.sig()}];
  return graph_emulated(h, ent, plan, gl, main_idx, probs, precision, cfg.bn, st);
}

// -------------------------------------------------------------- direct path
size_t grouped_direct_bytes(mm_handle_s* h, int count, const mm_problem* probs, int precision, const TileCfg& cfg,
                            size_t* host_bytes) {
  std::vector<int> main_idx, side_idx;
  partition(count, probs, precision, main_idx, side_idx);
  *host_bytes = 0;
  if (main_idx.empty()) return 0;
  if (precision == MM_FP64) {
    Fp64Plan plan;
    plan.build(main_idx, probs);
    Fp64Layout L;
    L.plan(static_cast<int>(main_idx.size()), static_cast<int>(plan.tiles.size()));
    *host_bytes = L.bytes;
    return L.bytes;
  }
  EmuPlan plan;
  plan.build(h, main_idx, probs, precision == MM_FP64_EMU, cfg.bn ? cfg.bn : 128);
  EmuLayout L;
  L.plan(static_cast<int>(main_idx.size()), static_cast<int>(plan.tiles.size()), static_cast<int>(plan.ftiles.size()));
  *host_bytes = L.bytes;
  return align_up(L.bytes, 1024) + plan.colmax_bytes + plan.ws_bytes;
}

int grouped_direct(mm_handle_s* h, int count, const mm_problem* probs, int precision, const TileCfg& cfg,
                   void* host_blob, size_t host_cap, cudaStream_t st, GroupedErrReport* rep) {
  std::vector<int> main_idx, side_idx;
  partition(count, probs, precision, main_idx, side_idx);
  if (rep) {
    rep->bytes = 0;
    rep->main_idx.clear();
  }
  int rc = run_side(h, side_idx, probs, precision, st);
  if (rc != MM_OK || main_idx.empty()) return rc;
  const int n = static_cast<int>(main_idx.size());
  char* hb = static_cast<char*>(host_blob);
  if (precision == MM_FP64) {
    Fp64Plan plan;
    plan.build(main_idx, probs);
    Fp64Layout L;
    L.plan(n, static_cast<int>(plan.tiles.size()));
    if (L.bytes > host_cap) return MM_ERR_INVALID_ARG;
    void* dev = nullptr;
    if ((rc = ws_alloc(h, L.bytes, st, &dev)) != MM_OK) return rc;
    fill_fp64_blob(plan, L, main_idx, probs, hb);
    cudaError_t e = cudaMemcpyAsync(dev, hb, L.bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      ProfScope ps(h, MM_KERNEL_FP64_GEMM, st);
      e = launch_fp64_group(h, cfg.kern, L, static_cast<char*>(dev), st);
    }
    ws_free(h, dev, L.bytes, st);
    count_launch(h, 1);
    return cuda_status(e, "grouped fp64");
  }
  const bool fp64 = precision == MM_FP64_EMU;
  const int bn = cfg.bn ? cfg.bn : 128;
  EmuPlan plan;
  plan.build(h, main_idx, probs, fp64, bn);
  const GroupLaunches gl = group_launches(h, plan, main_idx, probs, precision, bn);
  EmuLayout L;
  L.plan(n, static_cast<int>(plan.tiles.size()), static_cast<int>(plan.ftiles.size()));
  if (L.bytes > host_cap) return MM_ERR_INVALID_ARG;
  const size_t blob = align_up(L.bytes, 1024);
  const size_t total = blob + plan.colmax_bytes + plan.ws_bytes;
  void* dev = nullptr;
  if ((rc = ws_alloc(h, total, st, &dev)) != MM_OK) return rc;
  char* db = static_cast<char*>(dev);
  char* ws = db + blob;
  rc = fill_emu_blob(h, plan, L, main_idx, probs, fp64, hb, ws, plan.colmax_bytes, db, rep != nullptr);
  cudaError_t e = cudaSuccess;
  if (rc == MM_OK) {
    // with a report: the launch's own error word in the blob's header, next to
    // the per-problem words, both copied back into the host blob afterwards
    uint32_t* err = rep ? reinterpret_cast<uint32_t*>(db + L.off_hdr) + 3 : err_word(h, st);
    e = cudaMemcpyAsync(db, hb, L.bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      ProfScope ps(h, MM_KERNEL_SLICE_GEMM, st);
      e = launch_emu_group(h, fp64, gl, bn, L, db, ws, plan.colmax_bytes, err, st);
    }
    if (e == cudaSuccess && rep) {
      rep->bytes = L.off_perr + sizeof(uint32_t) * n;
      rep->off_perr = L.off_perr;
      rep->main_idx = main_idx;
      e = cudaMemcpyAsync(hb, db, rep->bytes, cudaMemcpyDeviceToHost, st);
    }
    count_launch(h, 2 + static_cast<uint64_t>(fp64) + (gl.crt ? 1 : 0) + static_cast<uint64_t>(gl.n) +
                       (gl.fallback ? 1 : 0));
  }
  ws_free(h, dev, total, st);
  if (rc != MM_OK) return rc;
  return cuda_status(e, "grouped emulated");
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
