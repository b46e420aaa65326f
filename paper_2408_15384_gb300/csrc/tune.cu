// tune.cu -- the launch-configuration autotuner.
//
// With MM_OPT_AUTOTUNE on, the first product (or group) that falls into a
// shape bucket times every candidate configuration on the caller's stream
// (one warm-up and two timed runs each, CUDA events), keeps the fastest in the
// handle's table and uses it for every later call in that bucket. Buckets:
//   single products  (precision, ceil(log2 m), ceil(log2 n), ceil(log2 k))
//   grouped calls    (precision, ceil(log2 count), ceil(log2 mean dimension)),
//                    the mean dimension being the mean over the group of
//                    (m n k)^(1/3).
// Candidates: emulated modes vary the tile width and CTA grouping, the plain
// mode the FP64 tile kernel (DFMA or DMMA). Every emulated candidate gives the
// same bits (the integer recombination does not depend on the tiling), so
// tuning never changes an FP64-accuracy result. Calls on a stream that is
// being captured into a graph are never tuned (they use the table or the
// defaults). mm_tune_save / mm_tune_load keep the table across processes as
// text, one entry per line.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "internal.h"

namespace mmhost {

struct TuneEntry {
  TileCfg cfg;
  double ms = 0;
};

struct TuneTable {
  std::mutex mu;
  std::map<std::vector<int>, TuneEntry> t;
};

static TuneTable* table(mm_handle_s* h) {
  // created at mm_create; never null afterwards
  return h->tune;
}

static int ceil_log2(int64_t x) {
  int b = 0;
  while (b < 62 && (int64_t(1) << b) < x) ++b;
  return b;
}

bool tile_options_set(const mm_handle_s* h) {
  return h->opt_tile_n != 0 || h->opt_cta_pair != 0 || h->opt_fp64_kernel != 0 || h->opt_fp32_bn != 0;
}

TileCfg default_cfg(const mm_handle_s* h, int precision, int64_t m, int64_t n, int s) {
  TileCfg c;
  if (precision == MM_FP64) {
    c.kern = h->opt_fp64_kernel == 1 ? 1 : 2;
    return c;
  }
  const bool fp64 = precision == MM_FP64_EMU;
  const int pairs = fp64 ? h->max_pairs_fp64 : h->max_pairs_fp32;
  // CTA pairs for FP32-accuracy products taller than one tile. FP64-accuracy
  // products take pairs on 256-wide tiles when the carry epilogue applies
  // (s <= 5) and there are at least as many 256 x 256 pair tiles as SMs;
  // otherwise single CTAs (measured at M = N = K = 2048, 4096 and 8192)
  const int64_t pair_tiles = ((m + 255) / 256) * ((n + 255) / 256);
  const int fp64_cg = (n > 128 && s <= 5 && pair_tiles >= h->sm_count) ? 2 : 1;
  c.cg = (h->opt_cta_pair == 1) ? 1 : (h->opt_cta_pair == 2 ? 2 : (h->opt_cta_pair == 3 ? 4 :
          (fp64 ? fp64_cg : (m > 128 ? 2 : 1))));
  if (pairs <= 0) c.cg = 1;
  if (fp64) {
    // 256-wide tiles whenever the product is wider than one 128-wide tile
    // (the tensor cores need N = 256 per MMA for full rate)
    c.bn = h->opt_tile_n ? h->opt_tile_n : (n > 128 ? 256 : 128);
  } else if (c.cg >= 2) {
    c.bn = 256;
  } else if (h->opt_fp32_bn == 128 || h->opt_fp32_bn == 256) {
    c.bn = h->opt_fp32_bn;
  } else {
    // 256-wide tiles halve the operand traffic per flop; narrow products keep 128
    const int64_t t256 = ((m + 127) / 128) * ((n + 255) / 256);
    c.bn = (n > 128 && t256 >= h->sm_count / 2) ? 256 : 128;
  }
  return c;
}

// mean over the group's non-empty problems of (m n k)^(1/3)
static double group_mean_dim(int count, const mm_problem* probs) {
  double sum = 0;
  int used = 0;
  for (int i = 0; i < count; ++i) {
    const mm_problem& p = probs[i];
    if (p.m == 0 || p.n == 0) continue;
    sum += std::cbrt(static_cast<double>(p.m) * static_cast<double>(p.n) * static_cast<double>(std::max<int64_t>(p.k, 1)));
    ++used;
  }
  return used ? sum / used : 0.0;
}

TileCfg grouped_default_cfg(const mm_handle_s* h, int precision, int count, const mm_problem* probs) {
  TileCfg c;
  if (precision == MM_FP64) {
    c.kern = h->opt_fp64_kernel == 1 ? 1 : 2;
  } else {
    // 256-wide tiles once the products are large enough to fill them (the
    // tensor cores need N = 256 per MMA for full rate); 128 for small ones
    const double d = group_mean_dim(count, probs);
    c.bn = (d >= (precision == MM_FP64_EMU ? 384.0 : 256.0)) ? 256 : 128;
    c.cg = 1;
  }
  return c;
}

void tune_key_single(int precision, int64_t m, int64_t n, int64_t k, int key[5]) {
  key[0] = TUNE_SINGLE;
  key[1] = precision;
  key[2] = ceil_log2(m);
  key[3] = ceil_log2(n);
  key[4] = ceil_log2(k);
}

void tune_key_grouped(int precision, int count, const mm_problem* probs, int key[5]) {
  key[0] = TUNE_GROUPED;
  key[1] = precision;
  key[2] = ceil_log2(count);
  key[3] = ceil_log2(static_cast<int64_t>(std::llround(std::max(group_mean_dim(count, probs), 1.0))));
  key[4] = 0;
}

bool tune_lookup(mm_handle_s* h, const int key[5], TileCfg* out) {
  TuneTable* T = table(h);
  std::lock_guard<std::mutex> lk(T->mu);
  auto it = T->t.find(std::vector<int>(key, key + 5));
  if (it == T->t.end()) return false;
  *out = it->second.cfg;
  return true;
}

static void tune_store(mm_handle_s* h, const int key[5], const TileCfg& c, double ms) {
  TuneTable* T = table(h);
  std::lock_guard<std::mutex> lk(T->mu);
  TuneEntry& e = T->t[std::vector<int>(key, key + 5)];
  e.cfg = c;
  e.ms = ms;
}

std::vector<TileCfg> tune_candidates(const mm_handle_s* h, int kind, int precision, int64_t m, int64_t n) {
  std::vector<TileCfg> v;
  auto add = [&](int bn, int cg, int kern) {
    TileCfg c;
    c.bn = bn;
    c.cg = cg;
    c.kern = kern;
    v.push_back(c);
  };
  if (precision == MM_FP64) {
    add(0, 0, 2);
    add(0, 0, 1);
    return v;
  }
  if (kind == TUNE_GROUPED) {
    add(128, 1, 0);
    add(256, 1, 0);
    return v;
  }
  const bool fp64 = precision == MM_FP64_EMU;
  const bool pairs = (fp64 ? h->max_pairs_fp64 : h->max_pairs_fp32) > 0 && m > 128;
  if (fp64) {
    const int widths[4] = {256, 240, 192, 128};
    for (int bn : widths) {
      if (bn > 128 && n <= 128) continue;
      add(bn, 1, 0);
      if (pairs) add(bn, 2, 0);
    }
  } else {
    add(128, 1, 0);
    if (n > 128) {
      add(256, 1, 0);
      if (pairs) add(256, 2, 0);
    }
  }
  return v;
}

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;   // be safe: do not synchronise on a stream we cannot query
  }
  return cs != cudaStreamCaptureStatusNone;
}

int tune_pick(mm_handle_s* h, const int key[5], const std::vector<TileCfg>& cands, cudaStream_t st,
              int (*run)(void* ctx, const TileCfg& cfg), void* ctx, TileCfg* best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return MM_ERR_CUDA;
  }
  double best_ms = INFINITY;
  int rc = MM_OK;
  for (const TileCfg& c : cands) {
    int r = run(ctx, c);                       // warm-up (and first use of the kernel)
    if (r == MM_ERR_BUDGET) continue;          // this candidate does not fit: skip it
    if (r != MM_OK) { rc = r; break; }
    float ms_min = INFINITY;
    for (int rep = 0; rep < 2 && r == MM_OK; ++rep) {
      cudaEventRecord(e0, st);
      r = run(ctx, c);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) { r = MM_ERR_CUDA; break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      ms_min = std::min(ms_min, ms);
    }
    if (r != MM_OK) { rc = r; break; }
    logf(2, "tune: key (%d %d %d %d %d) bn %d cg %d kern %d: %.4f ms", key[0], key[1], key[2], key[3], key[4],
         c.bn, c.cg, c.kern, ms_min);
    if (ms_min < best_ms) {
      best_ms = ms_min;
      *best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MM_OK) return rc;
  if (!std::isfinite(best_ms)) return MM_ERR_BUDGET;
  // a timeout or other device error during the runs makes the timings meaningless
  uint32_t dev_err = 0;
  if (cudaMemcpy(&dev_err, err_word(h, st), sizeof(dev_err), cudaMemcpyDeviceToHost) != cudaSuccess) return MM_ERR_CUDA;
  if (dev_err == 0) tune_store(h, key, *best, best_ms);
  return MM_OK;
}

void tune_init(mm_handle_s* h) { h->tune = new TuneTable(); }

void tune_release(mm_handle_s* h) {
  delete h->tune;
  h->tune = nullptr;
}

}  // namespace mmhost

using namespace mmhost;

int mm_tune_save(mm_handle h, const char* path) {
  if (!h || !path) return MM_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "w");
  if (!f) return MM_ERR_INVALID_ARG;
  std::fprintf(f, "# mm tune table v1: kind precision b0 b1 b2 bn cg kern ms\n");
  {
    std::lock_guard<std::mutex> lk(h->tune->mu);
    for (const auto& kv : h->tune->t) {
      const std::vector<int>& k = kv.first;
      const TuneEntry& e = kv.second;
      std::fprintf(f, "%d %d %d %d %d %d %d %d %.6f\n", k[0], k[1], k[2], k[3], k[4], e.cfg.bn, e.cfg.cg,
                   e.cfg.kern, e.ms);
    }
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? MM_OK : MM_ERR_INVALID_ARG;
}

int mm_tune_load(mm_handle h, const char* path) {
  if (!h || !path) return MM_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return MM_ERR_NOT_FOUND;
  char line[256];
  std::vector<std::pair<std::vector<int>, TuneEntry>> rows;
  int rc = MM_OK;
  if (!std::fgets(line, sizeof line, f) || std::string(line).rfind("# mm tune table v1", 0) != 0) rc = MM_ERR_INVALID_ARG;
  while (rc == MM_OK && std::fgets(line, sizeof line, f)) {
    int k[5], bn, cg, kern;
    double ms;
    if (line[0] == '\n' || line[0] == '#') continue;
    if (std::sscanf(line, "%d %d %d %d %d %d %d %d %lf", &k[0], &k[1], &k[2], &k[3], &k[4], &bn, &cg, &kern, &ms) != 9) {
      rc = MM_ERR_INVALID_ARG;
      break;
    }
    // accept only configurations the library can launch
    const bool emu = (k[1] == MM_FP64_EMU || k[1] == MM_FP32_EMU);
    bool valid = (k[0] == TUNE_SINGLE || k[0] == TUNE_GROUPED) && (emu || k[1] == MM_FP64);
    if (valid && emu)
      valid = slice_gemm_tile_ok(k[1] == MM_FP64_EMU ? SLICE_FP64EMU : SLICE_FP32EMU, bn, cg) &&
              (k[0] == TUNE_SINGLE || cg == 1);
    if (valid && !emu) valid = (kern == 1 || kern == 2);
    if (!valid) {
      rc = MM_ERR_INVALID_ARG;
      break;
    }
    TuneEntry e;
    e.cfg.bn = emu ? bn : 0;
    e.cfg.cg = emu ? cg : 0;
    e.cfg.kern = emu ? 0 : kern;
    e.ms = ms;
    rows.emplace_back(std::vector<int>(k, k + 5), e);
  }
  std::fclose(f);
  if (rc != MM_OK) return rc;
  std::lock_guard<std::mutex> lk(h->tune->mu);
  for (auto& r : rows) h->tune->t[r.first] = r.second;
  return MM_OK;
}

int mm_tune_lookup(mm_handle h, int grouped, int precision, int64_t a, int64_t b, int64_t c, int* bn, int* cg,
                   int* kern) {
  if (!h || !bn || !cg || !kern || a < 0 || b < 0 || c < 0) return MM_ERR_INVALID_ARG;
  int key[5];
  if (grouped) {
    key[0] = TUNE_GROUPED;
    key[1] = precision;
    key[2] = ceil_log2(a);
    key[3] = ceil_log2(b);
    key[4] = 0;
  } else {
    tune_key_single(precision, a, b, c, key);
  }
  TileCfg t;
  if (!tune_lookup(h, key, &t)) return MM_ERR_NOT_FOUND;
  *bn = t.bn;
  *cg = t.cg;
  *kern = t.kern;
  return MM_OK;
}
