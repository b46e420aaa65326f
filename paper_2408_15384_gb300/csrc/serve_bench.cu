// serve_bench.cu -- mm_serve_bench: an open-loop (Poisson) or closed-loop
// request stream driven through the public serving calls, for latency and
// throughput measurement. Host code only; the requests run on the serving
// engine like any client's.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

constexpr uint64_t GOLD = 0x9E3779B97F4A7C15ull;

// The counter-based generator of the input module (SplitMix64 finaliser).
uint64_t word(uint64_t seed, uint64_t stream, uint64_t i) {
  const uint64_t base = splitmix_mix_host(seed + stream * GOLD);
  return splitmix_mix_host(base + (i + 1) * GOLD);
}
double unit(uint64_t seed, uint64_t stream, uint64_t i) {
  return static_cast<double>(word(seed, stream, i) >> 11) * 0x1.0p-53;
}

struct Spec {
  int64_t m, n, k;
  int prec;
  double arrival_s;
};

double pct(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (v.size() - 1);
  const size_t lo = static_cast<size_t>(std::floor(pos));
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (v[hi] - v[lo]) * (pos - lo);
}

}  // namespace

using namespace mmhost;

int mm_serve_bench(mm_handle h, const mm_serve_load* L, mm_serve_load_result* res, mm_serve_sample* samples,
                   int64_t max_samples, int64_t* n_samples, double* sample_host, int64_t sample_cap) {
  if (!h || !L || !res || L->count <= 0 || L->dim_lo < 1 || L->dim_hi < L->dim_lo || L->slots < 1 ||
      L->fp64_share < 0 || L->fp64_share > 1)
    return MM_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (n_samples) *n_samples = 0;
  const int64_t D = L->dim_hi;
  const int S = L->slots;
  const size_t mat = static_cast<size_t>(D) * D * 8;
  // ---- request stream (dims on streams 5,6,7 of the generator: m, n, k interleaved)
  std::vector<Spec> spec(L->count);
  const double lnlo = std::log(static_cast<double>(L->dim_lo)), lnhi = std::log(static_cast<double>(D));
  double t = 0.0;
  for (int64_t i = 0; i < L->count; ++i) {
    int64_t d3[3];
    for (int j = 0; j < 3; ++j) {
      const double v = std::exp(lnlo + unit(L->seed, 5, 3 * i + j) * (lnhi - lnlo));
      d3[j] = std::min<int64_t>(D, std::max<int64_t>(L->dim_lo, static_cast<int64_t>(std::nearbyint(v))));
    }
    const int prec = (unit(L->seed, 7, i) < L->fp64_share) ? MM_FP64_EMU : MM_FP32_EMU;
    if (L->rate_per_s > 0) t += -std::log1p(-unit(L->seed, 6, i)) / L->rate_per_s;
    spec[i] = Spec{d3[0], d3[1], d3[2], prec, L->rate_per_s > 0 ? t : 0.0};
  }
  // ---- resident operand slots
  std::vector<double*> A(S, nullptr), B(S, nullptr), C(S, nullptr);
  cudaStream_t fs;
  if (cudaStreamCreateWithFlags(&fs, cudaStreamNonBlocking) != cudaSuccess) return MM_ERR_CUDA;
  int rc = MM_OK;
  for (int s = 0; s < S && rc == MM_OK; ++s) {
    if (cudaMalloc(&A[s], mat) != cudaSuccess || cudaMalloc(&B[s], mat) != cudaSuccess ||
        cudaMalloc(&C[s], mat) != cudaSuccess) {
      cudaGetLastError();
      rc = MM_ERR_BUDGET;
      break;
    }
    const uint64_t sd = L->seed * 1000003ull + static_cast<uint64_t>(s);
    if (launch_fill_uniform(A[s], D, D, D, sd, 1, 0, 0, fs) != cudaSuccess ||
        launch_fill_uniform(B[s], D, D, D, sd, 2, 0, 0, fs) != cudaSuccess)
      rc = MM_ERR_CUDA;
  }
  // Sampled outputs are copied device to device on the side stream while the
  // load runs (the slot stays held until its copy is done) and brought to the
  // host after the run, so sampling never stalls the arrival loop.
  const bool sampling = L->sample_every > 0 && samples && sample_host && max_samples > 0 && sample_cap > 0;
  double* samp_dev = nullptr;
  std::vector<cudaEvent_t> slot_ev(S, nullptr);
  std::vector<char> slot_copy(S, 0);
  if (rc == MM_OK && sampling) {
    if (cudaMalloc(&samp_dev, static_cast<size_t>(sample_cap) * 8) != cudaSuccess) {
      cudaGetLastError();
      samp_dev = nullptr;
      rc = MM_ERR_BUDGET;
    }
    for (int s = 0; s < S && rc == MM_OK; ++s)
      if (cudaEventCreateWithFlags(&slot_ev[s], cudaEventDisableTiming) != cudaSuccess) rc = MM_ERR_CUDA;
  }
  if (rc == MM_OK && cudaStreamSynchronize(fs) != cudaSuccess) rc = MM_ERR_CUDA;
  std::vector<double> lat(L->count, 0.0);
  std::vector<double> done_at(L->count, 0.0);
  int64_t completed = 0, failed = 0, ns = 0, host_used = 0;
  double flop = 0.0, t_first = 0.0, t_last = 0.0;
  if (rc == MM_OK) {
    std::vector<int64_t> slot_req(S, -1);
    std::vector<uint64_t> slot_ticket(S, 0);
    const double start_us = now_us(h) + 1000.0;   // first arrival 1 ms from now
    while (now_us(h) < start_us) std::this_thread::yield();
    t_first = start_us;
    int64_t next = 0;
    while (completed + failed < L->count) {
      bool progress = false;
      // completions
      for (int s = 0; s < S; ++s) {
        if (slot_req[s] < 0) continue;
        mm_req_status st;
        const int prc = mm_serve_poll(h, slot_ticket[s], &st);
        if (prc == MM_PENDING) continue;
        const int64_t i = slot_req[s];
        const Spec& q = spec[i];
        if (prc == MM_OK) {
          ++completed;
          const double arr = start_us + q.arrival_s * 1e6;
          lat[i] = (st.t_done_us - arr) * 1e-3;
          done_at[i] = st.t_done_us;
          t_last = std::max(t_last, st.t_done_us);
          flop += 2.0 * static_cast<double>(q.m) * q.n * q.k;
          if (sampling && i % L->sample_every == 0 && ns < max_samples && host_used + q.m * q.n <= sample_cap) {
            if (cudaMemcpy2DAsync(samp_dev + host_used, 8 * q.n, C[s], 8 * D, 8 * q.n, q.m, cudaMemcpyDeviceToDevice,
                                  fs) != cudaSuccess ||
                cudaEventRecord(slot_ev[s], fs) != cudaSuccess)
              rc = MM_ERR_CUDA;
            slot_copy[s] = 1;
            samples[ns] = mm_serve_sample{i, q.m, q.n, q.k, q.prec, s, host_used};
            host_used += q.m * q.n;
            ++ns;
          }
        } else {
          ++failed;
          lat[i] = -1.0;
        }
        slot_req[s] = -1;
        progress = true;
      }
      // arrivals that are due and whose slot is free
      const double now = now_us(h);
      while (next < L->count && start_us + spec[next].arrival_s * 1e6 <= now) {
        const int s = static_cast<int>(next % S);
        if (slot_req[s] >= 0) break;
        if (slot_copy[s]) {
          const cudaError_t qe = cudaEventQuery(slot_ev[s]);
          if (qe == cudaErrorNotReady) break;
          if (qe != cudaSuccess) rc = MM_ERR_CUDA;
          slot_copy[s] = 0;
        }
        const Spec& q = spec[next];
        mm_request r;
        r.prob = mm_problem{q.m, q.n, q.k, A[s], D, B[s], D, C[s], D};
        r.precision = q.prec;
        r.user_tag = static_cast<uint64_t>(next);
        uint64_t tk = 0;
        const int src = mm_serve_submit(h, &r, &tk);
        if (src != MM_OK) {
          ++failed;
          lat[next] = -1.0;
        } else {
          slot_req[s] = next;
          slot_ticket[s] = tk;
        }
        ++next;
        progress = true;
      }
      if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    mm_serve_drain(h);
  }
  // ---- statistics
  std::vector<double> all, l64, l32;
  double sum = 0.0;
  for (int64_t i = 0; i < L->count; ++i) {
    if (lat[i] < 0) continue;
    all.push_back(lat[i]);
    sum += lat[i];
    (spec[i].prec == MM_FP64_EMU ? l64 : l32).push_back(lat[i]);
  }
  res->completed = completed;
  res->failed = failed;
  res->wall_s = (t_last > t_first) ? (t_last - t_first) * 1e-6 : 0.0;
  res->req_per_s = res->wall_s > 0 ? completed / res->wall_s : 0.0;
  res->tflops = res->wall_s > 0 ? flop / res->wall_s / 1e12 : 0.0;
  res->p50_ms = pct(all, 0.50);
  res->p90_ms = pct(all, 0.90);
  res->p99_ms = pct(all, 0.99);
  res->max_ms = all.empty() ? 0.0 : *std::max_element(all.begin(), all.end());
  res->mean_ms = all.empty() ? 0.0 : sum / all.size();
  res->fp64_p99_ms = pct(l64, 0.99);
  res->fp32_p99_ms = pct(l32, 0.99);
  if (cudaStreamSynchronize(fs) != cudaSuccess && rc == MM_OK) rc = MM_ERR_CUDA;
  if (samp_dev && host_used > 0 &&
      cudaMemcpy(sample_host, samp_dev, static_cast<size_t>(host_used) * 8, cudaMemcpyDeviceToHost) != cudaSuccess &&
      rc == MM_OK)
    rc = MM_ERR_CUDA;
  if (n_samples) *n_samples = ns;
  for (cudaEvent_t ev : slot_ev)
    if (ev) cudaEventDestroy(ev);
  if (samp_dev) cudaFree(samp_dev);
  cudaStreamDestroy(fs);
  for (int s = 0; s < S; ++s) {
    if (A[s]) cudaFree(A[s]);
    if (B[s]) cudaFree(B[s]);
    if (C[s]) cudaFree(C[s]);
  }
  return rc;
}
