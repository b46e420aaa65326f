// serve.cu -- the serving engine behind mm_serve_submit / mm_serve_poll.
//
// Continuous batching under a device-memory budget:
//   * mm_serve_submit validates a request, computes its charge (operand bytes
//     A + B + C plus the split workspace its precision needs), queues it and
//     returns a ticket at once.
//   * One engine thread admits queued requests in arrival order while the
//     charges of everything admitted fit the handle's budget, groups requests of
//     the same accuracy class (up to MM_OPT_SERVE_MAX_BATCH) into one grouped
//     launch (the persistent grouped kernels), and issues it on the least
//     loaded of its streams, so batches admitted while others run overlap on
//     the device. A host function enqueued after each batch marks its requests
//     done, releases their charge and wakes the engine, which admits more.
//   * mm_serve_poll reports done / pending without blocking; timestamps of
//     submit, admission, launch and completion give the latency distribution.
// Each request's result depends only on its own problem (tile shapes and slice
// counts are functions of the shape), so it is the same alone and in a mix.
#include <algorithm>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace mmhost {


struct ServeReq {
  mm_request r;
  int status = MM_PENDING;
  size_t charge = 0;
  double t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
  int stream = -1;
  double t_gpu_start = 0, t_gpu_end = 0;
};

struct ServeEngine;

struct Batch {
  ServeEngine* eng = nullptr;
  std::vector<uint64_t> tickets;
  size_t charge = 0;
  int stream = 0;
  void* pinned = nullptr;
  size_t pinned_cap = 0;
  int status = MM_OK;
  GroupedErrReport rep;     // the launch's error words, copied back into `pinned`
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // device time at the batch's start and end
};

// The status of request i of a finished batch: the batch's launch status, else
// the device's report: a timed-out wait fails every request of the launch,
// non-finite input only the request that had it.
static int request_status(const Batch* b, std::vector<int>& out) {
  out.assign(b->tickets.size(), b->status);
  if (b->status != MM_OK || b->rep.bytes == 0) return b->status;
  const uint32_t* hdr = static_cast<const uint32_t*>(b->pinned);
  const uint32_t* perr = reinterpret_cast<const uint32_t*>(static_cast<const char*>(b->pinned) + b->rep.off_perr);
  const bool timeout = (hdr[3] & MM_DEV_ERR_TIMEOUT_H) != 0;
  for (size_t i = 0; i < b->rep.main_idx.size(); ++i) {
    const int r = b->rep.main_idx[i];
    if (timeout || (perr[i] & MM_DEV_ERR_TIMEOUT_H)) out[r] = MM_ERR_TIMEOUT;
    else if (perr[i] & MM_DEV_ERR_NONFINITE_H) out[r] = MM_ERR_NONFINITE;
  }
  return MM_OK;
}

struct ServeEngine {
  mm_handle_s* h = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, ServeReq> reqs;
  std::vector<Batch*> finished;           // completed batches not yet retired by the engine
  int inflight = 0;
  size_t charged = 0;
  uint64_t next_ticket = 1;
  uint64_t unfinished = 0;                // submitted and not yet completed
  uint64_t submit_gen = 0;                // bumped by every submit (wakes the engine)
  bool stop = false;
  std::thread th;
  std::vector<cudaStream_t> streams;
  std::vector<int> load;
  std::vector<std::pair<void*, size_t>> pinned_pool;
  cudaEvent_t ref = nullptr;              // device-clock origin of the batches' GPU times
  std::vector<cudaEvent_t> event_pool;
};

static cudaEvent_t take_event(ServeEngine& e) {
  if (!e.event_pool.empty()) {
    cudaEvent_t ev = e.event_pool.back();
    e.event_pool.pop_back();
    return ev;
  }
  cudaEvent_t ev = nullptr;
  if (cudaEventCreate(&ev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return ev;
}

// Microseconds of device time from the engine's reference event to ev (0 if
// either is missing).
static double gpu_us(const ServeEngine& e, cudaEvent_t ev) {
  float ms = 0.f;
  if (!e.ref || !ev || cudaEventElapsedTime(&ms, e.ref, ev) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return 1000.0 * static_cast<double>(ms);
}

static size_t request_charge(mm_handle_s* h, const mm_request& r) {
  const mm_problem& p = r.prob;
  size_t bytes = 8 * static_cast<size_t>(p.m * p.k + p.k * p.n + p.m * p.n);
  if (r.precision != MM_FP64 && p.k > 0) {
    // slice planes (seven for the automatic count, fourteen with the modular
    // form allowed, which also keeps its residue bytes), scan and spread records
    const bool crt = crt_allowed(h, r.precision, h->opt_slices, p.m, p.n, p.k);
    const int s = crt ? CRT_N_MAX : (r.precision == MM_FP64_EMU) ? emu_planes(h->opt_slices) : 3;
    const size_t kp = align_up(static_cast<size_t>(p.k), 8);
    bytes += 2 * static_cast<size_t>(s) * (p.m + p.n) * kp + 16 * static_cast<size_t>(p.m + p.n) +
             8 * static_cast<size_t>((p.k + 255) / 256) * p.n + 8192;
    if (crt) bytes += static_cast<size_t>(CRT_N_MAX) * p.m * align_up(static_cast<size_t>(p.n), 16);
  }
  return bytes;
}

// Host function run by CUDA after a batch's work: hand the batch back.
static void CUDART_CB batch_done(void* arg) {
  Batch* b = static_cast<Batch*>(arg);
  ServeEngine* e = b->eng;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    e->finished.push_back(b);
  }
  e->cv_work.notify_one();
}

static void retire(ServeEngine& e, Batch* b) {
  const double t = now_us(e.h);
  std::vector<int> status;
  request_status(b, status);
  const double g0 = gpu_us(e, b->ev0), g1 = gpu_us(e, b->ev1);
  for (size_t i = 0; i < b->tickets.size(); ++i) {
    auto it = e.reqs.find(b->tickets[i]);
    if (it == e.reqs.end()) continue;
    it->second.status = status[i];
    it->second.t_done = t;
    it->second.stream = b->stream;
    it->second.t_gpu_start = g0;
    it->second.t_gpu_end = g1;
  }
  if (b->ev0) e.event_pool.push_back(b->ev0);
  if (b->ev1) e.event_pool.push_back(b->ev1);
  e.charged -= b->charge;
  e.unfinished -= b->tickets.size();
  e.load[b->stream]--;
  e.inflight--;
  if (b->pinned) e.pinned_pool.push_back({b->pinned, b->pinned_cap});
  delete b;
}

static void engine_loop(ServeEngine* ep) {
  ServeEngine& e = *ep;
  mm_handle_s* h = e.h;
  // a new thread has no current context until a runtime call binds one; the
  // driver-level tensor-map encoder needs it bound before the first batch
  cudaSetDevice(h->device);
  std::unique_lock<std::mutex> lk(e.mu);
  for (;;) {
    for (Batch* b : e.finished) retire(e, b);
    if (!e.finished.empty()) {
      e.finished.clear();
      e.cv_done.notify_all();
    }
    const int max_inflight = 2 * static_cast<int>(e.streams.size());
    bool launched = false;
    while (!e.pending.empty() && e.inflight < max_inflight) {
      // a batch of the head request's accuracy class, in arrival order, within the budget
      const int prec = e.reqs[e.pending.front()].r.precision;
      std::vector<uint64_t> take;
      size_t add = 0;
      for (auto it = e.pending.begin(); it != e.pending.end() && static_cast<int>(take.size()) < h->opt_serve_max_batch;) {
        ServeReq& q = e.reqs[*it];
        if (q.r.precision != prec) { ++it; continue; }
        if (e.charged + add + q.charge > h->budget) break;
        add += q.charge;
        take.push_back(*it);
        it = e.pending.erase(it);
      }
      if (take.empty()) break;   // the head does not fit yet: wait for completions
      const double ta = now_us(h);
      std::vector<mm_problem> probs;
      probs.reserve(take.size());
      for (uint64_t tk : take) {
        ServeReq& q = e.reqs[tk];
        q.t_admit = ta;
        probs.push_back(q.r.prob);
      }
      e.charged += add;
      int si = static_cast<int>(std::min_element(e.load.begin(), e.load.end()) - e.load.begin());
      e.load[si]++;
      e.inflight++;
      Batch* b = new Batch();
      b->eng = &e;
      b->tickets = take;
      b->charge = add;
      b->stream = si;
      b->ev0 = take_event(e);
      b->ev1 = take_event(e);
      // pinned staging for the batch's descriptor blob
      size_t host_bytes = 0;
      const TileCfg cfg = grouped_cfg(h, static_cast<int>(probs.size()), probs.data(), prec);
      grouped_direct_bytes(h, static_cast<int>(probs.size()), probs.data(), prec, cfg, &host_bytes);
      for (size_t i = 0; i < e.pinned_pool.size(); ++i)
        if (e.pinned_pool[i].second >= host_bytes) {
          b->pinned = e.pinned_pool[i].first;
          b->pinned_cap = e.pinned_pool[i].second;
          e.pinned_pool.erase(e.pinned_pool.begin() + static_cast<long>(i));
          break;
        }
      lk.unlock();
      int rc = MM_OK;
      if (!b->pinned && host_bytes) {
        size_t cap = std::max<size_t>(host_bytes, size_t(1) << 20);
        if (cudaMallocHost(&b->pinned, cap) == cudaSuccess) {
          b->pinned_cap = cap;
        } else {
          b->pinned = nullptr;
          rc = MM_ERR_CUDA;
        }
      }
      const double tl = now_us(h);
      cudaStream_t st = e.streams[si];
      if (rc == MM_OK && b->ev0) cudaEventRecord(b->ev0, st);
      if (rc == MM_OK)
        rc = grouped_direct(h, static_cast<int>(probs.size()), probs.data(), prec, cfg, b->pinned, b->pinned_cap, st,
                            &b->rep);
      if (rc == MM_OK && b->ev1) cudaEventRecord(b->ev1, st);
      b->status = rc;
      if (rc != MM_OK || cudaLaunchHostFunc(st, batch_done, b) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(st);
        if (b->status == MM_OK) b->status = MM_ERR_CUDA;
        lk.lock();
        for (uint64_t tk : take) e.reqs[tk].t_launch = tl;
        e.finished.push_back(b);
      } else {
        lk.lock();
        for (uint64_t tk : take) e.reqs[tk].t_launch = tl;
      }
      launched = true;
    }
    if (launched) continue;   // retire anything that finished meanwhile
    if (e.stop && e.pending.empty() && e.inflight == 0 && e.finished.empty()) break;
    // Sleep until a batch finishes, a request arrives, or shutdown starts with
    // nothing left in flight. Every condition here must turn false again once
    // handled (a predicate that stays true would keep the mutex held and starve
    // the completion callbacks). Queued requests alone are no reason to wake:
    // they are known not to fit (budget or slots) until a completion.
    const uint64_t seen = e.submit_gen;
    e.cv_work.wait(lk, [&] {
      return !e.finished.empty() || e.submit_gen != seen || (e.stop && e.inflight == 0);
    });
  }
}

static ServeEngine* engine(mm_handle_s* h) {
  std::lock_guard<std::mutex> lk(h->serve_mu);
  if (h->serve) return h->serve;
  DeviceGuard g(h->device);
  ServeEngine* e = new ServeEngine();
  e->h = h;
  const int ns = std::max(1, h->opt_serve_streams);
  for (int i = 0; i < ns; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : e->streams) cudaStreamDestroy(x);
      delete e;
      return nullptr;
    }
    e->streams.push_back(s);
    e->load.push_back(0);
  }
  // Reserve pool memory up front (the pool keeps freed memory up to the
  // budget), so the first bursts do not wait on the driver for new memory,
  // and a few pinned staging buffers for batch descriptors.
  {
    const size_t warm = std::min<size_t>(h->budget / 2, size_t(16) << 30);
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, warm, h->pool, e->streams[0]) == cudaSuccess) {
      cudaFreeAsync(p, e->streams[0]);
      cudaStreamSynchronize(e->streams[0]);
    } else {
      cudaGetLastError();
    }
    for (int i = 0; i < 2 * ns; ++i) {
      void* hp = nullptr;
      if (cudaMallocHost(&hp, size_t(1) << 20) == cudaSuccess) e->pinned_pool.emplace_back(hp, size_t(1) << 20);
      else cudaGetLastError();
    }
  }
  if (cudaEventCreate(&e->ref) == cudaSuccess && cudaEventRecord(e->ref, e->streams[0]) == cudaSuccess) {
    cudaEventSynchronize(e->ref);
  } else {
    cudaGetLastError();
  }
  e->th = std::thread(engine_loop, e);
  h->serve = e;
  return e;
}

void serve_shutdown(mm_handle_s* h) {
  ServeEngine* e;
  {
    std::lock_guard<std::mutex> lk(h->serve_mu);
    e = h->serve;
    h->serve = nullptr;
  }
  if (!e) return;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    // queued requests are cancelled; admitted ones finish
    const double t = now_us(h);
    for (uint64_t tk : e->pending) {
      ServeReq& q = e->reqs[tk];
      q.status = MM_ERR_SHUTDOWN;
      q.t_done = t;
      e->unfinished--;
    }
    e->pending.clear();
    e->stop = true;
  }
  e->cv_work.notify_all();
  e->th.join();
  for (cudaStream_t s : e->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (auto& p : e->pinned_pool) cudaFreeHost(p.first);
  for (cudaEvent_t ev : e->event_pool) cudaEventDestroy(ev);
  if (e->ref) cudaEventDestroy(e->ref);
  delete e;
}

}  // namespace mmhost

using namespace mmhost;

int mm_serve_submit(mm_handle h, const mm_request* r, uint64_t* ticket) {
  if (!h || !r || !ticket) return MM_ERR_INVALID_ARG;
  const mm_problem& p = r->prob;
  int rc = validate_problem(p.m, p.n, p.k, p.A, p.lda, p.B, p.ldb, p.C, p.ldc, r->precision);
  if (rc != MM_OK) return rc;
  if ((p.m + 127) / 128 > 32767 || (p.n + 127) / 128 > 32767) return MM_ERR_INVALID_ARG;
  const size_t charge = request_charge(h, *r);
  if (charge > h->budget) return MM_ERR_BUDGET;
  ServeEngine* e = engine(h);
  if (!e) return MM_ERR_CUDA;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->stop) return MM_ERR_SHUTDOWN;
    const uint64_t t = e->next_ticket++;
    ServeReq& q = e->reqs[t];
    q.r = *r;
    q.charge = charge;
    q.t_submit = now_us(h);
    e->pending.push_back(t);
    e->unfinished++;
    e->submit_gen++;
    *ticket = t;
  }
  e->cv_work.notify_one();
  return MM_OK;
}

int mm_serve_poll(mm_handle h, uint64_t ticket, mm_req_status* st) {
  if (!h) return MM_ERR_INVALID_ARG;
  ServeEngine* e;
  {
    std::lock_guard<std::mutex> lk(h->serve_mu);
    e = h->serve;
  }
  if (!e) return MM_ERR_NOT_FOUND;
  std::lock_guard<std::mutex> lk(e->mu);
  auto it = e->reqs.find(ticket);
  if (it == e->reqs.end()) return MM_ERR_NOT_FOUND;
  const ServeReq& q = it->second;
  if (q.status == MM_PENDING) return MM_PENDING;
  if (st) {
    st->status = q.status;
    st->user_tag = q.r.user_tag;
    st->t_submit_us = q.t_submit;
    st->t_admit_us = q.t_admit;
    st->t_launch_us = q.t_launch;
    st->t_done_us = q.t_done;
    st->stream = q.stream;
    st->t_gpu_start_us = q.t_gpu_start;
    st->t_gpu_end_us = q.t_gpu_end;
  }
  const int rc = q.status;
  e->reqs.erase(it);
  return rc;
}

int mm_serve_drain(mm_handle h) {
  if (!h) return MM_ERR_INVALID_ARG;
  ServeEngine* e;
  {
    std::lock_guard<std::mutex> lk(h->serve_mu);
    e = h->serve;
  }
  if (!e) return MM_OK;
  std::unique_lock<std::mutex> lk(e->mu);
  e->cv_done.wait(lk, [&] { return e->unfinished == 0; });
  return MM_OK;
}
