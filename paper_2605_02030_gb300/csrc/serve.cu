// Continuous-batching query server over a resident index (the serving form of
// the query path; the paper answers one query at a time, Section 4.1.2).
//
// Requests arrive one by one (uhnsw_server_submit) and wait in a host queue.
// A dispatcher thread admits them into batches while the search state of the
// admitted-but-unfinished requests (beam, visited table and verification
// lists of each query, the bytes a query occupies while it runs) stays within
// the budget, and launches each batch on one of several streams as soon as
// one is free: requests that arrive while other batches are on the GPU are
// admitted as slots and state budget free up, and their batches run
// concurrently with those already on the device.  A completion thread moves
// finished batches' results to their requests and records each request's
// latency (submit to result available on the host).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "uhnsw.h"
#include "uhnsw_internal.h"

using uhnsw_internal::clear_error;
using uhnsw_internal::fail;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  std::vector<float> q;
  float p = 1.f;
  int32_t k = 1, ef = 1;
  int64_t state = 0;
  Clock::time_point t_submit, t_done;
  bool done = false;
  int32_t status = 0;
  std::vector<int64_t> ids;
  std::vector<float> dist;
};

struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t event = nullptr;
  float* d_q = nullptr;
  float* d_p = nullptr;
  int32_t* d_k = nullptr;
  int32_t* d_ef = nullptr;
  int64_t* d_ids = nullptr;
  float* d_dist = nullptr;
  float* h_q = nullptr;  // pinned
  float* h_p = nullptr;
  int32_t* h_k = nullptr;
  int32_t* h_ef = nullptr;
  int64_t* h_ids = nullptr;
  float* h_dist = nullptr;
  bool busy = false;      // reserved by the dispatcher for a batch
  bool launched = false;  // the batch's completion event is recorded
  std::vector<uint64_t> tickets;
  int64_t state = 0;
};

}  // namespace

struct uhnsw_server {
  uhnsw_index* idx = nullptr;
  uhnsw_server_opts o;
  int32_t d = 0;
  std::vector<Lane> lanes;
  std::mutex mu;
  std::condition_variable cv_work;   // dispatcher: new requests or a free lane
  std::condition_variable cv_done;   // waiters: a request finished
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_ticket = 1;
  int64_t inflight_state = 0;
  bool stop = false;
  int32_t error = 0;
  std::thread dispatcher, completer;
  // statistics: latencies of the last kLatWindow requests (a ring), and the
  // number finished in all
  static constexpr size_t kLatWindow = size_t(1) << 20;
  std::vector<double> lat_us;
  int64_t completed = 0;
  int64_t batches = 0, batched_queries = 0, peak_inflight = 0, inflight_queries = 0;
  int64_t peak_state = 0;
};

namespace {

void free_lane(Lane& L) {
  if (L.stream) cudaStreamDestroy(L.stream);
  if (L.event) cudaEventDestroy(L.event);
  cudaFree(L.d_q);
  cudaFree(L.d_p);
  cudaFree(L.d_k);
  cudaFree(L.d_ef);
  cudaFree(L.d_ids);
  cudaFree(L.d_dist);
  cudaFreeHost(L.h_q);
  cudaFreeHost(L.h_p);
  cudaFreeHost(L.h_k);
  cudaFreeHost(L.h_ef);
  cudaFreeHost(L.h_ids);
  cudaFreeHost(L.h_dist);
}

cudaError_t alloc_lane(Lane& L, int64_t B, int32_t d, int32_t kmax) {
  cudaError_t e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.event, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&L.d_q, B * d * 4);
  if (e == cudaSuccess) e = cudaMalloc(&L.d_p, B * 4);
  if (e == cudaSuccess) e = cudaMalloc(&L.d_k, B * 4);
  if (e == cudaSuccess) e = cudaMalloc(&L.d_ef, B * 4);
  if (e == cudaSuccess) e = cudaMalloc(&L.d_ids, B * kmax * 8);
  if (e == cudaSuccess) e = cudaMalloc(&L.d_dist, B * kmax * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&L.h_q, B * d * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&L.h_p, B * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&L.h_k, B * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&L.h_ef, B * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&L.h_ids, B * kmax * 8);
  if (e == cudaSuccess) e = cudaMallocHost(&L.h_dist, B * kmax * 4);
  return e;
}

// Launches one batch on lane L (caller holds no lock; the lane is reserved).
int launch_batch(uhnsw_server* s, Lane& L, int device) {
  const int64_t nb = (int64_t)L.tickets.size();
  cudaSetDevice(device);
  cudaError_t e = cudaMemcpyAsync(L.d_q, L.h_q, nb * s->d * 4, cudaMemcpyHostToDevice, L.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_p, L.h_p, nb * 4, cudaMemcpyHostToDevice, L.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_k, L.h_k, nb * 4, cudaMemcpyHostToDevice, L.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_ef, L.h_ef, nb * 4, cudaMemcpyHostToDevice, L.stream);
  if (e != cudaSuccess) return fail(UHNSW_ECUDA, "server: upload: %s", cudaGetErrorString(e));
  uhnsw_search_opts so = s->o.search;
  so.stats = nullptr;
  so.use_graph = 0;
  so.kernel_events = nullptr;
  so.t_per_query = nullptr;  // per-request t / tau are not part of a server request
  so.tau_per_query = nullptr;
  so.ef_max = s->o.ef_max;
  int rc = uhnsw_search(s->idx, L.d_q, L.d_p, L.d_k, L.d_ef, nb, s->o.k_max, s->o.ef_max, &so,
                        L.d_ids, L.d_dist, L.stream);
  if (rc != UHNSW_OK) return rc;
  e = cudaMemcpyAsync(L.h_ids, L.d_ids, nb * s->o.k_max * 8, cudaMemcpyDeviceToHost, L.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L.h_dist, L.d_dist, nb * s->o.k_max * 4, cudaMemcpyDeviceToHost, L.stream);
  if (e == cudaSuccess) e = cudaEventRecord(L.event, L.stream);
  if (e != cudaSuccess) return fail(UHNSW_ECUDA, "server: launch: %s", cudaGetErrorString(e));
  return UHNSW_OK;
}

void dispatcher_main(uhnsw_server* s, int device) {
  cudaSetDevice(device);
  const auto window = std::chrono::microseconds(s->o.max_delay_us);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    // a free lane and something to run
    Lane* L = nullptr;
    for (auto& ln : s->lanes)
      if (!ln.busy) {
        L = &ln;
        break;
      }
    if (!L || s->pending.empty()) {
      s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    // batching window: while other batches are running, let a partial batch
    // fill for up to max_delay_us after its oldest request arrived
    bool any_busy = false;
    for (auto& ln : s->lanes) any_busy |= ln.busy;
    if (any_busy && (int64_t)s->pending.size() < s->o.max_batch) {
      const auto oldest = s->reqs[s->pending.front()].t_submit;
      const auto now = Clock::now();
      if (now - oldest < window) {
        s->cv_work.wait_for(lk, window - (now - oldest));
        continue;
      }
    }
    // admission: requests in arrival order while the batch and the state budget allow
    L->tickets.clear();
    L->state = 0;
    while (!s->pending.empty() && (int64_t)L->tickets.size() < s->o.max_batch) {
      const uint64_t t = s->pending.front();
      Request& r = s->reqs[t];
      if (s->inflight_state + L->state + r.state > s->o.state_budget && !L->tickets.empty()) break;
      if (s->inflight_state + L->state + r.state > s->o.state_budget && s->inflight_state > 0) break;
      const int64_t i = (int64_t)L->tickets.size();
      std::memcpy(L->h_q + i * s->d, r.q.data(), sizeof(float) * s->d);
      L->h_p[i] = r.p;
      L->h_k[i] = r.k;
      L->h_ef[i] = r.ef;
      L->tickets.push_back(t);
      L->state += r.state;
      s->pending.pop_front();
    }
    if (L->tickets.empty()) {
      s->cv_work.wait_for(lk, std::chrono::milliseconds(1));
      continue;
    }
    L->busy = true;
    L->launched = false;
    s->inflight_state += L->state;
    s->inflight_queries += (int64_t)L->tickets.size();
    s->peak_inflight = std::max(s->peak_inflight, s->inflight_queries);
    s->peak_state = std::max(s->peak_state, s->inflight_state);
    s->batches += 1;
    s->batched_queries += (int64_t)L->tickets.size();
    lk.unlock();
    const int rc = launch_batch(s, *L, device);
    lk.lock();
    if (rc == UHNSW_OK) L->launched = true;
    if (rc != UHNSW_OK) {
      s->error = rc;
      for (uint64_t t : L->tickets) {
        Request& r = s->reqs[t];
        r.done = true;
        r.status = rc;
        r.t_done = Clock::now();
      }
      L->busy = false;
      s->inflight_state -= L->state;
      s->inflight_queries -= (int64_t)L->tickets.size();
      s->cv_done.notify_all();
    }
  }
}

void completer_main(uhnsw_server* s, int device) {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progressed = false;
    for (auto& L : s->lanes) {
      if (!L.busy || !L.launched) continue;
      const cudaError_t q = cudaEventQuery(L.event);
      if (q == cudaErrorNotReady) continue;
      const auto now = Clock::now();
      const int kmax = s->o.k_max;
      for (size_t i = 0; i < L.tickets.size(); ++i) {
        Request& r = s->reqs[L.tickets[i]];
        r.ids.assign(L.h_ids + i * kmax, L.h_ids + i * kmax + r.k);
        r.dist.assign(L.h_dist + i * kmax, L.h_dist + i * kmax + r.k);
        r.status = q == cudaSuccess ? 0 : UHNSW_ECUDA;
        r.done = true;
        r.t_done = now;
        const double us = std::chrono::duration<double, std::micro>(now - r.t_submit).count();
        if (s->lat_us.size() < uhnsw_server::kLatWindow) s->lat_us.push_back(us);
        else s->lat_us[(size_t)s->completed % uhnsw_server::kLatWindow] = us;
        ++s->completed;
      }
      if (q != cudaSuccess) s->error = UHNSW_ECUDA;
      L.busy = false;
      L.launched = false;
      s->inflight_state -= L.state;
      s->inflight_queries -= (int64_t)L.tickets.size();
      progressed = true;
    }
    if (progressed) {
      s->cv_done.notify_all();
      s->cv_work.notify_all();
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

}  // namespace

extern "C" int uhnsw_server_create(uhnsw_index* idx, const uhnsw_server_opts* opts,
                                   uhnsw_server** out) {
  clear_error();
  if (!idx || !out) return fail(UHNSW_EINVAL, "uhnsw_server_create: NULL argument");
  *out = nullptr;
  uhnsw_server_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.max_batch == 0) o.max_batch = 1024;
  if (o.streams == 0) o.streams = 4;
  if (o.k_max == 0) o.k_max = 100;
  if (o.ef_max == 0) o.ef_max = 512;
  if (o.max_delay_us == 0) o.max_delay_us = 200;
  if (o.max_batch < 1 || o.max_batch > (1 << 20) || o.streams < 1 || o.streams > 64 ||
      o.k_max < 1 || o.k_max > UHNSW_MAX_EF || o.ef_max < 1 || o.ef_max > UHNSW_MAX_EF ||
      o.max_delay_us < 0 || o.state_budget < 0)
    return fail(UHNSW_EINVAL, "uhnsw_server_create: option out of range");
  int64_t n = 0;
  int32_t d = 0;
  uhnsw_index_info(idx, &n, &d, nullptr, nullptr, nullptr);
  const int64_t per_query = uhnsw_internal::query_state_bytes(idx, o.ef_max, o.k_max, &o.search);
  if (per_query < 0) return (int)per_query;
  if (o.state_budget == 0) o.state_budget = per_query * o.max_batch * 2;
  if (o.state_budget < per_query)
    return fail(UHNSW_EINVAL, "uhnsw_server_create: state budget below one query (%lld bytes)",
                (long long)per_query);
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return fail(UHNSW_ECUDA, "uhnsw_server_create: %s", cudaGetErrorString(e));
  uhnsw_server* s = new (std::nothrow) uhnsw_server();
  if (!s) return fail(UHNSW_EOOM, "uhnsw_server_create: host memory");
  s->idx = idx;
  s->o = o;
  s->d = d;
  s->lanes.resize(o.streams);
  for (auto& L : s->lanes) {
    e = alloc_lane(L, o.max_batch, d, o.k_max);
    if (e != cudaSuccess) {
      for (auto& L2 : s->lanes) free_lane(L2);
      delete s;
      return fail(e == cudaErrorMemoryAllocation ? UHNSW_EOOM : UHNSW_ECUDA,
                  "uhnsw_server_create: %s", cudaGetErrorString(e));
    }
  }
  s->dispatcher = std::thread(dispatcher_main, s, device);
  s->completer = std::thread(completer_main, s, device);
  *out = s;
  return UHNSW_OK;
}

extern "C" int uhnsw_server_submit(uhnsw_server* s, const float* q, float p, int32_t k, int32_t ef,
                                   uint64_t* ticket) {
  clear_error();
  if (!s || !q || !ticket) return fail(UHNSW_EINVAL, "uhnsw_server_submit: NULL argument");
  if (!(p > 0.f) || !(p <= 2.f) || k < 1 || k > s->o.k_max || ef < 1 || ef > s->o.ef_max ||
      std::max(ef, k) > s->o.ef_max)
    return fail(UHNSW_EINVAL, "uhnsw_server_submit: p=%g k=%d ef=%d outside the server's limits",
                (double)p, k, ef);
  Request r;
  r.q.assign(q, q + s->d);
  r.p = p;
  r.k = k;
  r.ef = ef;
  r.state = uhnsw_internal::query_state_bytes(s->idx, std::max(ef, k), k, &s->o.search);
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return fail(s->error, "uhnsw_server_submit: server failed earlier (%d)", s->error);
    const uint64_t t = s->next_ticket++;
    s->reqs.emplace(t, std::move(r));
    s->pending.push_back(t);
    *ticket = t;
  }
  s->cv_work.notify_one();
  return UHNSW_OK;
}

static int take_result(uhnsw_server* s, uint64_t ticket, int64_t* ids, float* dist,
                       double* latency_us) {
  auto it = s->reqs.find(ticket);
  Request& r = it->second;
  const int status = r.status;
  if (ids) std::copy(r.ids.begin(), r.ids.end(), ids);
  if (dist) std::copy(r.dist.begin(), r.dist.end(), dist);
  if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
  s->reqs.erase(it);
  return status;
}

extern "C" int uhnsw_server_poll(uhnsw_server* s, uint64_t ticket, int64_t* ids, float* dist,
                                 int32_t* done) {
  clear_error();
  if (!s || !done) return fail(UHNSW_EINVAL, "uhnsw_server_poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(UHNSW_EINVAL, "uhnsw_server_poll: unknown ticket");
  *done = it->second.done ? 1 : 0;
  if (!*done) return UHNSW_OK;
  const int st = take_result(s, ticket, ids, dist, nullptr);
  return st == 0 ? UHNSW_OK : fail(st, "uhnsw_server_poll: request failed (%d)", st);
}

extern "C" int uhnsw_server_wait(uhnsw_server* s, uint64_t ticket, int64_t* ids, float* dist,
                                 int32_t timeout_ms) {
  clear_error();
  if (!s) return fail(UHNSW_EINVAL, "uhnsw_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(UHNSW_EINVAL, "uhnsw_server_wait: unknown ticket");
  // find(), not operator[]: another caller may release the ticket meanwhile
  auto finished_or_gone = [&] {
    auto jt = s->reqs.find(ticket);
    return jt == s->reqs.end() || jt->second.done;
  };
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished_or_gone);
  if (!ok) return fail(UHNSW_ETIMEOUT, "uhnsw_server_wait: not done after %d ms", timeout_ms);
  if (s->reqs.find(ticket) == s->reqs.end())
    return fail(UHNSW_EINVAL, "uhnsw_server_wait: ticket released by another call");
  const int st = take_result(s, ticket, ids, dist, nullptr);
  return st == 0 ? UHNSW_OK : fail(st, "uhnsw_server_wait: request failed (%d)", st);
}

extern "C" int uhnsw_server_replay(uhnsw_server* s, const float* q, const float* p,
                                   const int32_t* k, const int32_t* ef, int64_t nq,
                                   const double* arrival_us, int64_t* out_ids, float* out_dist,
                                   double* latency_us, int32_t timeout_ms) {
  clear_error();
  if (!s || !q || !p || !k || !ef || !arrival_us || nq < 0)
    return fail(UHNSW_EINVAL, "uhnsw_server_replay: NULL argument");
  std::vector<uint64_t> tickets(nq);
  const auto t0 = Clock::now();
  for (int64_t i = 0; i < nq; ++i) {
    const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                              std::chrono::duration<double, std::micro>(arrival_us[i]));
    while (Clock::now() < due) {
      if (due - Clock::now() > std::chrono::microseconds(200))
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    const int rc = uhnsw_server_submit(s, q + i * s->d, p[i], k[i], ef[i], &tickets[i]);
    if (rc != UHNSW_OK) return rc;
  }
  const int kmax = s->o.k_max;
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  std::unique_lock<std::mutex> lk(s->mu);
  for (int64_t i = 0; i < nq; ++i) {
    const uint64_t tk = tickets[i];
    const bool ok = s->cv_done.wait_until(lk, deadline, [&] {
      auto jt = s->reqs.find(tk);
      return jt == s->reqs.end() || jt->second.done;
    });
    if (!ok) return fail(UHNSW_ETIMEOUT, "uhnsw_server_replay: request %lld not done", (long long)i);
    if (s->reqs.find(tk) == s->reqs.end())
      return fail(UHNSW_EINVAL, "uhnsw_server_replay: request %lld released by another call",
                  (long long)i);
    for (int j = k[i]; j < kmax; ++j) {
      if (out_ids) out_ids[i * kmax + j] = -1;
      if (out_dist) out_dist[i * kmax + j] = __builtin_huge_valf();
    }
    const int st = take_result(s, tickets[i], out_ids ? out_ids + i * kmax : nullptr,
                               out_dist ? out_dist + i * kmax : nullptr,
                               latency_us ? latency_us + i : nullptr);
    if (st != 0) return fail(st, "uhnsw_server_replay: request %lld failed (%d)", (long long)i, st);
  }
  return UHNSW_OK;
}

extern "C" int uhnsw_server_stats(uhnsw_server* s, uhnsw_server_report* out) {
  clear_error();
  if (!s || !out) return fail(UHNSW_EINVAL, "uhnsw_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->batches = s->batches;
  out->mean_batch = s->batches ? (double)s->batched_queries / (double)s->batches : 0.0;
  out->peak_inflight = s->peak_inflight;
  out->peak_state = s->peak_state;
  if (!s->lat_us.empty()) {
    std::vector<double> v = s->lat_us;
    std::sort(v.begin(), v.end());
    auto pct = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_us = sum / (double)v.size();
    out->max_us = v.back();
  }
  out->error = s->error;
  return UHNSW_OK;
}

extern "C" void uhnsw_server_destroy(uhnsw_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->dispatcher.joinable()) s->dispatcher.join();
  if (s->completer.joinable()) s->completer.join();
  for (auto& L : s->lanes) {
    if (L.busy && L.launched) cudaEventSynchronize(L.event);
    free_lane(L);
  }
  delete s;
}
