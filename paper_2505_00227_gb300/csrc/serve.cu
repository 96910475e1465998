// Retrieval server: a device-resident request loop over refactored fields.
//
// Requests (one field at a relative L-infinity bound, or the velocity
// magnitude of a field triplet at a relative QoI bound) are queued on submit
// and run by `max_slots` worker threads, each with its own CUDA stream and
// library context, so the kernels of several requests overlap on the GPU.
// A request is admitted as soon as a slot is free, none of its handles is in
// use by a running request (a handle's plane cache is its retrieval state),
// and the HBM budget has room for the plane caches it will fill; older
// requests that cannot start yet do not hold back younger ones that can.
// Plane caches of idle handles are evicted least-recently-used first when the
// budget is short.  Because a retrieval's selection is the shortest prefix of
// a bound-independent group sequence, a request's result does not depend on
// what ran before it or beside it; the cache only saves decoding.
//
// Budget accounting: resident stored bytes of every added field + plane caches
// held + the component scratch of running QoI requests.
//
// Host-side failure handling: a queued request can be cancelled, and with a
// queue deadline a request that could not start in time fails with
// HPMDR_ERR_TIMEOUT (workers wake at least every deadline to expire them).
// Neither touches a running request: nothing is ever stopped on the device.
//
// Only the public entry points of the library are used here.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/hpmdr.h"

namespace {

typedef std::chrono::steady_clock Clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct FieldState {
  uint64_t resident = 0, cache = 0, cache_max = 0;
  bool busy = false;
  uint64_t last_use = 0;  // admission counter of its last request
  uint64_t n = 0;         // values
};

struct Req {
  hpmdr_request r;
  uint64_t ticket;
  int nh;
  int state = 0;  // 0 queued, 1 running, 2 done
  hpmdr_status status = HPMDR_OK;
  hpmdr_retrieve_info info[4];
  double t_submit = 0, t_start = 0, t_done = 0;
  uint64_t scratch = 0;  // transient device bytes while running
};

}  // namespace

struct hpmdr_server {
  hpmdr_server_config cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  std::unordered_map<hpmdr_handle*, FieldState> fields;
  uint64_t next_ticket = 1, admissions = 0;
  uint64_t used = 0, peak = 0, evictions = 0, completed = 0, running = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::vector<hpmdr_ctx*> ctxs;

  void account(hpmdr_handle* h, FieldState& fs) {  // refresh h's cache bytes
    uint64_t r = 0, c = 0, m = 0;
    hpmdr_handle_memory(h, &r, &c, &m);
    used = used - fs.cache + c;
    fs.cache = c;
    fs.cache_max = m;
    peak = std::max(peak, used);
  }

  // bytes request q would add: caches of its handles not yet held, + scratch
  uint64_t need(const Req* q) const {
    uint64_t b = q->scratch;
    for (int i = 0; i < q->nh; i++) {
      const FieldState& fs = fields.at(q->r.h[i]);
      if (fs.cache < fs.cache_max) b += fs.cache_max - fs.cache;
    }
    return b;
  }

  bool idle(const Req* q) const {
    for (int i = 0; i < q->nh; i++)
      if (fields.at(q->r.h[i]).busy) return false;
    return true;
  }

  bool in_request(const Req* q, hpmdr_handle* h) const {
    for (int i = 0; i < q->nh; i++)
      if (q->r.h[i] == h) return true;
    return false;
  }

  // drop idle caches, least recently used first, until `want` more bytes fit
  bool make_room(const Req* q, uint64_t want, hpmdr_ctx* ctx) {
    while (used + want > cfg.hbm_budget) {
      hpmdr_handle* victim = nullptr;
      uint64_t oldest = ~0ull;
      for (auto& kv : fields) {
        const FieldState& fs = kv.second;
        if (fs.busy || fs.cache == 0 || in_request(q, kv.first)) continue;
        if (fs.last_use < oldest) oldest = fs.last_use, victim = kv.first;
      }
      if (!victim) return false;
      hpmdr_handle_drop_cache(ctx, victim);
      account(victim, fields[victim]);
      evictions++;
    }
    return true;
  }

  // a queued request leaves the queue without running (lock held)
  void finish_unrun(Req* q, hpmdr_status st) {
    q->status = st;
    q->state = 2;
    q->t_start = q->t_done = now_s();
    cv_done.notify_all();
  }

  // queued requests past their deadline fail with HPMDR_ERR_TIMEOUT (lock held)
  void expire() {
    if (!(cfg.queue_timeout_s > 0.0)) return;
    const double t = now_s();
    for (auto it = queue.begin(); it != queue.end();) {
      if (t - (*it)->t_submit > cfg.queue_timeout_s) {
        finish_unrun(*it, HPMDR_ERR_TIMEOUT);
        it = queue.erase(it);
      } else {
        ++it;
      }
    }
  }

  // first queued request that can start now (lock held)
  Req* admit(hpmdr_ctx* ctx) {
    expire();
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Req* q = *it;
      if (!idle(q)) continue;
      const uint64_t want = need(q);
      if (used + want > cfg.hbm_budget && !make_room(q, want, ctx)) continue;
      queue.erase(it);
      for (int i = 0; i < q->nh; i++) {  // reserve the caches the request will fill
        FieldState& fs = fields[q->r.h[i]];
        fs.busy = true;
        fs.last_use = ++admissions;
        used += fs.cache_max - std::min(fs.cache, fs.cache_max);
        fs.cache = std::max(fs.cache, fs.cache_max);
      }
      used += q->scratch;
      peak = std::max(peak, used);
      running++;
      q->state = 1;
      q->t_start = now_s();
      return q;
    }
    return nullptr;
  }

  void run(Req* q, hpmdr_ctx* ctx) {
    memset(q->info, 0, sizeof(q->info));
    if (q->r.kind == HPMDR_REQ_FIELD) {
      q->status = hpmdr_retrieve(ctx, q->r.h[0], q->r.rel_bound, q->r.out[0], 1, &q->info[0]);
    } else {
      q->status = hpmdr_retrieve_qoi_vmag(ctx, q->r.h, q->r.rel_bound, q->r.out, q->r.out_vmag, 1,
                                          q->info);
    }
    if (!cfg.keep_cache)  // the plain per-request path keeps nothing between requests
      for (int i = 0; i < q->nh; i++) hpmdr_handle_drop_cache(ctx, q->r.h[i]);
  }

  void worker(int w) {
    cudaSetDevice(device);
    hpmdr_ctx* ctx = ctxs[w];
    std::unique_lock<std::mutex> lock(mu);
    while (true) {
      Req* q = nullptr;
      while (!stop && !(q = admit(ctx))) {
        if (cfg.queue_timeout_s > 0.0)  // wake to expire requests nobody else would
          cv_work.wait_for(lock, std::chrono::duration<double>(cfg.queue_timeout_s));
        else
          cv_work.wait(lock);
      }
      if (!q) return;
      lock.unlock();
      run(q, ctx);
      cudaStreamSynchronize(streams[w]);
      const double t = now_s();
      lock.lock();
      q->t_done = t;
      q->state = 2;
      used -= q->scratch;
      running--;
      completed++;
      for (int i = 0; i < q->nh; i++) {
        FieldState& fs = fields[q->r.h[i]];
        fs.busy = false;
        account(q->r.h[i], fs);
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

extern "C" hpmdr_status hpmdr_server_create(hpmdr_ctx* ctx, const hpmdr_server_config* cfg,
                                            hpmdr_server** out) {
  if (!ctx || !cfg || !out || cfg->max_slots < 1 || cfg->max_slots > 64 || cfg->hbm_budget == 0 ||
      !(cfg->queue_timeout_s >= 0.0))
    return HPMDR_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<hpmdr_server> S(new hpmdr_server());
  S->cfg = *cfg;
  if (cudaGetDevice(&S->device) != cudaSuccess) return HPMDR_ERR_CUDA;
  hpmdr_status st = HPMDR_OK;
  for (int w = 0; w < cfg->max_slots && st == HPMDR_OK; w++) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    S->streams.push_back(s);
    hpmdr_ctx* c = nullptr;
    if ((st = hpmdr_ctx_create(&c, nullptr, nullptr, s)) == HPMDR_OK) S->ctxs.push_back(c);
  }
  if (st != HPMDR_OK) {
    for (hpmdr_ctx* c : S->ctxs) hpmdr_ctx_destroy(c);
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    return st;
  }
  for (int w = 0; w < cfg->max_slots; w++)
    S->workers.emplace_back([srv = S.get(), w]() { srv->worker(w); });
  *out = S.release();
  return HPMDR_OK;
}

extern "C" void hpmdr_server_destroy(hpmdr_server* S) {
  if (!S) return;
  {
    std::unique_lock<std::mutex> lock(S->mu);
    // requests still queued are dropped; running ones finish
    S->queue.clear();
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (hpmdr_ctx* c : S->ctxs) hpmdr_ctx_destroy(c);
  for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
  delete S;
}

extern "C" hpmdr_status hpmdr_server_add_field(hpmdr_server* S, hpmdr_ctx* ctx, hpmdr_handle* h) {
  if (!S || !ctx || !h) return HPMDR_ERR_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  if (S->fields.count(h)) return HPMDR_OK;
  hpmdr_status st = hpmdr_handle_compact(ctx, h);
  if (st != HPMDR_OK) return st;
  FieldState fs;
  uint64_t r = 0, c = 0, m = 0;
  if ((st = hpmdr_handle_memory(h, &r, &c, &m)) != HPMDR_OK) return st;
  int dtype = 0;
  uint64_t dims[3];
  hpmdr_handle_field_info(h, &dtype, dims, nullptr, nullptr, nullptr, nullptr);
  fs.n = dims[0] * dims[1] * dims[2];
  if (S->used + r + c > S->cfg.hbm_budget) return HPMDR_ERR_NOMEM;
  fs.resident = r;
  fs.cache = c;
  fs.cache_max = m;
  S->used += r + c;
  S->peak = std::max(S->peak, S->used);
  S->fields[h] = fs;
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_server_submit(hpmdr_server* S, const hpmdr_request* r,
                                            uint64_t* ticket) {
  if (!S || !r || !ticket || !(r->rel_bound >= 0.0)) return HPMDR_ERR_ARG;
  std::unique_ptr<Req> q(new Req());
  q->r = *r;
  q->t_submit = now_s();
  {
    std::unique_lock<std::mutex> lock(S->mu);
    if (r->kind == HPMDR_REQ_FIELD) {
      q->nh = 1;
      if (!r->h[0] || !r->out[0]) return HPMDR_ERR_ARG;
    } else if (r->kind == HPMDR_REQ_VMAG) {
      q->nh = 3;
      if (!r->out_vmag) return HPMDR_ERR_ARG;
    } else {
      return HPMDR_ERR_ARG;
    }
    uint64_t total_fixed = 0;
    for (auto& kv : S->fields) total_fixed += kv.second.resident;
    uint64_t caches = 0;
    for (int i = 0; i < q->nh; i++) {
      auto it = S->fields.find(r->h[i]);
      if (it == S->fields.end()) return HPMDR_ERR_ARG;  // not added to this server
      for (int j = 0; j < i; j++)
        if (r->h[j] == r->h[i]) return HPMDR_ERR_ARG;
      caches += it->second.cache_max;
    }
    if (r->kind == HPMDR_REQ_VMAG)  // components the caller does not keep
      for (int c = 0; c < 3; c++)
        if (!r->out[c]) q->scratch += 4 * S->fields[r->h[0]].n;
    // even with every other cache evicted this request would not fit
    if (total_fixed + caches + q->scratch > S->cfg.hbm_budget) return HPMDR_ERR_NOMEM;
    q->ticket = S->next_ticket++;
    *ticket = q->ticket;
    S->queue.push_back(q.get());
    S->reqs[q->ticket] = std::move(q);
  }
  S->cv_work.notify_one();
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_server_poll(hpmdr_server* S, uint64_t ticket, int wait,
                                          hpmdr_retrieve_info info[4], double times[3]) {
  if (!S) return HPMDR_ERR_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return HPMDR_ERR_ARG;
  Req* q = it->second.get();
  if (q->state == 0) S->expire();
  if (q->state != 2) {
    if (!wait) return HPMDR_ERR_BUSY;
    S->cv_done.wait(lock, [q]() { return q->state == 2; });
  }
  if (info) memcpy(info, q->info, sizeof(q->info));
  if (times) {
    times[0] = q->t_submit;
    times[1] = q->t_start;
    times[2] = q->t_done;
  }
  const hpmdr_status st = q->status;
  S->reqs.erase(it);
  return st;
}

extern "C" hpmdr_status hpmdr_server_cancel(hpmdr_server* S, uint64_t ticket) {
  if (!S) return HPMDR_ERR_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return HPMDR_ERR_ARG;
  Req* q = it->second.get();
  if (q->state != 0) return HPMDR_ERR_BUSY;  // started or done: it completes
  S->queue.erase(std::find(S->queue.begin(), S->queue.end(), q));
  S->finish_unrun(q, HPMDR_ERR_CANCELLED);
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_server_stats(hpmdr_server* S, uint64_t stats[6]) {
  if (!S || !stats) return HPMDR_ERR_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  stats[0] = S->used;
  stats[1] = S->peak;
  stats[2] = S->evictions;
  stats[3] = S->completed;
  stats[4] = S->queue.size();
  stats[5] = S->running;
  return HPMDR_OK;
}
