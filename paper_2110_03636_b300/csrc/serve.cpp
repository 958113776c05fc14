// Request server: continuous batching of KKT solves over resident patterns
// (the serving form of the method: analysis once per pattern, then value
// refactorizations and solves, Sec. 2). See kkt_server_* in kkt.h.
//
// Each pattern keeps its host analysis and a list of slots (device handles
// made from that analysis with kkt_analyse_like, each with its own stream).
// Worker threads (max_inflight of them) take requests from the pending list
// in arrival order: the first request whose pattern has an idle slot, or
// whose new slot fits the HBM budget, starts; the others wait and do not
// block it. A slot is used by one worker at a time (a handle is not thread
// safe), so concurrent requests run on separate streams and overlap.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <shared_mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kkt.h"

namespace {

struct Slot {
  kkt_handle h = nullptr;
  cudaStream_t st = nullptr;
  bool busy = false;
  int64_t bytes = 0;        // device bytes accounted for this slot
  int32_t index = 0;
};

struct Pattern {
  kkt_handle host = nullptr;   // analysis only (no device memory)
  std::vector<Slot*> slots;
  int64_t slot_bytes = 0;      // bytes a new slot is expected to take
  int64_t n = 0, m = 0;
};

struct Req {
  int64_t id = 0;
  int32_t pattern = 0;
  const double *H = nullptr, *J = nullptr, *rx = nullptr, *ry = nullptr;
  double *dx = nullptr, *dy = nullptr;
  double delta = 0, gamma = 0;
  kkt_request_info info{};
  bool done = false;
};

// Refinement workspace a slot allocates at its first solve (flexible GMRES
// basis and directions, N = n + m): counted before it exists.
int64_t workspace_estimate(const Pattern& p) { return (int64_t)8 * (p.n + p.m) * 48; }

}  // namespace

struct kkt_server_s {
  kkt_options opt;
  int64_t budget = 0, used = 0, peak = 0;
  int32_t max_inflight = 1;
  std::vector<Pattern*> pats;   // stable addresses: workers hold them outside the lock
  std::deque<Req*> pending;
  std::unordered_map<int64_t, Req*> reqs;
  std::mutex mu;
  std::shared_mutex exclusive;   // held shared while a request runs, exclusively by a retry
  std::condition_variable cv_work, cv_done;
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_id = 0, submitted = 0, completed = 0, failed = 0;
  int32_t inflight = 0, peak_inflight = 0;
  std::chrono::steady_clock::time_point t0;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

// New slot of pattern p (device handle from the pattern's analysis + stream).
kkt_status make_slot(kkt_server s, Pattern& p, Slot** out) {
  Slot* sl = new (std::nothrow) Slot();
  if (!sl) return KKT_ERR_OOM;
  kkt_status st = kkt_analyse_like(p.host, &s->opt, &sl->h);
  if (st == KKT_OK && cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = KKT_ERR_CUDA;
  }
  if (st != KKT_OK) {
    if (sl->h) kkt_destroy(sl->h);
    delete sl;
    return st;
  }
  kkt_symbolic_info si;
  kkt_symbolic_info_get(sl->h, &si);
  sl->bytes = (int64_t)si.device_bytes + workspace_estimate(p);
  *out = sl;
  return KKT_OK;
}

// Under the lock: the first pending request that can start, with its slot
// (an idle one) or a budget reservation for a new one (*create).
bool pick(kkt_server s, Req** r, Slot** slot, bool* create) {
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
    Pattern& p = *s->pats[(*it)->pattern];
    for (Slot* sl : p.slots)
      if (!sl->busy) {
        sl->busy = true;
        *r = *it;
        *slot = sl;
        *create = false;
        s->pending.erase(it);
        return true;
      }
    if (s->used + p.slot_bytes <= s->budget) {
      s->used += p.slot_bytes;
      s->peak = std::max(s->peak, s->used);
      *r = *it;
      *slot = nullptr;
      *create = true;
      s->pending.erase(it);
      return true;
    }
  }
  return false;
}

void worker(kkt_server s) {
  cudaSetDevice(s->opt.device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    Req* r = nullptr;
    Slot* sl = nullptr;
    bool create = false;
    s->cv_work.wait(lk, [&] { return s->stop || pick(s, &r, &sl, &create); });
    if (!r) {
      if (s->stop && s->pending.empty()) return;
      continue;
    }
    s->inflight++;
    s->peak_inflight = std::max(s->peak_inflight, s->inflight);
    Pattern& p = *s->pats[r->pattern];
    const int64_t reserved = create ? p.slot_bytes : 0;
    lk.unlock();
    kkt_status st = KKT_OK;
    if (create) st = make_slot(s, p, &sl);
    r->info.t_start = s->now();
    if (st == KKT_OK) {
      {
        std::shared_lock<std::shared_mutex> run_lk(s->exclusive);
        st = kkt_factor(sl->h, r->H, r->J, r->delta, r->gamma, sl->st);
        if (st == KKT_OK) st = kkt_solve(sl->h, r->rx, r->ry, r->dx, r->dy, sl->st);
      }
      if (st == KKT_ERR_TIMEOUT) {
        // a bounded wait ran out while other requests' kernels were resident
        // (the persistent solve kernel needs all its CTAs on the device at
        // once): run the request again with nothing else in flight
        std::unique_lock<std::shared_mutex> alone(s->exclusive);
        st = kkt_factor(sl->h, r->H, r->J, r->delta, r->gamma, sl->st);
        if (st == KKT_OK) st = kkt_solve(sl->h, r->rx, r->ry, r->dx, r->dy, sl->st);
        r->info.retried = 1;
      }
      kkt_info inf{};
      kkt_get_info(sl->h, &inf);
      r->info.cg_iters = inf.cg_iters;
      r->info.ir_steps = inf.ir_steps;
      r->info.rr = inf.rr;
      r->info.be = inf.be;
    }
    r->info.t_end = s->now();
    r->info.status = st;
    lk.lock();
    if (create) {
      if (sl) {
        // account the slot at its measured size (its workspace now exists)
        kkt_symbolic_info si;
        kkt_symbolic_info_get(sl->h, &si);
        sl->bytes = std::max<int64_t>((int64_t)si.device_bytes, sl->bytes - workspace_estimate(p));
        s->used += sl->bytes - reserved;
        s->peak = std::max(s->peak, s->used);
        p.slot_bytes = std::max(p.slot_bytes, sl->bytes);
        sl->index = (int32_t)p.slots.size();
        p.slots.push_back(sl);
      } else {
        s->used -= reserved;
      }
    } else {
      kkt_symbolic_info si;
      kkt_symbolic_info_get(sl->h, &si);
      if ((int64_t)si.device_bytes > sl->bytes) {
        s->used += (int64_t)si.device_bytes - sl->bytes;
        s->peak = std::max(s->peak, s->used);
        sl->bytes = (int64_t)si.device_bytes;
        p.slot_bytes = std::max(p.slot_bytes, sl->bytes);
      }
    }
    if (sl) {
      sl->busy = false;
      r->info.slot = sl->index;
    }
    r->done = true;
    s->completed++;
    if (st != KKT_OK) s->failed++;
    s->inflight--;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

kkt_status kkt_server_create(int64_t budget_bytes, int32_t max_inflight, const kkt_options* opt, kkt_server* out) {
  if (!out || max_inflight < 1 || max_inflight > 64) return KKT_ERR_INVALID;
  *out = nullptr;
  kkt_server s = new (std::nothrow) kkt_server_s();
  if (!s) return KKT_ERR_OOM;
  if (opt) s->opt = *opt; else kkt_default_options(&s->opt);
  if (cudaSetDevice(s->opt.device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return KKT_ERR_CUDA;
  }
  if (budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return KKT_ERR_CUDA;
    }
    budget_bytes = (int64_t)(0.9 * (double)fr);
  }
  s->budget = budget_bytes;
  s->max_inflight = max_inflight;
  s->t0 = std::chrono::steady_clock::now();
  for (int k = 0; k < max_inflight; k++) s->workers.emplace_back(worker, s);
  *out = s;
  return KKT_OK;
}

kkt_status kkt_server_add_pattern(kkt_server s, int64_t n, int64_t m, const int64_t* H_colptr,
                                  const int32_t* H_rowidx, const int64_t* J_rowptr, const int32_t* J_colidx,
                                  int32_t* pattern_id) {
  if (!s || !pattern_id) return KKT_ERR_INVALID;
  Pattern* p = new (std::nothrow) Pattern();
  if (!p) return KKT_ERR_OOM;
  p->n = n;
  p->m = m;
  kkt_status st = kkt_analyse_host(n, m, H_colptr, H_rowidx, J_rowptr, J_colidx, &s->opt, &p->host);
  if (st) {
    delete p;
    return st;
  }
  Slot* sl = nullptr;
  if ((st = make_slot(s, *p, &sl))) {
    kkt_destroy(p->host);
    delete p;
    return st;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->used + sl->bytes > s->budget) {
    kkt_destroy(sl->h);
    cudaStreamDestroy(sl->st);
    delete sl;
    kkt_destroy(p->host);
    delete p;
    return KKT_ERR_OOM;
  }
  s->used += sl->bytes;
  s->peak = std::max(s->peak, s->used);
  p->slot_bytes = sl->bytes;
  p->slots.push_back(sl);
  *pattern_id = (int32_t)s->pats.size();
  s->pats.push_back(p);
  return KKT_OK;
}

kkt_status kkt_server_submit(kkt_server s, int32_t pattern_id, const double* H_vals, const double* J_vals,
                             double delta, double gamma, const double* r_x, const double* r_y, double* dx,
                             double* dy, int64_t* request_id) {
  if (!s || !request_id || !H_vals || !r_x || !dx) return KKT_ERR_INVALID;
  Req* r = new (std::nothrow) Req();
  if (!r) return KKT_ERR_OOM;
  r->H = H_vals; r->J = J_vals; r->rx = r_x; r->ry = r_y; r->dx = dx; r->dy = dy;
  r->delta = delta; r->gamma = gamma;
  std::lock_guard<std::mutex> lk(s->mu);
  if (pattern_id < 0 || pattern_id >= (int32_t)s->pats.size() || s->stop) {
    delete r;
    return KKT_ERR_INVALID;
  }
  if (s->pats[pattern_id]->m > 0 && (!J_vals || !r_y || !dy)) {
    delete r;
    return KKT_ERR_INVALID;
  }
  r->pattern = pattern_id;
  r->id = s->next_id++;
  r->info.pattern = pattern_id;
  r->info.slot = -1;
  r->info.t_submit = s->now();
  s->reqs[r->id] = r;
  s->pending.push_back(r);
  s->submitted++;
  *request_id = r->id;
  s->cv_work.notify_one();
  return KKT_OK;
}

kkt_status kkt_server_wait(kkt_server s, int64_t request_id, kkt_request_info* info) {
  if (!s) return KKT_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return KKT_ERR_INVALID;
  Req* r = it->second;
  s->cv_done.wait(lk, [&] { return r->done; });
  if (info) *info = r->info;
  s->reqs.erase(request_id);
  delete r;
  return KKT_OK;
}

kkt_status kkt_server_get_stats(kkt_server s, kkt_server_stats* o) {
  if (!s || !o) return KKT_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(o, 0, sizeof(*o));
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->failed = s->failed;
  o->bytes_used = s->used;
  o->bytes_peak = s->peak;
  o->budget = s->budget;
  o->patterns = (int32_t)s->pats.size();
  for (const Pattern* p : s->pats) o->slots += (int32_t)p->slots.size();
  o->inflight = s->inflight;
  o->peak_inflight = s->peak_inflight;
  o->waiting = (int32_t)s->pending.size();
  return KKT_OK;
}

kkt_status kkt_server_destroy(kkt_server s) {
  if (!s) return KKT_ERR_INVALID;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->pending.empty() && s->inflight == 0; });
    s->stop = true;
    s->cv_work.notify_all();
  }
  for (std::thread& t : s->workers) t.join();
  cudaSetDevice(s->opt.device);
  for (Pattern* p : s->pats) {
    for (Slot* sl : p->slots) {
      kkt_destroy(sl->h);
      cudaStreamDestroy(sl->st);
      delete sl;
    }
    kkt_destroy(p->host);
    delete p;
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return KKT_OK;
}

}  // extern "C"
