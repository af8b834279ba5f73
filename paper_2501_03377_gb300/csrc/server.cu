// Request server with continuous batching (tpcg_server_*).
//
// One worker thread owns the device work.  Requests wait in a FIFO queue and
// are admitted as soon as fewer than max_slots solves run and device memory is free; every
// admitted solve is a SolveJob on its own plan and stream, so solves of
// different sizes and boundary conditions overlap on the GPU while new ones
// keep arriving.  Plans (eigenbases and workspaces) are cached by (grid, BCs,
// spacing, precision) and evicted least-recently-used when idle and memory is
// needed.  A session keeps its last solution on the device and its next
// request starts from it (warm start), so the requests of one session are run
// in submission order; requests of different sessions are independent.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "tpcg_dev.cuh"

namespace tpcg {
namespace {

using Clock = std::chrono::steady_clock;

struct PlanKey {
  int nx, ny, nz, prec;
  int bc[3];
  double h[3];
  bool operator<(const PlanKey& o) const {
    return std::memcmp(this, &o, sizeof(PlanKey)) < 0;
  }
};

PlanKey make_key(const tpcg_request& r) {
  PlanKey k;
  std::memset(&k, 0, sizeof(k));
  k.nx = r.nx;
  k.ny = r.ny;
  k.nz = r.nz;
  k.prec = r.prec;
  const int naxes = (r.nz == 1) ? 2 : 3;
  for (int m = 0; m < 3; ++m) {
    k.bc[m] = (m < naxes) ? r.bc[m] : 0;
    k.h[m] = (m < naxes) ? r.h[m] : 1.0;
  }
  return k;
}

struct Request {
  unsigned long long ticket = 0;
  tpcg_request req{};
  const double* eta_borrowed = nullptr;  // caller's buffer (TPCG_REQ_BORROW_*)
  PlanKey key{};
  double* eta_host = nullptr;  // pinned copy of eta
  double* ups_host = nullptr;  // pinned result
  long long N = 0;
  Clock::time_point t_submit, t_done;
  Clock::time_point t_admit, t_started, t_solved;  // admitted; plan ready and solve enqueued; solution on device
  bool admitted = false, solved = false;
  int plan_built = 0;  // the plan was created for this request (not found idle in the cache)
  int status = TPCG_PENDING;
  tpcg_info info{};
};

struct Slot {
  tpcg_plan* plan = nullptr;
  PlanKey key{};
  cudaStream_t stream = nullptr;
  double* d_eta = nullptr;
  double* d_ups = nullptr;  // used when the request has no session
  size_t bytes = 0;         // plan + buffers
  Request* req = nullptr;   // running request (nullptr: idle, cached)
  SolveJob job;
  int stage = 0;            // 0 idle, 1 solving, 2 copying the result back
  cudaEvent_t ev = nullptr;
  Clock::time_point last_used;
};

struct Session {
  double* d_ups = nullptr;
  long long N = 0;
  PlanKey key{};
  bool has_solution = false;
  size_t bytes = 0;
};

}  // namespace
}  // namespace tpcg

struct tpcg_server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool shutdown = false;
  std::thread worker;
  unsigned long long next_ticket = 1;
  std::deque<tpcg::Request*> queue;                       // waiting, in arrival order
  std::map<unsigned long long, tpcg::Request*> requests;  // every unreleased request
  std::list<tpcg::Slot> slots;
  std::map<unsigned long long, tpcg::Session> sessions;
  std::map<unsigned long long, int> session_pending;      // requests of a session not yet finished
  size_t used = 0;
  unsigned long long submitted = 0, completed = 0, failed = 0, rejected = 0;
  std::vector<double> latencies_ms;
  std::vector<tpcg_request_timing> timings;  // one record per finished request since the last reset
  std::multimap<size_t, void*> pinned_pool;  // released pinned host buffers, by size
  tpcg::Clock::time_point t_first, t_last_done;
  bool have_first = false;
};

namespace tpcg {
namespace {

// Pinned host buffers are recycled: allocating or freeing pinned memory can
// synchronise the device, which would stall every running solve.
double* pinned_get(tpcg_server* s, size_t bytes) {
  auto it = s->pinned_pool.find(bytes);
  if (it != s->pinned_pool.end()) {
    void* p = it->second;
    s->pinned_pool.erase(it);
    return static_cast<double*>(p);
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<double*>(p);
}

void pinned_put(tpcg_server* s, size_t bytes, void* p) {
  if (p) s->pinned_pool.emplace(bytes, p);
}

// Device bytes a plan of this key will hold, plus the slot's eta/ups buffers
// (upper estimate matching tpcg_plan_create's allocations).
size_t estimate_slot_bytes(const PlanKey& k) {
  const size_t N = (size_t)k.nx * k.ny * k.nz;
  const bool fp64 = (k.prec == TPCG_FP64);
  // bytes of a tensor-core operand (TF32: FP32 containers; split: hi and lo BF16 planes)
  const size_t lpb = (k.prec == TPCG_MIXED_TF32 || k.prec == TPCG_MIXED_BF16X3) ? 4 : 2;
  size_t b = N * 8 + (fp64 ? N * 8 * 3 : N * 4 * 2);  // R; P[2] and W (FP64) or P[2] in int32
  b += N * (fp64 ? 8 : 4);                   // Z
  b += fp64 ? 0 : N * lpb + (size_t)k.ny * k.nz * 8 * lpb;  // low-precision copy of R (padded rows)
  b += 2 * N * (fp64 ? 8 : lpb) + 2 * (size_t)(k.nx + k.ny + k.nz) * 64;  // mode-product intermediates
  const size_t l2 = (size_t)k.nx * k.nx + (size_t)k.ny * k.ny + (size_t)k.nz * k.nz;
  b += l2 * (16 + (fp64 ? 0 : 4 * lpb));     // eigenbases
  b += (1 << 20) + 16384 * 4 * 8;            // state, partial sums, slack
  b += N * 8 * 2;                            // slot's eta / ups buffers
  return b;
}

void release_slot(tpcg_server* s, std::list<Slot>::iterator it) {
  if (it->plan) tpcg_plan_destroy(it->plan);
  cudaFree(it->d_eta);
  cudaFree(it->d_ups);
  if (it->stream) cudaStreamDestroy(it->stream);
  if (it->ev) cudaEventDestroy(it->ev);
  s->used -= it->bytes;
  s->slots.erase(it);
}

// Evict least-recently-used idle slots until `need` more bytes fit.
bool make_room(tpcg_server* s, size_t need) {
  while (s->used + need > s->budget) {
    auto victim = s->slots.end();
    for (auto it = s->slots.begin(); it != s->slots.end(); ++it)
      if (!it->req && (victim == s->slots.end() || it->last_used < victim->last_used)) victim = it;
    if (victim == s->slots.end()) return false;
    release_slot(s, victim);
  }
  return true;
}

int running_slots(const tpcg_server* s) {
  int n = 0;
  for (const auto& sl : s->slots) n += sl.req ? 1 : 0;
  return n;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

constexpr size_t kMaxTimingRecords = 1u << 20;

void finish_request(tpcg_server* s, Request* r, int status) {
  r->status = status;
  r->t_done = Clock::now();
  s->t_last_done = r->t_done;
  const double ms = ms_between(r->t_submit, r->t_done);
  s->latencies_ms.push_back(ms);
  if (s->timings.size() < kMaxTimingRecords) {
    tpcg_request_timing t;
    std::memset(&t, 0, sizeof(t));
    t.ticket = r->ticket;
    t.session = r->req.session;
    t.nx = r->req.nx;
    t.ny = r->req.ny;
    t.nz = r->req.nz;
    t.prec = r->req.prec;
    t.status = status;
    t.iters = r->info.iters;
    t.plan_built = r->plan_built;
    const Clock::time_point ta = r->admitted ? r->t_admit : r->t_done;
    const Clock::time_point tb = r->admitted ? r->t_started : r->t_done;
    const Clock::time_point tc = r->solved ? r->t_solved : r->t_done;
    t.queue_ms = ms_between(r->t_submit, ta);
    t.build_ms = ms_between(ta, tb);
    t.solve_ms = r->admitted ? ms_between(tb, tc) : 0.0;
    t.copy_ms = r->solved ? ms_between(tc, r->t_done) : 0.0;
    t.total_ms = ms;
    s->timings.push_back(t);
  }
  if (status == TPCG_OK) ++s->completed;
  else ++s->failed;
  if (r->req.session) {
    auto it = s->session_pending.find(r->req.session);
    if (it != s->session_pending.end() && --it->second <= 0) s->session_pending.erase(it);
  }
  pinned_put(s, (size_t)r->N * 8, r->eta_host);
  r->eta_host = nullptr;
  s->cv_done.notify_all();
}

// Try to start `r`: find or build a slot and session storage; false if it must wait.
bool try_admit(tpcg_server* s, Request* r, bool* reject) {
  *reject = false;
  // an idle cached slot with the same plan key
  auto slot = s->slots.end();
  for (auto it = s->slots.begin(); it != s->slots.end(); ++it)
    if (!it->req && !(it->key < r->key) && !(r->key < it->key)) {
      slot = it;
      break;
    }
  Session* ses = nullptr;
  size_t ses_need = 0;
  if (r->req.session) {
    auto sit = s->sessions.find(r->req.session);
    if (sit == s->sessions.end() || sit->second.N != r->N) ses_need = (size_t)r->N * 8;
    else ses = &sit->second;
  }
  const size_t slot_need = (slot == s->slots.end()) ? estimate_slot_bytes(r->key) : 0;
  if (slot != s->slots.end()) slot->req = r;  // reserved: not an eviction candidate
  auto unreserve = [&]() {
    if (slot != s->slots.end()) slot->req = nullptr;
  };
  if (slot_need + ses_need > s->budget) {
    unreserve();
    *reject = true;  // can never fit
    return false;
  }
  if (!make_room(s, slot_need + ses_need)) {  // wait for running solves
    unreserve();
    return false;
  }
  r->t_admit = Clock::now();
  r->admitted = true;
  r->plan_built = 0;
  if (ses_need) {
    auto sit = s->sessions.find(r->req.session);
    if (sit != s->sessions.end()) {  // grid changed: drop the old solution
      cudaFree(sit->second.d_ups);
      s->used -= sit->second.bytes;
      s->sessions.erase(sit);
    }
    Session ns;
    if (cudaMalloc((void**)&ns.d_ups, ses_need) != cudaSuccess) {
      cudaGetLastError();
      unreserve();
      r->admitted = false;
      return false;
    }
    ns.N = r->N;
    ns.key = r->key;
    ns.bytes = ses_need;
    s->used += ses_need;
    ses = &(s->sessions[r->req.session] = ns);
  }
  if (slot == s->slots.end()) {
    r->plan_built = 1;
    Slot ns;
    ns.key = r->key;
    if (cudaStreamCreateWithFlags(&ns.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ns.ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (ns.stream) cudaStreamDestroy(ns.stream);
      return false;
    }
    const int rc = tpcg_plan_create(r->req.nx, r->req.ny, r->req.nz, r->key.bc, r->key.h, r->req.prec, ns.stream,
                                    &ns.plan);
    if (rc != TPCG_OK) {
      cudaStreamDestroy(ns.stream);
      cudaEventDestroy(ns.ev);
      if (rc == TPCG_ERR_OOM) return false;
      *reject = true;
      return false;
    }
    if (cudaMalloc((void**)&ns.d_eta, (size_t)r->N * 8) != cudaSuccess ||
        cudaMalloc((void**)&ns.d_ups, (size_t)r->N * 8) != cudaSuccess) {
      cudaGetLastError();
      tpcg_plan_destroy(ns.plan);
      cudaFree(ns.d_eta);
      cudaStreamDestroy(ns.stream);
      cudaEventDestroy(ns.ev);
      return false;
    }
    size_t pb = 0;
    tpcg_plan_device_bytes(ns.plan, &pb);
    ns.bytes = pb + (size_t)r->N * 16;
    s->used += ns.bytes;
    s->slots.push_back(ns);
    slot = std::prev(s->slots.end());
  }
  // start the solve
  r->t_started = Clock::now();
  Slot& sl = *slot;
  sl.req = r;
  sl.last_used = Clock::now();
  sl.stage = 1;
  double* ups = ses ? ses->d_ups : sl.d_ups;
  const bool warm = ses && ses->has_solution;
  const double* eta_src = r->eta_borrowed ? r->eta_borrowed : r->eta_host;
  const double* eta_dev = sl.d_eta;
  cudaError_t ce = cudaSuccess;
  if (r->req.flags & TPCG_REQ_BORROW_DEVICE)
    eta_dev = eta_src;  // read in place: the solve never writes eta
  else
    ce = cudaMemcpyAsync(sl.d_eta, eta_src, (size_t)r->N * 8, cudaMemcpyHostToDevice, sl.stream);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    sl.req = nullptr;
    sl.stage = 0;
    finish_request(s, r, TPCG_ERR_CUDA);
    return true;
  }
  SolveJob j;
  j.p = sl.plan;
  j.eta = eta_dev;
  j.ups = ups;
  j.tol = r->req.tol;
  j.maxit = r->req.maxit;
  j.flags = warm ? 0u : TPCG_ZERO_GUESS;
  sl.job = j;
  const int rc = job_start(sl.job);
  if (rc) {
    sl.req = nullptr;
    sl.stage = 0;
    finish_request(s, r, rc);
  }
  return true;
}

void worker_main(tpcg_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (true) {
    bool progressed = false;
    if (s->shutdown) {  // queued requests are cancelled; running ones finish
      while (!s->queue.empty()) {
        Request* r = s->queue.front();
        s->queue.pop_front();
        finish_request(s, r, TPCG_ERR_CANCELLED);
      }
    }
    // admission: first admissible request in arrival order (a session's requests stay in order)
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      Request* r = *it;
      bool blocked = false;
      if (r->req.session) {
        for (auto jt = s->queue.begin(); jt != it; ++jt)
          if ((*jt)->req.session == r->req.session) blocked = true;
        for (const auto& sl : s->slots)
          if (sl.req && sl.req->req.session == r->req.session) blocked = true;
      }
      if (blocked || running_slots(s) >= s->max_slots) {
        ++it;
        continue;
      }
      bool reject = false;
      if (try_admit(s, r, &reject)) {
        it = s->queue.erase(it);
        progressed = true;
      } else if (reject) {
        it = s->queue.erase(it);
        ++s->rejected;
        finish_request(s, r, TPCG_ERR_ADMISSION);
        progressed = true;
      } else {
        break;  // wait for memory or a slot; keep arrival order
      }
    }
    // progress every running solve
    for (auto& sl : s->slots) {
      if (!sl.req) continue;
      if (sl.stage == 1 && job_ready(sl.job)) {
        progressed = true;
        int rc = job_step(sl.job);
        if (rc == TPCG_OK && sl.job.phase == 3) {
          Request* r = sl.req;
          r->info = sl.job.info;
          r->t_solved = Clock::now();
          r->solved = true;
          if (cudaMemcpyAsync(r->ups_host, sl.job.ups, (size_t)r->N * 8, cudaMemcpyDeviceToHost, sl.stream) !=
                  cudaSuccess ||
              cudaEventRecord(sl.ev, sl.stream) != cudaSuccess)
            rc = TPCG_ERR_CUDA;
          else
            sl.stage = 2;
        }
        if (rc != TPCG_OK) {
          cudaGetLastError();
          Request* r = sl.req;
          sl.req = nullptr;
          sl.stage = 0;
          finish_request(s, r, rc);
        }
      } else if (sl.stage == 2 && cudaEventQuery(sl.ev) != cudaErrorNotReady) {
        progressed = true;
        Request* r = sl.req;
        if (r->req.session) {
          auto sit = s->sessions.find(r->req.session);
          if (sit != s->sessions.end()) sit->second.has_solution = (sl.job.status == TPCG_OK);
        }
        sl.req = nullptr;
        sl.stage = 0;
        sl.last_used = Clock::now();
        finish_request(s, r, sl.job.status);
      }
    }
    if (s->shutdown && s->queue.empty() && running_slots(s) == 0) break;
    if (!progressed) {
      if (running_slots(s) > 0) {
        lock.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lock.lock();
      } else {
        s->cv_work.wait_for(lock, std::chrono::milliseconds(5));
      }
    }
  }
}

}  // namespace
}  // namespace tpcg

using namespace tpcg;

extern "C" {

int tpcg_server_create(size_t hbm_budget, int max_slots, tpcg_server** out) {
  if (!out || max_slots < 1) return TPCG_ERR_INVALID_ARG;
  *out = nullptr;
  tpcg_server* s = new (std::nothrow) tpcg_server();
  if (!s) return TPCG_ERR_OOM;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return TPCG_ERR_CUDA;
  }
  if (hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return TPCG_ERR_CUDA;
    }
    hbm_budget = (size_t)(0.9 * (double)fr);
  }
  s->budget = hbm_budget;
  s->max_slots = max_slots;
  s->worker = std::thread(worker_main, s);
  *out = s;
  return TPCG_OK;
}

int tpcg_server_submit(tpcg_server* s, const tpcg_request* req, unsigned long long* ticket) {
  if (!s || !req || !ticket || !req->eta) return TPCG_ERR_INVALID_ARG;
  if (req->nx < 3 || req->ny < 3 || !(req->nz == 1 || req->nz >= 3)) return TPCG_ERR_INVALID_ARG;
  if (!(req->tol > 0.0 && req->tol < 1.0) || req->maxit < 1) return TPCG_ERR_INVALID_ARG;
  const int naxes = (req->nz == 1) ? 2 : 3;
  for (int m = 0; m < naxes; ++m)
    if (req->bc[m] < 0 || req->bc[m] > 4 || !(req->h[m] > 0.0)) return TPCG_ERR_INVALID_ARG;
  const Clock::time_point t_call = Clock::now();  // latency is counted from the submit call
  Request* r = new (std::nothrow) Request();
  if (!r) return TPCG_ERR_OOM;
  r->req = *req;
  r->req.eta = nullptr;
  r->key = make_key(*req);
  r->N = (long long)req->nx * req->ny * req->nz;
  const size_t bytes = (size_t)r->N * 8;
  std::unique_lock<std::mutex> lock(s->mu);
  if (s->shutdown) {
    delete r;
    return TPCG_ERR_INVALID_ARG;
  }
  const bool borrow = (req->flags & (TPCG_REQ_BORROW_HOST | TPCG_REQ_BORROW_DEVICE)) != 0;
  r->eta_host = borrow ? nullptr : pinned_get(s, bytes);
  r->ups_host = pinned_get(s, bytes);
  if ((!borrow && !r->eta_host) || !r->ups_host) {
    pinned_put(s, bytes, r->eta_host);
    pinned_put(s, bytes, r->ups_host);
    delete r;
    return TPCG_ERR_OOM;
  }
  if (borrow) {
    r->eta_borrowed = req->eta;
  } else {
    lock.unlock();
    std::memcpy(r->eta_host, req->eta, bytes);  // outside the lock: the worker keeps running
    lock.lock();
  }
  r->ticket = s->next_ticket++;
  r->t_submit = t_call;
  if (!s->have_first) {
    s->t_first = r->t_submit;
    s->have_first = true;
  }
  if (req->session) s->session_pending[req->session] += 1;
  s->requests[r->ticket] = r;
  s->queue.push_back(r);
  ++s->submitted;
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return TPCG_OK;
}

static int take_result(tpcg_server* s, std::map<unsigned long long, Request*>::iterator it, double* ups_out,
                       tpcg_info* info) {
  Request* r = it->second;
  if (ups_out && r->ups_host) std::memcpy(ups_out, r->ups_host, (size_t)r->N * 8);
  if (info) {
    *info = r->info;
    info->status = r->status;
  }
  const int st = r->status;
  pinned_put(s, (size_t)r->N * 8, r->ups_host);
  s->requests.erase(it);
  delete r;
  return st;
}

int tpcg_server_poll(tpcg_server* s, unsigned long long ticket, double* ups_out, tpcg_info* info) {
  if (!s) return TPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return TPCG_ERR_UNKNOWN_TICKET;
  if (it->second->status == TPCG_PENDING) return TPCG_PENDING;
  return take_result(s, it, ups_out, info);
}

int tpcg_server_wait(tpcg_server* s, unsigned long long ticket, double timeout_s, double* ups_out, tpcg_info* info) {
  if (!s) return TPCG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return TPCG_ERR_UNKNOWN_TICKET;
  Request* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s);
  while (r->status == TPCG_PENDING) {
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && r->status == TPCG_PENDING)
      return TPCG_PENDING;
  }
  return take_result(s, s->requests.find(ticket), ups_out, info);
}

int tpcg_server_get_stats(tpcg_server* s, tpcg_server_stats* out) {
  if (!s || !out) return TPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->rejected = s->rejected;
  out->queued = (int)s->queue.size();
  out->running = running_slots(s);
  out->device_bytes = s->used;
  std::vector<double> l = s->latencies_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
      const double x = p * (double)(l.size() - 1);
      const size_t i = (size_t)x;
      const double f = x - (double)i;
      return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double v : l) sum += v;
    out->mean_ms = sum / (double)l.size();
  }
  if (s->have_first && (s->completed + s->failed) > 0)
    out->elapsed_s = std::chrono::duration<double>(s->t_last_done - s->t_first).count();
  return TPCG_OK;
}

int tpcg_server_get_timings(tpcg_server* s, tpcg_request_timing* out, int max_records, int* n_records) {
  if (!s || !n_records || max_records < 0 || (max_records > 0 && !out)) return TPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  const int n = (int)std::min<size_t>(s->timings.size(), (size_t)max_records);
  if (n > 0) std::memcpy(out, s->timings.data(), sizeof(tpcg_request_timing) * (size_t)n);
  *n_records = max_records == 0 ? (int)s->timings.size() : n;
  return TPCG_OK;
}

int tpcg_server_reset_stats(tpcg_server* s) {
  if (!s) return TPCG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  s->latencies_ms.clear();
  s->timings.clear();
  s->submitted = s->completed = s->failed = s->rejected = 0;
  s->have_first = false;
  return TPCG_OK;
}

int tpcg_server_destroy(tpcg_server* s) {
  if (!s) return TPCG_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->shutdown = true;
    s->cv_work.notify_all();
  }
  s->worker.join();
  cudaSetDevice(s->device);
  while (!s->slots.empty()) release_slot(s, s->slots.begin());
  for (auto& kv : s->sessions) cudaFree(kv.second.d_ups);
  for (auto& kv : s->requests) {
    cudaFreeHost(kv.second->eta_host);
    cudaFreeHost(kv.second->ups_host);
    delete kv.second;
  }
  for (auto& kv : s->pinned_pool) cudaFreeHost(kv.second);
  delete s;
  return TPCG_OK;
}

}  // extern "C"
