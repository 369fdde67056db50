// The serving loop (include/spca_server.h): one worker thread owns the sessions and all CUDA
// work; callers only queue requests. Each session runs on its own stream; the worker issues
// whatever is queued for every admitted session, folds one session's waiting row blocks into
// one launch of the pass, and polls events to complete requests. Closed sessions (and those
// reserved ahead of time) wait in a pool, keeping their device and pinned memory, so that an
// admission of the same shape is a reset of their state instead of a round of allocations.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "spca.h"
#include "spca_internal.cuh"
#include "spca_server.h"

namespace {

using Clock = std::chrono::steady_clock;

enum Kind { kOpen, kUpdate, kFinalize, kClose, kReserve };

struct Request {
  uint64_t ticket = 0;
  int kind = kUpdate;
  int32_t id = -1;
  const float* rows = nullptr;
  int64_t m = 0, ld = 0;
  double* sigma = nullptr;
  double* V = nullptr;
  int64_t n = 0;                // reserve: shape, math, footprint and number of sessions
  int k = 0, p = 0, math = 0, count = 0;
  size_t bytes = 0;
  Clock::time_point t_submit;
};

struct Inflight {
  cudaEvent_t ev = nullptr;
  int kind = kUpdate;
  std::vector<Request> reqs;
};

struct Slot {
  bool used = false;        // open and not yet closed by the caller (guarded by the server mutex)
  bool held = false;        // from open until the worker frees the slot (guarded by the server
                            // mutex): a slot closed by the caller stays held while the worker
                            // still has its requests, so open cannot hand it out again
  bool admitted = false;    // session created (worker)
  bool failed = false;
  spca_status fail_status = SPCA_OK;
  int64_t n = 0;
  int k = 0, p = 0, math = 0;
  uint64_t seed = 0;
  size_t bytes = 0;
  spca_session* s = nullptr;
  double* sig_dev = nullptr;
  double* V_dev = nullptr;
  double* res_host = nullptr;   // pinned: k sigma then n k V
  int* flags_host = nullptr;    // pinned
  std::deque<Request> queue;    // not yet issued (worker)
  std::deque<Inflight> inflight;
};

// A session out of service: its handle and result buffers, kept for the next admission of
// the same (n, k, p, math).
struct Pooled {
  int64_t n = 0;
  int k = 0, p = 0, math = 0;
  size_t bytes = 0;
  spca_session* s = nullptr;
  double* sig_dev = nullptr;
  double* V_dev = nullptr;
  double* res_host = nullptr;
  int* flags_host = nullptr;

  bool fits(const Slot& sl) const { return n == sl.n && k == sl.k && p == sl.p && math == sl.math; }
};

// Create the session and its result buffers; on failure, what was allocated stays in e.
spca_status create_session(Pooled& e, uint64_t seed, int32_t max_block_rows) {
  spca_options o;
  spca_default_options(&o);
  o.math = e.math;
  o.max_block_rows = max_block_rows;
  spca_status st = spca_create(e.n, e.k, e.p, seed, &o, &e.s);
  const size_t vbytes = sizeof(double) * static_cast<size_t>(e.n) * e.k;
  if (st == SPCA_OK && (cudaMalloc(&e.sig_dev, sizeof(double) * e.k) != cudaSuccess ||
                        cudaMalloc(&e.V_dev, vbytes) != cudaSuccess ||
                        cudaMallocHost(&e.res_host, sizeof(double) * e.k + vbytes) != cudaSuccess ||
                        cudaMallocHost(&e.flags_host, sizeof(int)) != cudaSuccess)) {
    cudaGetLastError();
    st = SPCA_E_NOMEM;
  }
  return st;
}

void free_session(spca_session* s, double* sig_dev, double* V_dev, double* res_host, int* flags_host) {
  if (s) spca_destroy(s);
  if (sig_dev) cudaFree(sig_dev);
  if (V_dev) cudaFree(V_dev);
  if (res_host) cudaFreeHost(res_host);
  if (flags_host) cudaFreeHost(flags_host);
}

void free_session(Pooled& e) { free_session(e.s, e.sig_dev, e.V_dev, e.res_host, e.flags_host); }

struct TicketState {
  bool done = false;
  spca_status st = SPCA_OK;
  std::string msg;   // what went wrong, for a failed request
};

// A completed request: its ticket, status and (when it failed) the reason, taken from the
// session that ran it at the time it failed.
struct Done {
  uint64_t ticket;
  spca_status st;
  std::string msg;
};

std::string reason(spca_session* s, spca_status st, const char* what) {
  char buf[320];
  const char* e = s ? spca_last_error(s) : "";
  std::snprintf(buf, sizeof(buf), "%s (status %d)%s%s", what, static_cast<int>(st), e[0] ? ": " : "", e);
  return buf;
}

// Latencies of the most recent kLatWindow completed requests of one kind (a ring, so a
// long-running server holds a bounded record).
constexpr size_t kLatWindow = size_t(1) << 20;
struct LatRing {
  std::vector<double> v;
  size_t next = 0;
  void add(double ms) {
    if (v.size() < kLatWindow) {
      v.push_back(ms);
    } else {
      v[next] = ms;
      next = (next + 1) % kLatWindow;
    }
  }
};

double pct(std::vector<double>& v, double q) {   // reorders v
  if (v.empty()) return 0.0;
  const size_t i = static_cast<size_t>(q * static_cast<double>(v.size() - 1) + 0.5);
  std::nth_element(v.begin(), v.begin() + static_cast<std::ptrdiff_t>(i), v.end());
  return v[i];
}

thread_local char g_srv_err[256] = "";

spca_status srv_fail(spca_status st, const char* msg) {
  std::snprintf(g_srv_err, sizeof(g_srv_err), "%s", msg);
  return st;
}

}  // namespace

struct spca_server {
  int device = 0;
  spca_server_options opt{};
  size_t budget = 0, in_use = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> incoming;
  std::vector<Slot> slots;
  std::unordered_map<uint64_t, TicketState> tickets;
  uint64_t next_ticket = 1;
  LatRing lat_update, lat_finalize;
  int64_t updates_done = 0, finalizes_done = 0, admitted = 0, waiting = 0;
  int64_t n_pooled = 0, from_pool = 0, created = 0;   // written by the worker under mu
  size_t pooled_bytes = 0;
  double rows_bytes = 0.0, active_s = 0.0;
  bool stop = false;
  std::deque<int32_t> admission;   // worker
  std::deque<Request> reserves;    // worker
  std::vector<Pooled> pool;        // worker: oldest first
  std::vector<cudaEvent_t> events;  // worker: free events
  std::thread worker;

  void run();
  bool admit(int32_t id);
  void release(Slot& sl, bool to_pool);
  spca_status reserve(const Request& r);
  void to_pool(Pooled e);
  void evict_oldest();
  void issue(int32_t id, std::vector<Done>& done);
  void complete(Slot& sl, Inflight& f, std::vector<Done>& done);
  cudaEvent_t event();
};

cudaEvent_t spca_server::event() {
  if (!events.empty()) {
    cudaEvent_t e = events.back();
    events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  return e;
}

void spca_server::to_pool(Pooled e) {
  pool.push_back(e);
  std::lock_guard<std::mutex> lock(mu);
  pooled_bytes += e.bytes;
  ++n_pooled;
}

void spca_server::evict_oldest() {
  Pooled e = pool.front();
  pool.erase(pool.begin());
  free_session(e);
  std::lock_guard<std::mutex> lock(mu);
  pooled_bytes -= e.bytes;
  --n_pooled;
}

bool spca_server::admit(int32_t id) {
  Slot& sl = slots[static_cast<size_t>(id)];
  Pooled e;
  bool have = false;
  // a pooled session of the same shape: no allocation, its state reset for the new seed
  size_t j = 0;
  while (j < pool.size() && !pool[j].fits(sl)) ++j;
  if (j < pool.size()) {
    e = pool[j];
    pool.erase(pool.begin() + static_cast<std::ptrdiff_t>(j));
    {
      std::lock_guard<std::mutex> lock(mu);
      pooled_bytes -= e.bytes;
      --n_pooled;
    }
    if (spca_reset(e.s, sl.seed) == SPCA_OK) {
      have = true;
    } else {
      free_session(e);   // not handed out again; a new session is made below
      e = Pooled();
    }
  }
  spca_status st = SPCA_OK;
  if (!have) {
    // room for a new session: pooled sessions of other shapes are freed first, oldest first
    while (in_use + pooled_bytes + sl.bytes > budget && !pool.empty()) evict_oldest();
    if (in_use + pooled_bytes + sl.bytes > budget) return false;
    e.n = sl.n; e.k = sl.k; e.p = sl.p; e.math = sl.math; e.bytes = sl.bytes;
    st = create_session(e, sl.seed, opt.max_block_rows);
  }
  sl.s = e.s;
  sl.sig_dev = e.sig_dev;
  sl.V_dev = e.V_dev;
  sl.res_host = e.res_host;
  sl.flags_host = e.flags_host;
  std::lock_guard<std::mutex> lock(mu);
  sl.admitted = true;
  in_use += sl.bytes;
  ++(have ? from_pool : created);
  if (st != SPCA_OK) {
    sl.failed = true;
    sl.fail_status = st;
  }
  return true;
}

// Sessions made ahead of time go straight to the pool; the budget bounds them as it bounds
// admitted sessions (a reservation frees no pooled session of another shape).
spca_status spca_server::reserve(const Request& r) {
  for (int c = 0; c < r.count; ++c) {
    if (in_use + pooled_bytes + r.bytes > budget) return SPCA_E_NOMEM;
    Pooled e;
    e.n = r.n; e.k = r.k; e.p = r.p; e.math = r.math; e.bytes = r.bytes;
    spca_status st = create_session(e, 0, opt.max_block_rows);
    // staging buffers that a first update would otherwise allocate on the worker
    if (st == SPCA_OK) st = spca::session_prepare_staging(e.s);
    if (st != SPCA_OK) {
      free_session(e);
      return st;
    }
    to_pool(e);
    std::lock_guard<std::mutex> lock(mu);
    ++created;
  }
  return SPCA_OK;
}

// A closed session that is still usable goes back to the pool with its memory; a failed one,
// and every session at shutdown, is freed.
void spca_server::release(Slot& sl, bool pool_it) {
  for (Inflight& f : sl.inflight)
    if (f.ev) events.push_back(f.ev);
  sl.inflight.clear();
  if (pool_it && sl.admitted && !sl.failed && sl.s) {
    Pooled e;
    e.n = sl.n; e.k = sl.k; e.p = sl.p; e.math = sl.math; e.bytes = sl.bytes;
    e.s = sl.s; e.sig_dev = sl.sig_dev; e.V_dev = sl.V_dev; e.res_host = sl.res_host; e.flags_host = sl.flags_host;
    to_pool(e);
  } else {
    free_session(sl.s, sl.sig_dev, sl.V_dev, sl.res_host, sl.flags_host);
  }
  std::lock_guard<std::mutex> lock(mu);
  if (sl.admitted) in_use -= sl.bytes;
  sl = Slot();
}

// Issue what is queued for one admitted session, in order. Updates are folded into one
// flushed batch; a finalisation waits until the previous one has completed (its result
// buffers are per session); a close waits until nothing is in flight.
void spca_server::issue(int32_t id, std::vector<Done>& done) {
  Slot& sl = slots[static_cast<size_t>(id)];
  Inflight batch;
  batch.kind = kUpdate;
  auto flush_batch = [&]() {
    if (batch.reqs.empty()) return;
    spca_status st = spca::session_flush(sl.s);
    cudaEvent_t ev = st == SPCA_OK ? event() : nullptr;
    if (st == SPCA_OK && ev && cudaEventRecord(ev, spca::session_stream(sl.s)) == cudaSuccess) {
      batch.ev = ev;
      sl.inflight.push_back(std::move(batch));
    } else {
      const spca_status fs = st == SPCA_OK ? SPCA_E_CUDA : st;
      const std::string why = reason(sl.s, fs, "launching the batched updates failed");
      for (Request& r : batch.reqs) done.push_back({r.ticket, fs, why});
    }
    batch = Inflight();
    batch.kind = kUpdate;
  };
  while (!sl.queue.empty()) {
    Request& r = sl.queue.front();
    if (sl.failed) {
      if (r.kind == kClose) {
        flush_batch();
        if (!sl.inflight.empty()) break;
        done.push_back({r.ticket, SPCA_OK, std::string()});
        sl.queue.pop_front();
        release(sl, false);
        return;
      }
      done.push_back({r.ticket, sl.fail_status, reason(nullptr, sl.fail_status, "the session could not be created")});
      sl.queue.pop_front();
      continue;
    }
    if (r.kind == kUpdate) {
      const spca_status st = spca_update(sl.s, r.rows, r.m, r.ld, SPCA_F32, nullptr, 1, nullptr);
      if (st != SPCA_OK) {
        done.push_back({r.ticket, st, reason(sl.s, st, "update rejected")});
      } else {
        batch.reqs.push_back(r);
      }
      sl.queue.pop_front();
      continue;
    }
    flush_batch();
    if (r.kind == kFinalize) {
      bool fin_busy = false;
      for (const Inflight& f : sl.inflight) fin_busy = fin_busy || f.kind == kFinalize;
      if (fin_busy) break;
      spca_status st = spca::session_finalize_async(sl.s, sl.sig_dev, sl.V_dev, sl.flags_host);
      cudaStream_t s_st = spca::session_stream(sl.s);
      const size_t vbytes = sizeof(double) * static_cast<size_t>(sl.n) * sl.k;
      if (st == SPCA_OK &&
          (cudaMemcpyAsync(sl.res_host, sl.sig_dev, sizeof(double) * sl.k, cudaMemcpyDeviceToHost, s_st) !=
               cudaSuccess ||
           cudaMemcpyAsync(sl.res_host + sl.k, sl.V_dev, vbytes, cudaMemcpyDeviceToHost, s_st) != cudaSuccess))
        st = SPCA_E_CUDA;
      cudaEvent_t ev = st == SPCA_OK ? event() : nullptr;
      if (st == SPCA_OK && ev && cudaEventRecord(ev, s_st) == cudaSuccess) {
        Inflight f;
        f.ev = ev;
        f.kind = kFinalize;
        f.reqs.push_back(r);
        sl.inflight.push_back(std::move(f));
      } else {
        const spca_status fs = st == SPCA_OK ? SPCA_E_CUDA : st;
        done.push_back({r.ticket, fs, reason(sl.s, fs, "finalisation could not be queued")});
      }
      sl.queue.pop_front();
      continue;
    }
    // close
    if (!sl.inflight.empty()) break;
    done.push_back({r.ticket, SPCA_OK, std::string()});
    sl.queue.pop_front();
    release(sl, true);
    return;
  }
  flush_batch();
}

void spca_server::complete(Slot& sl, Inflight& f, std::vector<Done>& done) {
  const Clock::time_point now = Clock::now();
  if (f.kind == kUpdate) {
    std::lock_guard<std::mutex> lock(mu);
    for (const Request& r : f.reqs) {
      lat_update.add(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
      rows_bytes += 4.0 * static_cast<double>(r.m) * static_cast<double>(sl.n);
      ++updates_done;
    }
  }
  for (const Request& r : f.reqs) {
    spca_status st = SPCA_OK;
    if (f.kind == kFinalize) {
      st = spca::session_flags_status(sl.s, *sl.flags_host);
      if (st == SPCA_OK) {
        std::memcpy(r.sigma, sl.res_host, sizeof(double) * sl.k);
        std::memcpy(r.V, sl.res_host + sl.k, sizeof(double) * static_cast<size_t>(sl.n) * sl.k);
      }
      std::lock_guard<std::mutex> lock(mu);
      lat_finalize.add(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
      ++finalizes_done;
    }
    done.push_back({r.ticket, st, st == SPCA_OK ? std::string() : reason(sl.s, st, "the finalisation failed")});
  }
}

void spca_server::run() {
  cudaSetDevice(device);
  Clock::time_point last = Clock::now();
  for (;;) {
    bool busy = false;
    for (const Slot& sl : slots) busy = busy || !sl.inflight.empty() || (sl.admitted && !sl.queue.empty());
    {
      std::unique_lock<std::mutex> lock(mu);
      if (incoming.empty() && !stop) {
        if (busy || !admission.empty())
          cv_work.wait_for(lock, std::chrono::microseconds(20));
        else
          cv_work.wait(lock, [&] { return !incoming.empty() || stop; });
      }
      while (!incoming.empty()) {
        Request r = incoming.front();
        incoming.pop_front();
        if (r.kind == kOpen)
          admission.push_back(r.id);
        else if (r.kind == kReserve)
          reserves.push_back(r);
        else
          slots[static_cast<size_t>(r.id)].queue.push_back(r);
      }
      if (stop && !admission.empty()) {
        // stopping: sessions that were never admitted are dropped with their requests
        for (int32_t id : admission) {
          Slot& sl = slots[static_cast<size_t>(id)];
          for (const Request& r : sl.queue) {
            auto it = tickets.find(r.ticket);   // closes have no waiter and no entry
            if (it == tickets.end()) continue;
            it->second.done = true;
            it->second.st = SPCA_E_STATE;
            it->second.msg = "the server stopped before the session was admitted";
          }
          sl = Slot();
        }
        admission.clear();
        cv_done.notify_all();
      }
      const Clock::time_point now = Clock::now();
      if (busy) active_s += std::chrono::duration<double>(now - last).count();
      last = now;
      if (stop && !busy && admission.empty() && reserves.empty()) {
        bool queued = false;
        for (const Slot& sl : slots) queued = queued || !sl.queue.empty();
        if (!queued) break;
      }
    }
    std::vector<Done> done;
    // reservations before the admissions that arrived with them
    while (!reserves.empty()) {
      const spca_status rs = reserve(reserves.front());
      done.push_back({reserves.front().ticket, rs,
                      rs == SPCA_OK ? std::string() : reason(nullptr, rs, "the reservation stopped short")});
      reserves.pop_front();
    }
    // closes that can go now, so that their sessions are in the pool for these admissions
    for (size_t i = 0; i < slots.size(); ++i) {
      const Slot& sl = slots[i];
      if (sl.admitted && sl.inflight.empty() && !sl.queue.empty() && sl.queue.front().kind == kClose)
        issue(static_cast<int32_t>(i), done);
    }
    // admission in arrival order
    while (!admission.empty() && admit(admission.front())) admission.pop_front();
    // issue
    for (size_t i = 0; i < slots.size(); ++i)
      if (slots[i].admitted && !slots[i].queue.empty()) issue(static_cast<int32_t>(i), done);
    // complete
    for (Slot& sl : slots) {
      while (!sl.inflight.empty()) {
        Inflight& f = sl.inflight.front();
        const cudaError_t q = cudaEventQuery(f.ev);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) {
          cudaGetLastError();
          for (const Request& r : f.reqs)
            done.push_back({r.ticket, SPCA_E_CUDA, std::string("a CUDA error ended the request: ") + cudaGetErrorString(q)});
        } else {
          complete(sl, f, done);
        }
        events.push_back(f.ev);
        sl.inflight.pop_front();
      }
    }
    // a session whose only queued request is a close can go now
    for (size_t i = 0; i < slots.size(); ++i)
      if (slots[i].admitted && !slots[i].queue.empty() && slots[i].inflight.empty()) issue(static_cast<int32_t>(i), done);
    {
      std::lock_guard<std::mutex> lock(mu);
      int64_t adm = 0;
      for (const Slot& sl : slots) adm += sl.admitted ? 1 : 0;
      admitted = adm;
      waiting = static_cast<int64_t>(admission.size());
      for (Done& d : done) {
        auto it = tickets.find(d.ticket);   // closes have no waiter and no entry
        if (it == tickets.end()) continue;
        it->second.done = true;
        it->second.st = d.st;
        it->second.msg = std::move(d.msg);
      }
    }
    if (!done.empty()) cv_done.notify_all();
  }
  for (Slot& sl : slots)
    if (sl.held || sl.admitted) release(sl, false);
  while (!pool.empty()) evict_oldest();
  for (cudaEvent_t e : events) cudaEventDestroy(e);
  events.clear();
}

extern "C" {

void spca_server_default_options(spca_server_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->math = SPCA_SERVER_AUTO_MATH;
  opt->max_sessions = 1024;
  opt->max_block_rows = 4096;
}

spca_status spca_server_create(const spca_server_options* opt, spca_server** out) {
  if (!out) return srv_fail(SPCA_E_INVALID, "out is NULL");
  *out = nullptr;
  spca_server_options o;
  spca_server_default_options(&o);
  if (opt) o = *opt;
  if (o.reserved != 0 || o.max_sessions < 1 || o.max_sessions > 4096 || o.max_block_rows < 1 ||
      !(o.math == SPCA_SERVER_AUTO_MATH || o.math == SPCA_MATH_FP32 || o.math == SPCA_MATH_BF16 ||
        o.math == SPCA_MATH_FP16))
    return srv_fail(SPCA_E_INVALID, "invalid server options");
  spca_server* sv = new (std::nothrow) spca_server();
  if (!sv) return srv_fail(SPCA_E_NOMEM, "host allocation failed");
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return srv_fail(SPCA_E_CUDA, "cudaGetDevice failed");
  }
  sv->opt = o;
  sv->budget = o.device_bytes;
  if (sv->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete sv;
      return srv_fail(SPCA_E_CUDA, "cudaMemGetInfo failed");
    }
    sv->budget = fr / 10 * 8;
  }
  sv->slots.resize(static_cast<size_t>(o.max_sessions));
  sv->worker = std::thread([sv] { sv->run(); });
  *out = sv;
  return SPCA_OK;
}

// The math form a session of these sizes gets and its device footprint with the result buffers.
static spca_status session_shape(spca_server* sv, int64_t n, int32_t k, int32_t p, int* math_out, size_t* bytes_out) {
  if (n < 1 || k < 1 || p < 0 || k + p > 256 || k + p > n) return srv_fail(SPCA_E_INVALID, "bad sizes");
  int old = 0;
  cudaGetDevice(&old);
  cudaSetDevice(sv->device);
  int math = sv->opt.math;
  size_t bytes = 0;
  if (math == SPCA_SERVER_AUTO_MATH) {
    math = SPCA_MATH_FP16;
    bytes = spca::session_footprint(n, k, p, math, sv->opt.max_block_rows);
    if (bytes == 0) math = SPCA_MATH_FP32;
  }
  if (bytes == 0) bytes = spca::session_footprint(n, k, p, math, sv->opt.max_block_rows);
  cudaSetDevice(old);
  if (bytes == 0) return srv_fail(SPCA_E_UNSUPPORTED, "the tensor-core pass does not fit these sizes");
  bytes += sizeof(double) * (static_cast<size_t>(n) * k + k);   // result buffers
  if (bytes > sv->budget) return srv_fail(SPCA_E_NOMEM, "the session alone exceeds the device budget");
  *math_out = math;
  *bytes_out = bytes;
  return SPCA_OK;
}

spca_status spca_server_open(spca_server* sv, int64_t n, int32_t k, int32_t p, uint64_t seed, int32_t* id) {
  if (!sv || !id) return srv_fail(SPCA_E_INVALID, "NULL server or id");
  int math = 0;
  size_t bytes = 0;
  const spca_status sst = session_shape(sv, n, k, p, &math, &bytes);
  if (sst != SPCA_OK) return sst;
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) return srv_fail(SPCA_E_STATE, "server is stopping");
  for (size_t i = 0; i < sv->slots.size(); ++i) {
    Slot& sl = sv->slots[i];
    if (sl.used || sl.held) continue;
    // a slot that is not held was reset by the worker (or never used): only its scalars are set
    // here, the worker's queues are left alone
    sl.used = true;
    sl.held = true;
    sl.n = n; sl.k = k; sl.p = p; sl.seed = seed; sl.math = math; sl.bytes = bytes;
    Request r;
    r.kind = kOpen;
    r.id = static_cast<int32_t>(i);
    r.t_submit = Clock::now();
    sv->incoming.push_back(r);
    *id = static_cast<int32_t>(i);
    sv->cv_work.notify_one();
    return SPCA_OK;
  }
  return srv_fail(SPCA_E_INVALID, "no free session slot");
}

spca_status spca_server_reserve(spca_server* sv, int64_t n, int32_t k, int32_t p, int32_t count, uint64_t* ticket) {
  if (!sv || !ticket) return srv_fail(SPCA_E_INVALID, "NULL server or ticket");
  if (count < 1) return srv_fail(SPCA_E_INVALID, "count < 1");
  Request r;
  r.kind = kReserve;
  const spca_status sst = session_shape(sv, n, k, p, &r.math, &r.bytes);
  if (sst != SPCA_OK) return sst;
  r.n = n; r.k = k; r.p = p; r.count = count;
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) return srv_fail(SPCA_E_STATE, "server is stopping");
  r.ticket = sv->next_ticket++;
  r.t_submit = Clock::now();
  sv->tickets[r.ticket] = TicketState();
  sv->incoming.push_back(r);
  *ticket = r.ticket;
  sv->cv_work.notify_one();
  return SPCA_OK;
}

static spca_status queue_request(spca_server* sv, Request r, uint64_t* ticket) {
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) return srv_fail(SPCA_E_STATE, "server is stopping");
  if (r.id < 0 || static_cast<size_t>(r.id) >= sv->slots.size() || !sv->slots[static_cast<size_t>(r.id)].used)
    return srv_fail(SPCA_E_INVALID, "unknown session id");
  if (r.kind == kClose) sv->slots[static_cast<size_t>(r.id)].used = false;
  r.ticket = sv->next_ticket++;
  r.t_submit = Clock::now();
  sv->tickets[r.ticket] = TicketState();
  sv->incoming.push_back(r);
  if (ticket) *ticket = r.ticket;
  sv->cv_work.notify_one();
  return SPCA_OK;
}

spca_status spca_server_update(spca_server* sv, int32_t id, const float* rows, int64_t m_i, int64_t ld,
                               uint64_t* ticket) {
  if (!sv || !rows || m_i < 1) return srv_fail(SPCA_E_INVALID, "NULL server or rows, or m_i < 1");
  Request r;
  r.kind = kUpdate;
  r.id = id;
  r.rows = rows;
  r.m = m_i;
  r.ld = ld;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (id >= 0 && static_cast<size_t>(id) < sv->slots.size() && sv->slots[static_cast<size_t>(id)].used &&
        (ld < sv->slots[static_cast<size_t>(id)].n || m_i > sv->opt.max_block_rows))
      return srv_fail(SPCA_E_INVALID, "ld < n, or more rows than max_block_rows");
  }
  return queue_request(sv, r, ticket);
}

spca_status spca_server_finalize(spca_server* sv, int32_t id, double* sigma, double* V, uint64_t* ticket) {
  if (!sv || !sigma || !V) return srv_fail(SPCA_E_INVALID, "NULL server, sigma or V");
  Request r;
  r.kind = kFinalize;
  r.id = id;
  r.sigma = sigma;
  r.V = V;
  return queue_request(sv, r, ticket);
}

spca_status spca_server_close(spca_server* sv, int32_t id) {
  if (!sv) return srv_fail(SPCA_E_INVALID, "NULL server");
  Request r;
  r.kind = kClose;
  r.id = id;
  uint64_t t = 0;
  spca_status st = queue_request(sv, r, &t);
  if (st != SPCA_OK) return st;
  std::lock_guard<std::mutex> lock(sv->mu);
  sv->tickets.erase(t);   // nobody waits for a close
  return SPCA_OK;
}

spca_status spca_server_wait(spca_server* sv, uint64_t ticket, double timeout_s) {
  if (!sv) return srv_fail(SPCA_E_INVALID, "NULL server");
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return srv_fail(SPCA_E_INVALID, "unknown ticket");
  auto ready = [&] { return sv->tickets[ticket].done; };
  if (timeout_s < 0) {
    sv->cv_done.wait(lock, ready);
  } else if (!sv->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ready)) {
    return srv_fail(SPCA_E_TIMEOUT, "request still running");
  }
  const spca_status st = sv->tickets[ticket].st;
  if (st != SPCA_OK) srv_fail(st, sv->tickets[ticket].msg.empty() ? "request failed" : sv->tickets[ticket].msg.c_str());
  sv->tickets.erase(ticket);
  return st;
}

spca_status spca_server_get_stats(spca_server* sv, spca_server_stats* out) {
  if (!sv || !out) return srv_fail(SPCA_E_INVALID, "NULL server or out");
  std::vector<double> lu, lf;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    std::memset(out, 0, sizeof(*out));
    out->updates_done = sv->updates_done;
    out->finalizes_done = sv->finalizes_done;
    out->sessions_admitted = sv->admitted;
    out->sessions_waiting = sv->waiting;
    out->rows_bytes = sv->rows_bytes;
    out->active_seconds = sv->active_s;
    out->device_bytes_in_use = sv->in_use;
    out->device_bytes_budget = sv->budget;
    out->sessions_pooled = sv->n_pooled;
    out->admissions_from_pool = sv->from_pool;
    out->sessions_created = sv->created;
    out->device_bytes_pooled = sv->pooled_bytes;
    lu = sv->lat_update.v;
    lf = sv->lat_finalize.v;
  }
  // the selections run on the copies, outside the lock the worker takes
  out->update_p50_ms = pct(lu, 0.50);
  out->update_p99_ms = pct(lu, 0.99);
  out->finalize_p50_ms = pct(lf, 0.50);
  out->finalize_p99_ms = pct(lf, 0.99);
  return SPCA_OK;
}

spca_status spca_server_destroy(spca_server* sv) {
  if (!sv) return SPCA_OK;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
    // close every session that is still open once its queue drains
    for (size_t i = 0; i < sv->slots.size(); ++i) {
      if (!sv->slots[i].used) continue;
      Request r;
      r.kind = kClose;
      r.id = static_cast<int32_t>(i);
      r.ticket = sv->next_ticket++;
      sv->slots[i].used = false;
      sv->incoming.push_back(r);
    }
  }
  sv->cv_work.notify_one();
  if (sv->worker.joinable()) sv->worker.join();
  delete sv;
  return SPCA_OK;
}

const char* spca_server_last_error(void) { return g_srv_err; }

}  // extern "C"
