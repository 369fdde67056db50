// A host-only stand-in for the CUDA runtime calls and the session calls that the serving loop
// (csrc/server.cu) makes, so that its threading, admission, pooling and ticket logic can be
// tested on a machine without a GPU. Compiled with server.cu into a test library; nothing of
// the product links it.
//
// Device memory is host memory; a stream is a clock that each enqueued operation pushes
// forward by a configurable delay, and an event recorded on it is ready once that time has
// passed. A session folds its rows into a 64-bit FNV-1a digest (the 32-bit words of each row,
// rows in order) and its "finalisation" writes values derived from (seed, rows, digest), so a
// test can tell whether every session received exactly its own rows, in order, and that each
// result went to the request that asked for it.
#include <cuda_runtime_api.h>

#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>

#include "spca.h"
#include "spca_internal.cuh"

using Clock = std::chrono::steady_clock;

struct CUstream_st {
  std::mutex mu;
  Clock::time_point busy_until = Clock::now();
  void push(int64_t us) {
    std::lock_guard<std::mutex> lock(mu);
    const Clock::time_point now = Clock::now();
    if (busy_until < now) busy_until = now;
    busy_until += std::chrono::microseconds(us);
  }
  Clock::time_point until() {
    std::lock_guard<std::mutex> lock(mu);
    return busy_until;
  }
};

struct CUevent_st {
  std::atomic<int64_t> ready_ns{0};
};

struct spca_session {
  int64_t n = 0;
  int k = 0, p = 0, math = 0;
  uint64_t seed = 0;
  int64_t m = 0;
  uint64_t digest = 1469598103934665603ull;
  char err[128] = "";
  CUstream_st stream;
};

namespace {

std::atomic<int64_t> g_live_allocs{0};
std::atomic<int64_t> g_live_sessions{0};
std::atomic<int64_t> g_creates{0};
std::atomic<int64_t> g_delay_create_us{0}, g_delay_update_us{0}, g_delay_finalize_us{0};
std::atomic<int64_t> g_fail_create_every{0};

int64_t ns_of(Clock::time_point t) {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(t.time_since_epoch()).count();
}

void* fake_alloc(size_t bytes) {
  void* p = std::malloc(bytes ? bytes : 1);
  if (p) g_live_allocs.fetch_add(1);
  return p;
}

void fake_free(void* p) {
  if (!p) return;
  std::free(p);
  g_live_allocs.fetch_sub(1);
}

uint64_t result_word(uint64_t digest, uint64_t seed, int64_t i) {
  return (digest ^ seed) + static_cast<uint64_t>(i) * 0x9E3779B97F4A7C15ull;
}

double to_unit(uint64_t x) { return static_cast<double>(x >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

// ------------------------------------------------------------------ the CUDA runtime subset

extern "C" {

cudaError_t cudaGetDevice(int* device) {
  *device = 0;
  return cudaSuccess;
}

cudaError_t cudaSetDevice(int) { return cudaSuccess; }

cudaError_t cudaGetLastError(void) { return cudaSuccess; }

const char* cudaGetErrorString(cudaError_t e) { return e == cudaSuccess ? "no error" : "stand-in CUDA error"; }

cudaError_t cudaMemGetInfo(size_t* free_bytes, size_t* total) {
  *free_bytes = size_t(64) << 30;
  *total = size_t(80) << 30;
  return cudaSuccess;
}

cudaError_t cudaMalloc(void** p, size_t bytes) {
  *p = fake_alloc(bytes);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

cudaError_t cudaFree(void* p) {
  fake_free(p);
  return cudaSuccess;
}

cudaError_t cudaHostAlloc(void** p, size_t bytes, unsigned int) {
  *p = fake_alloc(bytes);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

cudaError_t cudaFreeHost(void* p) {
  fake_free(p);
  return cudaSuccess;
}

cudaError_t cudaEventCreateWithFlags(cudaEvent_t* ev, unsigned int) {
  *ev = new CUevent_st();
  g_live_allocs.fetch_add(1);
  return cudaSuccess;
}

cudaError_t cudaEventDestroy(cudaEvent_t ev) {
  if (ev) {
    delete ev;
    g_live_allocs.fetch_sub(1);
  }
  return cudaSuccess;
}

cudaError_t cudaEventRecord(cudaEvent_t ev, cudaStream_t st) {
  ev->ready_ns.store(st ? ns_of(st->until()) : 0);
  return cudaSuccess;
}

cudaError_t cudaEventQuery(cudaEvent_t ev) {
  return ns_of(Clock::now()) >= ev->ready_ns.load() ? cudaSuccess : cudaErrorNotReady;
}

// Copies at once: the data a fake stream would copy is final when it is enqueued.
cudaError_t cudaMemcpyAsync(void* dst, const void* src, size_t count, cudaMemcpyKind, cudaStream_t) {
  std::memmove(dst, src, count);
  return cudaSuccess;
}

// ------------------------------------------------------------------ the session calls

void spca_default_options(spca_options* opt) {
  std::memset(opt, 0, sizeof(*opt));
  opt->math = SPCA_MATH_FP32;
  opt->center = 1;
}

spca_status spca_create(int64_t n, int32_t k, int32_t p, uint64_t seed, const spca_options* opt,
                        spca_session** out) {
  const int64_t c = g_creates.fetch_add(1) + 1;
  const int64_t d = g_delay_create_us.load();
  if (d > 0) std::this_thread::sleep_for(std::chrono::microseconds(d));
  const int64_t every = g_fail_create_every.load();
  if (every > 0 && c % every == 0) return SPCA_E_NOMEM;
  spca_session* s = new spca_session();
  s->n = n; s->k = k; s->p = p; s->seed = seed; s->math = opt ? opt->math : 0;
  g_live_sessions.fetch_add(1);
  *out = s;
  return SPCA_OK;
}

spca_status spca_destroy(spca_session* s) {
  if (s) {
    delete s;
    g_live_sessions.fetch_sub(1);
  }
  return SPCA_OK;
}

spca_status spca_reset(spca_session* s, uint64_t seed) {
  s->seed = seed;
  s->m = 0;
  s->digest = 1469598103934665603ull;
  return SPCA_OK;
}

spca_status spca_update(spca_session* s, const void* rows, int64_t m_i, int64_t ld, int32_t, const float*,
                        int32_t, float*) {
  if (m_i == 97) {   // a block the stand-in refuses, to test how a failure is reported
    std::snprintf(s->err, sizeof(s->err), "the stand-in refuses 97-row blocks (session seed %llu)",
                  static_cast<unsigned long long>(s->seed));
    return SPCA_E_INVALID;
  }
  const uint32_t* w = static_cast<const uint32_t*>(rows);
  for (int64_t r = 0; r < m_i; ++r)
    for (int64_t j = 0; j < s->n; ++j) {
      s->digest ^= w[r * ld + j];
      s->digest *= 1099511628211ull;
    }
  s->m += m_i;
  s->stream.push(g_delay_update_us.load());
  return SPCA_OK;
}

const char* spca_last_error(const spca_session* s) { return s ? s->err : ""; }

// Test controls.
void fake_set_delays(int64_t create_us, int64_t update_us, int64_t finalize_us) {
  g_delay_create_us.store(create_us);
  g_delay_update_us.store(update_us);
  g_delay_finalize_us.store(finalize_us);
}

void fake_fail_create_every(int64_t every) { g_fail_create_every.store(every); }

int64_t fake_live_allocations(void) { return g_live_allocs.load(); }

int64_t fake_live_sessions(void) { return g_live_sessions.load(); }

int64_t fake_creates(void) { return g_creates.load(); }

}  // extern "C"

namespace spca {

// Every session fits the FP16 form up to l = 127, as the grouped kernel does.
size_t session_footprint(int64_t n, int k, int p, int math, int64_t) {
  if ((math == SPCA_MATH_FP16 || math == SPCA_MATH_BF16) && k + p > 127) return 0;
  return size_t(1) << 20 | size_t(n) * size_t(k + p) * 8;
}

cudaStream_t session_stream(spca_session* s) { return &s->stream; }

spca_status session_flush(spca_session*) { return SPCA_OK; }

spca_status session_prepare_staging(spca_session*) { return SPCA_OK; }

spca_status session_finalize_async(spca_session* s, double* sigma_dev, double* V_dev, int* flags_host) {
  if (s->m < 1) return SPCA_E_NUMERIC;
  for (int i = 0; i < s->k; ++i) sigma_dev[i] = to_unit(result_word(s->digest, s->seed, i));
  const int64_t nv = s->n * s->k;
  for (int64_t t = 0; t < nv; ++t) V_dev[t] = to_unit(result_word(s->digest, s->seed, s->k + t));
  *flags_host = 0;
  s->stream.push(g_delay_finalize_us.load());
  return SPCA_OK;
}

spca_status session_flags_status(spca_session*, int) { return SPCA_OK; }

}  // namespace spca
