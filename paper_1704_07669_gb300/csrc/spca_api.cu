// C ABI of the library (include/spca.h): sessions, argument checks, streams,
// host staging, and the order of the launches that make up the pass.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "spca.h"
#include "spca_internal.cuh"

using namespace spca;

namespace {

thread_local char g_thread_err[512] = "";

constexpr size_t kStageBytes = size_t(256) << 20;   // per staging buffer (two of them)

size_t dtype_size(int dtype) {
  switch (dtype) {
    case SPCA_F32: return 4;
    case SPCA_BF16: return 2;
    case SPCA_F8E4M3: return 1;
    case SPCA_F64: return 8;
    default: return 0;
  }
}

// features covered by the pre-swizzled Omega: the larger padding of the two kernels
int64_t tc_npad(const TcWork& t) {
  const int64_t a = t.cfg_ok ? static_cast<int64_t>(t.cfg.CS) * t.cfg.w : 0;
  const int64_t b = t.v3 ? static_cast<int64_t>(t.cfg3.CS) * t.cfg3.w : 0;
  const int64_t c = t.use_grp ? static_cast<int64_t>(t.grp.nbt) * 64 : 0;
  const int64_t ab = a > b ? a : b;
  return ab > c ? ab : c;
}

// Configurations of the tensor-core kernels for (n, l, L) and the sizes (elements) of their
// buffers; false when no kernel takes the shape.
struct TcSizes {
  int64_t npad, hpart, nctas, img, part, gbuf, cnt;
};
bool tc_setup(int64_t n, int l, int L, int fmt, TcWork* t, TcSizes* z) {
  t->cfg_ok = tc_config(n, L, fmt, &t->cfg);
  t->v3 = t->cfg_ok && tc3_config(n, L, fmt, &t->cfg3);
  t->use_grp = spca::grp_config(n, l, L, fmt, &t->grp);
  if (!t->cfg_ok && !t->use_grp) return false;
  z->npad = tc_npad(*t);
  const int64_t hp = t->cfg_ok ? int64_t(t->cfg.nclusters) * t->cfg.CS * t->cfg.w : 0;
  const int64_t hp3 = t->v3 ? int64_t(t->cfg3.nclusters) * t->cfg3.CS * t->cfg3.w : 0;
  const int64_t hpg = t->use_grp ? int64_t(t->grp.NG) * t->grp.nbt * 64 : 0;
  z->hpart = hp > hp3 ? hp : hp3;
  if (hpg > z->hpart) z->hpart = hpg;
  int64_t nc = t->cfg_ok ? int64_t(t->cfg.nclusters) * t->cfg.CS : 0;
  if (t->v3 && int64_t(t->cfg3.nclusters) * t->cfg3.CS > nc) nc = int64_t(t->cfg3.nclusters) * t->cfg3.CS;
  if (t->use_grp && int64_t(t->grp.NG) * t->grp.S > nc) nc = int64_t(t->grp.NG) * t->grp.S;
  z->nctas = nc;
  const int64_t img3 = t->v3 ? hp3 * 256 : 0;
  const int64_t imgg = t->use_grp ? static_cast<int64_t>(spca::grp_img_elems(t->grp)) : 0;
  z->img = img3 > imgg ? img3 : imgg;
  z->part = t->use_grp ? static_cast<int64_t>(spca::grp_part_elems(t->grp, L)) : 0;
  z->gbuf = t->use_grp ? static_cast<int64_t>(spca::grp_gbuf_elems(t->grp, L, fmt)) : 0;
  z->cnt = t->use_grp ? static_cast<int64_t>(spca::grp_cnt_elems(t->grp)) : 0;
  return true;
}

}  // namespace

namespace spca {

void Prof::begin(int id, cudaStream_t st) {
  launches[id] += 1;
  if (!timing) return;
  if (nmarks == cap) {
    const int ncap = cap ? 2 * cap : 256;
    Mark* nm = static_cast<Mark*>(realloc(marks, sizeof(Mark) * ncap));
    if (!nm) { timing = false; return; }
    for (int i = cap; i < ncap; ++i) {
      nm[i].a = nullptr;
      nm[i].b = nullptr;
    }
    marks = nm;
    cap = ncap;
  }
  Mark& mk = marks[nmarks];
  if (!mk.a) cudaEventCreate(&mk.a);
  if (!mk.b) cudaEventCreate(&mk.b);
  mk.id = id;
  cudaEventRecord(mk.a, st);
}

void Prof::end(int id, cudaStream_t st) {
  if (!timing || nmarks >= cap || marks[nmarks].id != id) return;
  cudaEventRecord(marks[nmarks].b, st);
  ++nmarks;
}

void Prof::release() {
  for (int i = 0; i < cap; ++i) {
    if (marks[i].a) cudaEventDestroy(marks[i].a);
    if (marks[i].b) cudaEventDestroy(marks[i].b);
  }
  free(marks);
  marks = nullptr;
  cap = nmarks = 0;
}

}  // namespace spca

struct spca_session {
  int device = 0;
  int64_t n = 0;
  int k = 0, p = 0, l = 0, L = 0;
  uint64_t seed = 0;
  spca_options opt{};
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;
  bool own_stream = false;
  bool failed = false;
  int64_t m = 0;
  bool shift_set = false;
  bool scale_set = false;     // FP16 form: operand scale computed from the first rows
  bool u_ready = false;       // a finalize has formed the map to U since the last change of the state
  bool omega_orth = false;    // Omega is orth(H) of a previous pass (power scheme), not the Philox draw
  char err[512] = "";
  char desc[256] = "";

  // state
  float* omega32 = nullptr;
  double* H = nullptr;
  float* shift = nullptr;
  double* colsum = nullptr;
  double* sG = nullptr;
  double* gram = nullptr;
  int* flags = nullptr;
  int* host_flags = nullptr;   // pinned mirror of flags[0..3]

  // workspace
  SimtWork simt{};
  int64_t gp_rows = 0;
  double* shift_part = nullptr;
  FinalWork fin{};
  double* fin_sigma = nullptr;
  double* fin_V = nullptr;
  float* upass_W = nullptr;       // n x L: V Sigma^-1 of the last finalize (FP32), for spca_left_vectors_pass
  double* upass_corr = nullptr;   // L: its centring term
  float* upass_gpart = nullptr;   // tensor-core sessions: split-K partials of the second pass (made on first use)
  bool upass_corr_ready = false;  // upass_corr formed since the last finalize

  // host staging
  void* pinned[2] = {nullptr, nullptr};
  void* dstage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  cudaEvent_t copied[2] = {nullptr, nullptr};
  cudaEvent_t consumed[2] = {nullptr, nullptr};
  int next_stage = 0;

  // tensor-core path (math = BF16)
  bool tc = false;
  TcWork tcw{};
  TcPending pend;

  Prof prof;

  State state() const {
    State s;
    s.n = n; s.l = l; s.L = L;
    s.omega32 = omega32; s.H = H; s.shift = shift; s.colsum = colsum; s.sG = sG; s.gram = gram; s.flags = flags;
    return s;
  }
};

namespace {

spca_status fail(spca_session* s, spca_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (s) {
    std::strncpy(s->err, buf, sizeof(s->err) - 1);
    if (st == SPCA_E_CUDA) s->failed = true;
  }
  std::strncpy(g_thread_err, buf, sizeof(g_thread_err) - 1);
  return st;
}

#define CU(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(s, SPCA_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Allocation-failure injection for tests of the error paths: with SPCA_FAIL_ALLOC_AT=N in the
// environment, the N-th device allocation (from 0) of a spca_create call reports
// cudaErrorMemoryAllocation without allocating. Armed per call, on the calling thread.
thread_local int64_t t_fail_alloc_at = -1;
thread_local int64_t t_alloc_count = 0;

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (t_fail_alloc_at >= 0 && t_alloc_count++ == t_fail_alloc_at) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

struct AllocFailArm {   // arms the injection for one spca_create, disarms on every exit
  AllocFailArm() {
    const char* v = std::getenv("SPCA_FAIL_ALLOC_AT");
    t_fail_alloc_at = (v && *v) ? std::atoll(v) : -1;
    t_alloc_count = 0;
  }
  ~AllocFailArm() { t_fail_alloc_at = -1; }
};

// the grouped kernel's wait limit: SPCA_WAIT_LIMIT_MS (1 .. 60000), else half a second
uint64_t wait_limit_ns() {
  const char* v = std::getenv("SPCA_WAIT_LIMIT_MS");
  if (!v || !*v) return 500000000ull;
  long long ms = std::atoll(v);
  if (ms < 1) ms = 1;
  if (ms > 60000) ms = 60000;
  return static_cast<uint64_t>(ms) * 1000000ull;
}

void free_all(spca_session* s) {
  void* bufs[] = {s->omega32, s->H, s->shift, s->colsum, s->sG, s->gram, s->flags, s->simt.Gpart, s->simt.G,
                  s->simt.gram_part, s->simt.sG_part, s->simt.Hpart, s->simt.cs_part, s->shift_part, s->fin.Hbar,
                  s->fin.gbar, s->fin.T, s->fin.X, s->fin.W, s->fin.lam, s->fin.Bt, s->fin.Cpart, s->fin.C,
                  s->fin.sig, s->fin.info, s->fin.flip, s->fin.Tu, s->fin.M, s->fin.mrow, s->fin_sigma, s->fin_V,
                  s->upass_W, s->upass_corr, s->upass_gpart,
                  s->dstage[0], s->dstage[1],
                  s->tcw.om16, s->tcw.Hpart, s->tcw.gram_part, s->tcw.sG_part, s->tcw.scale, s->tcw.scale_bits,
                  s->tcw.img, s->tcw.zero8k, s->tcw.part, s->tcw.gbuf, s->tcw.cnt, s->tcw.gfull};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int i = 0; i < 2; ++i) {
    if (s->pinned[i]) cudaFreeHost(s->pinned[i]);
    if (s->copied[i]) cudaEventDestroy(s->copied[i]);
    if (s->consumed[i]) cudaEventDestroy(s->consumed[i]);
  }
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  if (s->host_flags) cudaFreeHost(s->host_flags);
  s->prof.release();
}

spca_status check_usable(spca_session* s) {
  if (!s) return fail(nullptr, SPCA_E_INVALID, "NULL session");
  if (s->failed) return fail(s, SPCA_E_STATE, "session is in an error state after a CUDA failure: %s", s->err);
  return SPCA_OK;
}

// Launch the tensor-core pass over the row blocks batched so far.
spca_status flush_tc(spca_session* s) {
  if (!s->tc || s->pend.nseg == 0) return SPCA_OK;
  bool used = false;
  if (s->tcw.use_grp) CU(grp_pass(s->state(), s->tcw, s->pend, s->stream, &s->prof, &used));
  if (!used && s->pend.dtype != SPCA_F32) {   // the other tensor-core kernels read FP32 rows only
    s->pend.nseg = 0;
    s->pend.rows_total = 0;
    return fail(s, SPCA_E_UNSUPPORTED,
                "BF16 and FP8 rows reach the tensor cores through the grouped kernel only, which needs 16-byte "
                "aligned row blocks whose rows are a multiple of 16 bytes apart");
  }
  if (!used && s->tcw.v3) CU(tc3_pass(s->state(), s->tcw, s->pend, s->stream, &s->prof, &used));
  if (!used) {
    if (!s->tcw.cfg_ok) {
      s->pend.nseg = 0;
      s->pend.rows_total = 0;
      return fail(s, SPCA_E_UNSUPPORTED,
                  "the tensor-core pass at n = %lld, l = %d reads rows through tensor maps only: row blocks "
                  "must start 16-byte aligned with a leading dimension that is a multiple of 4",
                  (long long)s->n, s->l);
    }
    CU(tc_pass(s->state(), s->tcw, s->pend, s->stream, &s->prof));
  }
  s->pend.nseg = 0;
  s->pend.rows_total = 0;
  return SPCA_OK;
}

// One piece of rows resident on the device. The FP32 path processes it at once; the
// tensor-core path batches device-resident blocks (defer) into one persistent launch.
spca_status run_piece(spca_session* s, const void* rows, int64_t m, int64_t ld, int dtype, float scale,
                      float* G_out, bool defer) {
  if (s->opt.center && !s->shift_set) {
    CU(launch_shift(rows, dtype, m, s->n, ld, scale, s->shift, s->shift_part, s->stream, &s->prof));
    s->shift_set = true;
  }
  if (s->tc && s->tcw.fmt == 1 && !s->scale_set) {
    CU(launch_op_scale(rows, dtype, scale, m, s->n, ld, s->shift, s->tcw.scale_bits, s->tcw.scale,
                       s->omega_orth ? 1.0 : std::sqrt(static_cast<double>(s->n)), s->stream, &s->prof));
    s->scale_set = true;
  }
  if (s->tc) {
    // one launch reads one storage format: a block of another format flushes the batch first
    if (s->pend.nseg == kTcPendingMax || (s->pend.nseg > 0 && s->pend.dtype != dtype)) {
      spca_status st = flush_tc(s);
      if (st != SPCA_OK) return st;
    }
    const int i = s->pend.nseg++;
    s->pend.dtype = dtype;
    s->pend.rows[i] = rows;
    s->pend.m[i] = m;
    s->pend.ld[i] = ld;
    s->pend.gout[i] = G_out;
    s->pend.dscale[i] = scale;
    s->pend.rows_total += m;
    s->m += m;
    if (!defer || s->pend.rows_total >= kTcPendingRows) return flush_tc(s);
    return SPCA_OK;
  }
  SimtWork w = s->simt;
  CU(simt_pass(s->state(), w, rows, dtype, scale, m, ld, G_out, s->stream, &s->prof));
  s->m += m;
  return SPCA_OK;
}

}  // namespace

namespace spca {

// Device bytes that spca_create allocates for these parameters (each allocation rounded up
// to 512 bytes); the serving loop admits sessions against this figure.
size_t session_footprint(int64_t n, int k, int p, int math, int64_t max_block_rows) {
  const int l = k + p;
  const bool tc = (math == SPCA_MATH_BF16 || math == SPCA_MATH_FP16);
  const int L = tc ? pad_l(l + 1) : pad_l(l);
  TcWork t{};
  TcSizes z{};
  if (tc && !tc_setup(n, l, L, math == SPCA_MATH_FP16 ? 1 : 0, &t, &z)) return 0;
  const int64_t mb = max_block_rows > 0 ? max_block_rows : kDefaultBlockRows;
  size_t b = 0;
  auto add = [&](int64_t count, size_t es) {
    const size_t bytes = size_t(count < 1 ? 1 : count) * es;
    b += (bytes + 511) & ~size_t(511);
  };
  if (!tc) add(n * L, 4);
  add(n * L, 8); add(n, 4); add(n, 8); add(L, 8); add(int64_t(L) * L, 8); add(4, 4);
  add(n * L, 4); add(L, 8);   // the second pass's V Sigma^-1 and centring term
  if (!tc) {
    const int64_t mb_pad = ((mb + 127) / 128) * 128;
    const int64_t gp_rows = mb_pad > 65536 ? mb_pad : 65536;
    int64_t tmax = (int64_t(16) << 20) / (n * L);
    const int64_t T = tmax < 1 ? 1 : (tmax > 16 ? 16 : tmax);
    const int64_t groups = (mb + 31) / 32;
    add(gp_rows * L, 4); add(mb * L, 4); add(groups * L * L, 8); add(groups * L, 8); add(T * n * L, 4); add(T * n, 4);
  } else {
    add(z.npad * L, 2); add(1, 4); add(1, 4); add(z.hpart * L, 4); add(z.nctas * L * L, 8);
    add(z.nctas * L, 8);
    if (z.img) add(z.img, 2);
    if (t.use_grp) {
      add(4096, 2); add(z.part, 4); add(z.gbuf, 2); add(z.cnt, 4);
      const int64_t gr = static_cast<int64_t>(grp_gfull_rows(t.grp, mb));
      if (gr) add(gr * L, 4);
    }
  }
  add(int64_t(kShiftParts) * n, 8);
  const int64_t per = int64_t(L) * L * 8;
  int64_t np = (int64_t(8) << 20) / per;
  np = np < 4 ? 4 : (np > 304 ? 304 : np);
  add(n * L, 8); for (int i = 0; i < 4; ++i) add(int64_t(L) * L, 8);
  add(L, 8); add(n * L, 8); add(np * L * L, 8); add(int64_t(L) * L, 8); add(L, 8); add(8, 4); add(k, 8); add(n * k, 8);
  add(L, 8); add(int64_t(L) * L, 8); add(int64_t(L) * L, 8); add(L, 8);
  return b;
}

cudaStream_t session_stream(spca_session* s) { return s->stream; }

// Launch the tensor-core blocks batched so far, without waiting.
spca_status session_flush(spca_session* s) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  CU(cudaSetDevice(s->device));
  return flush_tc(s);
}

// Enqueue the finalisation: sigma, V (device) and the flags word (pinned host) are written
// when the session stream reaches them; session_flags_status interprets the flags then.
spca_status session_finalize_async(spca_session* s, double* sigma_dev, double* V_dev, int* flags_host) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (s->m < 1) return fail(s, SPCA_E_NUMERIC, "no rows accumulated yet");
  CU(cudaSetDevice(s->device));
  st = flush_tc(s);
  if (st != SPCA_OK) return st;
  CU(finalize_run(s->state(), s->fin, s->opt.center ? s->m : 0, s->k, sigma_dev, V_dev, s->stream, &s->prof, s->m,
                  s->opt.center != 0));
  CU(cudaMemcpyAsync(flags_host, s->flags, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  return SPCA_OK;
}

spca_status session_flags_status(spca_session* s, int flags) {
  if (flags & 16)
    return fail(s, SPCA_E_CUDA, "the grouped tensor-core kernel was launched with a configuration it does not take");
  if (flags & 8) return fail(s, SPCA_E_CUDA, "a copy of the tensor-core pass was out of its buffer (skipped)");
  if (flags & 2) return fail(s, SPCA_E_TIMEOUT, "a bounded device wait gave up during the pass");
  if (flags & 1) return fail(s, SPCA_E_NUMERIC, "non-finite values (NaN/Inf) reached the sketch");
  return SPCA_OK;
}

int session_k(const spca_session* s) { return s->k; }
int64_t session_n(const spca_session* s) { return s->n; }

}  // namespace spca

extern "C" {

void spca_default_options(spca_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->math = SPCA_MATH_FP32;
  opt->center = 1;
  opt->max_block_rows = 0;
  opt->cuda_stream = nullptr;
}

spca_status spca_create(int64_t n, int32_t k, int32_t p, uint64_t seed, const spca_options* opt,
                        spca_session** out) {
  spca_session* s = nullptr;
  if (!out) return fail(nullptr, SPCA_E_INVALID, "out is NULL");
  *out = nullptr;
  const AllocFailArm arm;
  if (n < 1 || k < 1 || p < 0) return fail(nullptr, SPCA_E_INVALID, "need n >= 1, k >= 1, p >= 0 (n=%lld k=%d p=%d)",
                                           (long long)n, k, p);
  const int64_t l = static_cast<int64_t>(k) + p;
  if (l > kMaxL || l > n)
    return fail(nullptr, SPCA_E_INVALID, "l = k + p = %lld must be <= min(n, %d)", (long long)l, kMaxL);
  spca_options o;
  spca_default_options(&o);
  if (opt) o = *opt;
  if (o.reserved != 0 || (o.center != 0 && o.center != 1) || o.max_block_rows < 0)
    return fail(nullptr, SPCA_E_INVALID, "invalid options");
  const bool tc_math = (o.math == SPCA_MATH_BF16 || o.math == SPCA_MATH_FP16);
  if (o.math != SPCA_MATH_FP32 && !tc_math)
    return fail(nullptr, SPCA_E_UNSUPPORTED, "math form %d is not available in this build", o.math);
  TcWork tcw0{};
  TcSizes tcz{};
  // the tensor-core pass keeps one spare column (index l) for the column sums
  const int L_tc = pad_l(static_cast<int>(l) + 1);
  if (tc_math && !tc_setup(n, static_cast<int>(l), L_tc, o.math == SPCA_MATH_FP16 ? 1 : 0, &tcw0, &tcz))
    return fail(nullptr, SPCA_E_UNSUPPORTED, "no tensor-core kernel takes n=%lld, l=%lld: %s; %s", (long long)n,
                (long long)l, grp_config_reason(), tc_config_reason());

  s = new (std::nothrow) spca_session();
  if (!s) return fail(nullptr, SPCA_E_NOMEM, "host allocation failed");
  s->n = n; s->k = k; s->p = p; s->l = static_cast<int>(l); s->seed = seed;
  s->L = tc_math ? L_tc : pad_l(static_cast<int>(l));
  s->opt = o;
  const int64_t mb = o.max_block_rows > 0 ? o.max_block_rows : kDefaultBlockRows;
  const int L = s->L;

#define CC(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      spca_status st_ = (e_ == cudaErrorMemoryAllocation) ? SPCA_E_NOMEM : SPCA_E_CUDA; \
      fail(nullptr, st_, "%s: %s", #call, cudaGetErrorString(e_));                  \
      free_all(s);                                                                  \
      delete s;                                                                     \
      return st_;                                                                   \
    }                                                                               \
  } while (0)

  CC(cudaGetDevice(&s->device));
  if (o.cuda_stream) {
    s->stream = static_cast<cudaStream_t>(o.cuda_stream);
  } else {
    CC(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  CC(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
  s->tc = tc_math;
  s->tcw.fmt = (o.math == SPCA_MATH_FP16) ? 1 : 0;
  if (!s->tc) CC(dalloc(&s->omega32, n * L));
  CC(dalloc(&s->H, n * L));
  CC(dalloc(&s->shift, n));
  CC(dalloc(&s->colsum, n));
  CC(dalloc(&s->sG, L));
  CC(dalloc(&s->gram, size_t(L) * L));
  CC(dalloc(&s->flags, 4));
  CC(cudaMallocHost(&s->host_flags, sizeof(int) * 4));

  SimtWork& w = s->simt;
  w.mb = mb;
  if (!s->tc) {
    const int64_t mb_pad = ((mb + 127) / 128) * 128;
    w.gp_rows = mb_pad > 65536 ? mb_pad : 65536;
    s->gp_rows = w.gp_rows;
    int64_t tmax = (int64_t(16) << 20) / (n * L);
    w.T = static_cast<int>(tmax < 1 ? 1 : (tmax > 16 ? 16 : tmax));
    CC(dalloc(&w.Gpart, size_t(s->gp_rows) * L));
    CC(dalloc(&w.G, size_t(mb) * L));
    const int64_t groups = (mb + 31) / 32;
    CC(dalloc(&w.gram_part, size_t(groups) * L * L));
    CC(dalloc(&w.sG_part, size_t(groups) * L));
    CC(dalloc(&w.Hpart, size_t(w.T) * n * L));
    CC(dalloc(&w.cs_part, size_t(w.T) * n));
  } else {
    TcWork& t = s->tcw;
    const int fmt = t.fmt;
    t = tcw0;   // the configurations (the grouped kernel preferred, the others as fallbacks)
    t.fmt = fmt;
    t.wait_ns = wait_limit_ns();
    CC(dalloc(&t.om16, size_t(tcz.npad) * L));
    CC(dalloc(&t.scale, 1));
    CC(dalloc(&t.scale_bits, 1));
    CC(dalloc(&t.Hpart, size_t(tcz.hpart) * L));
    CC(dalloc(&t.gram_part, size_t(tcz.nctas) * L * L));
    CC(dalloc(&t.sG_part, size_t(tcz.nctas) * L));
    if (tcz.img) CC(dalloc(&t.img, size_t(tcz.img)));
    if (t.use_grp) {
      CC(dalloc(&t.zero8k, 4096));
      CC(cudaMemsetAsync(t.zero8k, 0, 8192, s->stream));
      CC(dalloc(&t.part, size_t(tcz.part)));
      CC(dalloc(&t.gbuf, size_t(tcz.gbuf)));
      CC(dalloc(&t.cnt, size_t(tcz.cnt)));
      t.gfull_rows = static_cast<int64_t>(grp_gfull_rows(t.grp, mb));
      if (t.gfull_rows) CC(dalloc(&t.gfull, size_t(t.gfull_rows) * L));
    }
  }
  CC(dalloc(&s->shift_part, size_t(kShiftParts) * n));

  FinalWork& f = s->fin;
  // partial C = B B^T per block of the n x l product: about 8 MiB of them, at least 4
  // (the eigensolver reuses the space as scratch)
  {
    const int64_t per = int64_t(L) * L * int64_t(sizeof(double));
    int64_t np = (int64_t(8) << 20) / per;
    f.nparts = static_cast<int>(np < 4 ? 4 : (np > 304 ? 304 : np));
  }
  CC(dalloc(&f.Hbar, size_t(n) * L));
  CC(dalloc(&f.gbar, size_t(L) * L));
  CC(dalloc(&f.T, size_t(L) * L));
  CC(dalloc(&f.X, size_t(L) * L));
  CC(dalloc(&f.W, size_t(L) * L));
  CC(dalloc(&f.lam, L));
  CC(dalloc(&f.Bt, size_t(n) * L));
  CC(dalloc(&f.Cpart, size_t(f.nparts) * L * L));
  CC(dalloc(&f.C, size_t(L) * L));
  CC(dalloc(&f.sig, L));
  CC(dalloc(&f.info, 8));
  CC(dalloc(&f.flip, L));
  CC(dalloc(&f.Tu, size_t(L) * L));
  CC(dalloc(&f.M, size_t(L) * L));
  CC(dalloc(&f.mrow, L));
  CC(dalloc(&s->fin_sigma, k));
  CC(dalloc(&s->fin_V, size_t(n) * k));
  CC(dalloc(&s->upass_W, size_t(n) * L));
  CC(dalloc(&s->upass_corr, L));

  CC(cudaMemsetAsync(s->H, 0, sizeof(double) * n * L, s->stream));
  CC(cudaMemsetAsync(s->shift, 0, sizeof(float) * n, s->stream));
  CC(cudaMemsetAsync(s->colsum, 0, sizeof(double) * n, s->stream));
  CC(cudaMemsetAsync(s->sG, 0, sizeof(double) * L, s->stream));
  CC(cudaMemsetAsync(s->gram, 0, sizeof(double) * L * L, s->stream));
  CC(cudaMemsetAsync(s->flags, 0, sizeof(int) * 4, s->stream));
  if (s->tc) {
    CC(launch_omega_op(s->tcw.fmt, seed, n, tc_npad(s->tcw), s->l, L, s->tcw.om16, s->stream,
                       nullptr));
  } else {
    CC(launch_omega_f32(seed, n, s->l, L, s->omega32, L, s->stream));
  }
  CC(cudaStreamSynchronize(s->stream));
#undef CC
  *out = s;
  return SPCA_OK;
}

namespace {

// Staged rows are laid out with a leading dimension rounded up to 4 elements, so that every
// staged FP32 row starts on a 16-byte boundary (a tensor map can describe it).
// leading dimension of the staged copies: rows a multiple of 16 bytes apart (tensor maps)
int64_t stage_ld(int64_t n, size_t es) {
  const int64_t q = es >= 16 ? 1 : static_cast<int64_t>(16 / es);
  return ((n + q - 1) / q) * q;
}

// The two pinned host buffers and two device buffers of the staged paths (made once). An
// allocation that fails leaves none of them behind, so a later call tries again.
spca_status ensure_staging(spca_session* s, size_t row_bytes) {
  if (s->dstage[1]) return SPCA_OK;
  size_t want = kStageBytes;
  if (want < row_bytes) want = row_bytes;
  s->stage_bytes = want;
  for (int i = 0; i < 2; ++i) {
    void* ph = nullptr;
    void* pd = nullptr;
    if (cudaMallocHost(&ph, want) != cudaSuccess || cudaMalloc(&pd, want) != cudaSuccess) {
      cudaGetLastError();
      if (ph) cudaFreeHost(ph);
      for (int j = 0; j < i; ++j) {
        cudaFreeHost(s->pinned[j]);
        cudaFree(s->dstage[j]);
        cudaEventDestroy(s->copied[j]);
        cudaEventDestroy(s->consumed[j]);
        s->pinned[j] = s->dstage[j] = nullptr;
        s->copied[j] = s->consumed[j] = nullptr;
      }
      return fail(s, SPCA_E_NOMEM, "staging allocation of %zu bytes failed", want);
    }
    s->pinned[i] = ph;
    s->dstage[i] = pd;
    CU(cudaEventCreateWithFlags(&s->copied[i], cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&s->consumed[i], cudaEventDisableTiming));
    CU(cudaEventRecord(s->consumed[i], s->stream));
    CU(cudaEventRecord(s->copied[i], s->copy_stream));
  }
  return SPCA_OK;
}

}  // namespace

extern "C++" {
namespace spca {

// Make the staging buffers now where FP32 device rows with leading dimension n go through
// them (only the grouped kernel takes this session, and n x 4 bytes is not a multiple of 16, so
// no tensor map describes the caller's rows): the first such update then allocates nothing.
spca_status session_prepare_staging(spca_session* s) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (!(s->tc && s->tcw.use_grp && !s->tcw.cfg_ok) || (s->n * 4) % 16 == 0) return SPCA_OK;
  CU(cudaSetDevice(s->device));
  return ensure_staging(s, size_t(stage_ld(s->n, 4)) * 4);
}

}  // namespace spca
}  // extern "C++"

spca_status spca_update(spca_session* s, const void* rows, int64_t m_i, int64_t ld, int32_t dtype,
                        const float* block_scale, int32_t rows_on_device, float* G_out) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (m_i < 0) return fail(s, SPCA_E_INVALID, "m_i < 0");
  if (m_i == 0) return SPCA_OK;
  if (!rows) return fail(s, SPCA_E_INVALID, "rows is NULL");
  s->u_ready = false;
  if (ld < s->n) return fail(s, SPCA_E_INVALID, "ld (%lld) < n (%lld)", (long long)ld, (long long)s->n);
  const size_t es = dtype_size(dtype);
  if (es == 0) return fail(s, SPCA_E_INVALID, "unknown dtype %d", dtype);
  float scale = 1.0f;
  if (dtype == SPCA_F8E4M3) {
    if (!block_scale) return fail(s, SPCA_E_INVALID, "FP8 rows need a block_scale");
    scale = *block_scale;
    if (!(scale > 0.0f) || scale != scale) return fail(s, SPCA_E_INVALID, "block_scale must be positive");
  }
  if (rows_on_device != 0 && rows_on_device != 1) return fail(s, SPCA_E_INVALID, "rows_on_device must be 0 or 1");
  CU(cudaSetDevice(s->device));
  if (s->tc && dtype != SPCA_F32 && !(s->tcw.use_grp && (dtype == SPCA_BF16 || dtype == SPCA_F8E4M3)))
    return fail(s, SPCA_E_UNSUPPORTED,
                "this tensor-core session reads FP32 rows (the grouped kernel, which also reads BF16 and FP8 rows, "
                "does not take n = %lld, l = %d)", (long long)s->n, s->l);
  const int64_t mb = s->simt.mb;
  if (rows_on_device) {
    cudaPointerAttributes attr;
    std::memset(&attr, 0, sizeof(attr));
    const bool ok_attr = cudaPointerGetAttributes(&attr, rows) == cudaSuccess;
    cudaGetLastError();
    if (!ok_attr || (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged))
      return fail(s, SPCA_E_INVALID, "rows_on_device=1 but rows is not a device pointer");
    // rows a tensor map cannot describe (not 16-byte aligned, or rows not a multiple of 16
    // bytes apart) go through the staging buffers when only the tensor-map kernel reads them
    const bool tma_ok = (reinterpret_cast<uintptr_t>(rows) % 16 == 0) && ((ld * static_cast<int64_t>(es)) % 16 == 0);
    const bool grp_only = s->tc && s->tcw.use_grp && (!s->tcw.cfg_ok || dtype != SPCA_F32);
    if (!(grp_only && !tma_ok)) {
      for (int64_t r0 = 0; r0 < m_i; r0 += mb) {
        const int64_t mr = (m_i - r0) < mb ? (m_i - r0) : mb;
        const char* base = static_cast<const char*>(rows) + size_t(r0) * ld * es;
        st = run_piece(s, base, mr, ld, dtype, scale, G_out ? G_out + r0 * s->l : nullptr, true);
        if (st != SPCA_OK) return st;
      }
      return SPCA_OK;
    }
    st = flush_tc(s);   // blocks batched before these stay in order
    if (st != SPCA_OK) return st;
    const int64_t lds = stage_ld(s->n, es);
    const size_t row_st = size_t(lds) * es;
    st = ensure_staging(s, row_st);
    if (st != SPCA_OK) return st;
    int64_t piece = static_cast<int64_t>(s->stage_bytes / row_st);
    if (piece > mb) piece = mb;
    for (int64_t r0 = 0; r0 < m_i; r0 += piece) {
      const int64_t mr = (m_i - r0) < piece ? (m_i - r0) : piece;
      const int b = s->next_stage;
      s->next_stage ^= 1;
      const char* src = static_cast<const char*>(rows) + size_t(r0) * ld * es;
      CU(cudaMemcpy2DAsync(s->dstage[b], row_st, src, size_t(ld) * es, size_t(s->n) * es, mr,
                           cudaMemcpyDeviceToDevice, s->stream));
      st = run_piece(s, s->dstage[b], mr, lds, dtype, scale, G_out ? G_out + r0 * s->l : nullptr, false);
      if (st != SPCA_OK) return st;
    }
    return SPCA_OK;
  }
  // Host rows: copy pieces through two staging buffers so the copy of piece i+1
  // overlaps the kernels of piece i.
  const size_t row_bytes = size_t(s->n) * es;
  const int64_t lds = stage_ld(s->n, es);
  const size_t row_st = size_t(lds) * es;
  st = ensure_staging(s, row_st);
  if (st != SPCA_OK) return st;
  int64_t piece = static_cast<int64_t>(s->stage_bytes / row_st);
  if (piece > mb) piece = mb;
  cudaPointerAttributes attr;
  std::memset(&attr, 0, sizeof(attr));
  bool host_pinned = false;
  if (cudaPointerGetAttributes(&attr, rows) == cudaSuccess) host_pinned = (attr.type == cudaMemoryTypeHost);
  cudaGetLastError();
  for (int64_t r0 = 0; r0 < m_i; r0 += piece) {
    const int64_t mr = (m_i - r0) < piece ? (m_i - r0) : piece;
    const int b = s->next_stage;
    s->next_stage ^= 1;
    const char* src = static_cast<const char*>(rows) + size_t(r0) * ld * es;
    CU(cudaStreamWaitEvent(s->copy_stream, s->consumed[b], 0));
    if (host_pinned) {
      CU(cudaMemcpy2DAsync(s->dstage[b], row_st, src, size_t(ld) * es, row_bytes, mr, cudaMemcpyHostToDevice,
                           s->copy_stream));
    } else {
      CU(cudaEventSynchronize(s->copied[b]));   // pinned[b] free again
      char* dst = static_cast<char*>(s->pinned[b]);
      if (ld == lds && lds == s->n) {
        std::memcpy(dst, src, row_st * mr);
      } else {
        for (int64_t r = 0; r < mr; ++r) std::memcpy(dst + r * row_st, src + size_t(r) * ld * es, row_bytes);
      }
      CU(cudaMemcpyAsync(s->dstage[b], dst, row_st * mr, cudaMemcpyHostToDevice, s->copy_stream));
    }
    CU(cudaEventRecord(s->copied[b], s->copy_stream));
    CU(cudaStreamWaitEvent(s->stream, s->copied[b], 0));
    st = run_piece(s, s->dstage[b], mr, lds, dtype, scale, G_out ? G_out + r0 * s->l : nullptr, false);
    if (st != SPCA_OK) return st;
    CU(cudaEventRecord(s->consumed[b], s->stream));
  }
  if (!host_pinned) {
    // the caller's buffer has been copied into pinned memory already; nothing more to wait for
  } else {
    CU(cudaStreamSynchronize(s->copy_stream));   // caller may reuse its pinned buffer on return
  }
  return SPCA_OK;
}

spca_status spca_finalize(spca_session* s, double* sigma, double* V, int32_t out_on_device) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (!sigma || !V) return fail(s, SPCA_E_INVALID, "sigma and V must be non-NULL");
  if (s->m < 1) return fail(s, SPCA_E_NUMERIC, "no rows accumulated yet");
  CU(cudaSetDevice(s->device));
  st = flush_tc(s);
  if (st != SPCA_OK) return st;
  double* sd = out_on_device ? sigma : s->fin_sigma;
  double* vd = out_on_device ? V : s->fin_V;
  CU(finalize_run(s->state(), s->fin, s->opt.center ? s->m : 0, s->k, sd, vd, s->stream, &s->prof, s->m,
                  s->opt.center != 0));
  CU(launch_upass_w(s->state(), vd, sd, s->k, s->upass_W, s->stream));
  s->upass_corr_ready = false;
  if (!out_on_device) {
    CU(cudaMemcpyAsync(sigma, sd, sizeof(double) * s->k, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaMemcpyAsync(V, vd, sizeof(double) * s->n * s->k, cudaMemcpyDeviceToHost, s->stream));
  }
  // the non-finite flag is read after the finalisation kernels so that the stream never idles mid-call
  CU(cudaMemcpyAsync(s->host_flags, s->flags, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CU(cudaStreamSynchronize(s->stream));
  if (s->host_flags[0] & 16)
    return fail(s, SPCA_E_CUDA, "the grouped tensor-core kernel was launched with a configuration it does not take");
  if (s->host_flags[0] & 8) return fail(s, SPCA_E_CUDA, "a copy of the tensor-core pass was out of its buffer (skipped)");
  if (s->host_flags[0] & 2) return fail(s, SPCA_E_TIMEOUT, "a bounded device wait gave up during the pass");
  if (s->host_flags[0] & 1) return fail(s, SPCA_E_NUMERIC, "non-finite values (NaN/Inf) reached the sketch");
  s->u_ready = true;
  return SPCA_OK;
}

spca_status spca_left_vectors(spca_session* s, const float* G, int64_t m, double* U, int32_t out_on_device) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (!s->u_ready) return fail(s, SPCA_E_STATE, "spca_left_vectors needs a spca_finalize after the last update");
  if (m < 0) return fail(s, SPCA_E_INVALID, "m < 0");
  if (m == 0) return SPCA_OK;
  if (!G || !U) return fail(s, SPCA_E_INVALID, "G and U must be non-NULL");
  if (out_on_device != 0 && out_on_device != 1) return fail(s, SPCA_E_INVALID, "out_on_device must be 0 or 1");
  CU(cudaSetDevice(s->device));
  {
    cudaPointerAttributes attr;
    std::memset(&attr, 0, sizeof(attr));
    const bool ok = cudaPointerGetAttributes(&attr, G) == cudaSuccess;
    cudaGetLastError();
    if (!ok || (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged))
      return fail(s, SPCA_E_INVALID, "G must be device memory (the G_out rows of spca_update)");
  }
  CU(launch_u_map(s->state(), s->fin, s->k, s->opt.center ? s->m : 0, s->stream));
  if (out_on_device) {
    CU(launch_left_vectors(s->state(), s->fin, s->k, G, 0, m, U, m, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return SPCA_OK;
  }
  // host output: through the finalisation's n x k scratch, in pieces of rows
  const int64_t piece = s->n;
  for (int64_t r0 = 0; r0 < m; r0 += piece) {
    const int64_t mc = (m - r0) < piece ? (m - r0) : piece;
    CU(launch_left_vectors(s->state(), s->fin, s->k, G, r0, mc, s->fin_V, mc, s->stream));
    CU(cudaMemcpy2DAsync(U + r0, sizeof(double) * m, s->fin_V, sizeof(double) * mc, sizeof(double) * mc, s->k,
                         cudaMemcpyDeviceToHost, s->stream));
  }
  CU(cudaStreamSynchronize(s->stream));
  return SPCA_OK;
}

spca_status spca_left_vectors_pass(spca_session* s, const void* rows, int64_t m, int64_t ld, int32_t dtype,
                                   const float* block_scale, double* U, int64_t ldu) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (!s->u_ready) return fail(s, SPCA_E_STATE, "spca_left_vectors_pass needs a spca_finalize after the last update");
  if (m < 0) return fail(s, SPCA_E_INVALID, "m < 0");
  if (m == 0) return SPCA_OK;
  if (!rows || !U) return fail(s, SPCA_E_INVALID, "rows and U must be non-NULL");
  if (ld < s->n) return fail(s, SPCA_E_INVALID, "ld (%lld) < n (%lld)", (long long)ld, (long long)s->n);
  if (ldu < m) return fail(s, SPCA_E_INVALID, "ldu (%lld) < m (%lld)", (long long)ldu, (long long)m);
  if (dtype_size(dtype) == 0) return fail(s, SPCA_E_INVALID, "unknown dtype %d", dtype);
  float scale = 1.0f;
  if (dtype == SPCA_F8E4M3) {
    if (!block_scale) return fail(s, SPCA_E_INVALID, "FP8 rows need a block_scale");
    scale = *block_scale;
    if (!(scale > 0.0f) || scale != scale) return fail(s, SPCA_E_INVALID, "block_scale must be positive");
  }
  CU(cudaSetDevice(s->device));
  for (const void* p : {static_cast<const void*>(rows), static_cast<const void*>(U)}) {
    cudaPointerAttributes attr;
    std::memset(&attr, 0, sizeof(attr));
    const bool ok = cudaPointerGetAttributes(&attr, p) == cudaSuccess;
    cudaGetLastError();
    if (!ok || (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged))
      return fail(s, SPCA_E_INVALID, "rows and U must be device memory");
  }
  float* gpart = s->simt.Gpart;
  int64_t gp_rows = s->simt.gp_rows;
  if (!gpart) {   // tensor-core sessions keep no split-K workspace: one for this pass, made once
    gp_rows = 65536;
    if (!s->upass_gpart) {
      const cudaError_t e = cudaMalloc(&s->upass_gpart, sizeof(float) * size_t(gp_rows) * s->L);
      if (e != cudaSuccess) {
        cudaGetLastError();
        s->upass_gpart = nullptr;
        return fail(s, e == cudaErrorMemoryAllocation ? SPCA_E_NOMEM : SPCA_E_CUDA, "second-pass workspace: %s",
                    cudaGetErrorString(e));
      }
    }
    gpart = s->upass_gpart;
  }
  if (!s->upass_corr_ready) {   // the centring term, once per finalize (the state is unchanged since)
    CU(launch_upass_corr(s->state(), s->upass_W, s->opt.center ? s->m : 0, s->upass_corr, s->stream));
    s->upass_corr_ready = true;
  }
  CU(launch_u_pass(rows, dtype, scale, m, s->n, ld, s->shift, s->upass_W, s->L, s->k, s->upass_corr, gpart, gp_rows,
                   U, ldu, s->stream));
  return SPCA_OK;
}

spca_status spca_wait_selftest(int64_t limit_ns, void* cuda_stream) {
  if (limit_ns < 1 || limit_ns > 60000000000LL)
    return fail(nullptr, SPCA_E_INVALID, "spca_wait_selftest: limit_ns must be in [1, 6e10]");
  bool ran_out = false;
  const cudaError_t e = grp_wait_selftest(static_cast<uint64_t>(limit_ns), static_cast<cudaStream_t>(cuda_stream),
                                          &ran_out);
  if (e != cudaSuccess) return fail(nullptr, SPCA_E_CUDA, "spca_wait_selftest: %s", cudaGetErrorString(e));
  if (ran_out) return fail(nullptr, SPCA_E_TIMEOUT, "the bounded wait gave up after %lld ns", (long long)limit_ns);
  return SPCA_OK;
}

// ---------------------------------------------------------------- checkpoint / resume
// Layout: the header below, then H (n L doubles), the Gram matrix (L L doubles), the column
// sums (n doubles), the sums of G (L doubles), the shift (n floats), the FP16 operand scale
// (one float) and, after a power step, Omega (n L floats, or the tensor-core operand layout:
// npad L halves).
namespace {
struct CkptHeader {
  char magic[8];           // "SPCAST1"
  int64_t n, m;
  int32_t k, p, l, L, math, center;
  uint64_t seed;
  int32_t shift_set, scale_set, omega_orth, reserved;
  int64_t omega_bytes;
};
constexpr char kCkptMagic[8] = {'S', 'P', 'C', 'A', 'S', 'T', '1', 0};

int64_t ckpt_omega_bytes(const spca_session* s) {
  if (!s->omega_orth) return 0;
  return s->tc ? tc_npad(s->tcw) * s->L * int64_t(sizeof(uint16_t)) : s->n * s->L * int64_t(sizeof(float));
}

size_t ckpt_bytes(const spca_session* s) {
  const size_t n = size_t(s->n), L = size_t(s->L);
  return sizeof(CkptHeader) + sizeof(double) * (n * L + L * L + n + L) + sizeof(float) * (n + 1) +
         size_t(ckpt_omega_bytes(s));
}
}  // namespace

spca_status spca_state_bytes(spca_session* s, size_t* bytes) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (!bytes) return fail(s, SPCA_E_INVALID, "bytes is NULL");
  *bytes = ckpt_bytes(s);
  return SPCA_OK;
}

spca_status spca_save_state(spca_session* s, void* buf, size_t bytes) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (!buf) return fail(s, SPCA_E_INVALID, "buf is NULL");
  if (bytes < ckpt_bytes(s)) return fail(s, SPCA_E_INVALID, "buffer of %zu bytes < %zu", bytes, ckpt_bytes(s));
  CU(cudaSetDevice(s->device));
  st = flush_tc(s);
  if (st != SPCA_OK) return st;
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kCkptMagic, sizeof(h.magic));
  h.n = s->n; h.m = s->m; h.k = s->k; h.p = s->p; h.l = s->l; h.L = s->L;
  h.math = s->opt.math; h.center = s->opt.center; h.seed = s->seed;
  h.shift_set = s->shift_set; h.scale_set = s->scale_set; h.omega_orth = s->omega_orth;
  h.omega_bytes = ckpt_omega_bytes(s);
  char* out = static_cast<char*>(buf);
  std::memcpy(out, &h, sizeof(h));
  size_t off = sizeof(h);
  const size_t n = size_t(s->n), L = size_t(s->L);
  auto get = [&](const void* dev, size_t nb) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(out + off, dev, nb, cudaMemcpyDeviceToHost, s->stream);
    off += nb;
    return e;
  };
  CU(get(s->H, sizeof(double) * n * L));
  CU(get(s->gram, sizeof(double) * L * L));
  CU(get(s->colsum, sizeof(double) * n));
  CU(get(s->sG, sizeof(double) * L));
  CU(get(s->shift, sizeof(float) * n));
  if (s->tc) {
    CU(get(s->tcw.scale, sizeof(float)));
  } else {
    const float one = 1.0f;
    std::memcpy(out + off, &one, sizeof(float));
    off += sizeof(float);
  }
  if (h.omega_bytes > 0) CU(get(s->tc ? static_cast<const void*>(s->tcw.om16) : s->omega32, size_t(h.omega_bytes)));
  CU(cudaStreamSynchronize(s->stream));
  return SPCA_OK;
}

spca_status spca_load_state(spca_session* s, const void* buf, size_t bytes) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (!buf) return fail(s, SPCA_E_INVALID, "buf is NULL");
  CkptHeader h;
  if (bytes < sizeof(h)) return fail(s, SPCA_E_INVALID, "buffer shorter than a checkpoint header");
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kCkptMagic, sizeof(h.magic)) != 0) return fail(s, SPCA_E_INVALID, "not a checkpoint");
  if (h.n != s->n || h.k != s->k || h.p != s->p || h.L != s->L || h.math != s->opt.math ||
      h.center != s->opt.center || h.seed != s->seed)
    return fail(s, SPCA_E_INVALID, "checkpoint of another session (n, k, p, seed, math or centering differ)");
  if (h.m < 0 || (h.omega_orth != 0 && h.omega_orth != 1)) return fail(s, SPCA_E_INVALID, "corrupt checkpoint header");
  const bool orth = h.omega_orth != 0;
  const int64_t ob = orth ? (s->tc ? tc_npad(s->tcw) * s->L * int64_t(sizeof(uint16_t))
                                   : s->n * s->L * int64_t(sizeof(float)))
                          : 0;
  if (h.omega_bytes != ob) return fail(s, SPCA_E_INVALID, "corrupt checkpoint header");
  const size_t n = size_t(s->n), L = size_t(s->L);
  const size_t need = sizeof(h) + sizeof(double) * (n * L + L * L + n + L) + sizeof(float) * (n + 1) + size_t(ob);
  if (bytes < need) return fail(s, SPCA_E_INVALID, "checkpoint of %zu bytes is truncated (%zu needed)", bytes, need);
  CU(cudaSetDevice(s->device));
  st = flush_tc(s);
  if (st != SPCA_OK) return st;
  s->pend.nseg = 0;
  s->pend.rows_total = 0;
  const char* in = static_cast<const char*>(buf);
  size_t off = sizeof(h);
  auto put = [&](void* dev, size_t nb) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(dev, in + off, nb, cudaMemcpyHostToDevice, s->stream);
    off += nb;
    return e;
  };
  CU(put(s->H, sizeof(double) * n * L));
  CU(put(s->gram, sizeof(double) * L * L));
  CU(put(s->colsum, sizeof(double) * n));
  CU(put(s->sG, sizeof(double) * L));
  CU(put(s->shift, sizeof(float) * n));
  if (s->tc) CU(put(s->tcw.scale, sizeof(float)));
  else off += sizeof(float);
  if (orth) {
    CU(put(s->tc ? static_cast<void*>(s->tcw.om16) : static_cast<void*>(s->omega32), size_t(ob)));
  } else if (s->omega_orth) {   // back to the seed's Gaussian Omega
    if (s->tc) CU(launch_omega_op(s->tcw.fmt, s->seed, s->n, tc_npad(s->tcw), s->l, s->L, s->tcw.om16, s->stream, &s->prof));
    else CU(launch_omega_f32(s->seed, s->n, s->l, s->L, s->omega32, s->L, s->stream, &s->prof));
  }
  CU(cudaMemsetAsync(s->flags, 0, sizeof(int) * 4, s->stream));
  CU(cudaStreamSynchronize(s->stream));
  s->m = h.m;
  s->shift_set = h.shift_set != 0;
  s->scale_set = h.scale_set != 0;
  s->omega_orth = orth;
  s->u_ready = false;
  return SPCA_OK;
}

spca_status spca_power_step(spca_session* s) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (s->m < 1) return fail(s, SPCA_E_NUMERIC, "no rows accumulated yet");
  CU(cudaSetDevice(s->device));
  st = flush_tc(s);
  if (st != SPCA_OK) return st;
  const double* Q = nullptr;
  CU(power_omega_run(s->state(), s->fin, s->opt.center ? s->m : 0, s->stream, &Q));
  CU(cudaMemcpyAsync(s->host_flags, s->fin.info + 6, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CU(cudaStreamSynchronize(s->stream));
  if (s->host_flags[0] != 0)
    return fail(s, SPCA_E_NUMERIC, "H is numerically rank deficient: no orthonormal basis of rank l for the power step");
  // Omega <- orth(H_bar) in the pass's operand format, then the accumulators of the next pass
  if (s->tc) {
    CU(launch_omega_from_q_op(s->tcw.fmt, Q, s->n, tc_npad(s->tcw), s->l, s->L, s->tcw.om16, s->stream));
  } else {
    CU(launch_omega_from_q_f32(Q, s->n, s->l, s->L, s->omega32, s->stream));
  }
  const int L = s->L;
  CU(cudaMemsetAsync(s->H, 0, sizeof(double) * s->n * L, s->stream));
  CU(cudaMemsetAsync(s->colsum, 0, sizeof(double) * s->n, s->stream));
  CU(cudaMemsetAsync(s->sG, 0, sizeof(double) * L, s->stream));
  CU(cudaMemsetAsync(s->gram, 0, sizeof(double) * L * L, s->stream));
  CU(cudaStreamSynchronize(s->stream));
  s->m = 0;                  // the shift c stays: the next pass centres on the same c
  s->scale_set = false;      // FP16: the operand scale of the new Omega (unit columns)
  s->u_ready = false;
  s->omega_orth = true;
  return SPCA_OK;
}

spca_status spca_get_state(spca_session* s, double* H_bar, double* gram_bar, double* colsum, float* shift,
                           int64_t* m) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  CU(cudaSetDevice(s->device));
  st = flush_tc(s);
  if (st != SPCA_OK) return st;
  CU(centered_state(s->state(), s->fin, s->opt.center ? s->m : 0, s->stream));
  const int L = s->L, l = s->l;
  if (H_bar)
    CU(cudaMemcpy2DAsync(H_bar, sizeof(double) * l, s->fin.Hbar, sizeof(double) * L, sizeof(double) * l, s->n,
                         cudaMemcpyDeviceToHost, s->stream));
  if (gram_bar)
    CU(cudaMemcpy2DAsync(gram_bar, sizeof(double) * l, s->fin.gbar, sizeof(double) * L, sizeof(double) * l, l,
                         cudaMemcpyDeviceToHost, s->stream));
  if (colsum) CU(cudaMemcpyAsync(colsum, s->colsum, sizeof(double) * s->n, cudaMemcpyDeviceToHost, s->stream));
  if (shift) CU(cudaMemcpyAsync(shift, s->shift, sizeof(float) * s->n, cudaMemcpyDeviceToHost, s->stream));
  CU(cudaStreamSynchronize(s->stream));
  if (m) *m = s->m;
  return SPCA_OK;
}

spca_status spca_merge(spca_session* dst, const spca_session* src) {
  spca_session* s = dst;
  spca_status st = check_usable(dst);
  if (st != SPCA_OK) return st;
  if (!src) return fail(s, SPCA_E_INVALID, "src is NULL");
  if (src->failed) return fail(s, SPCA_E_STATE, "src session is in an error state");
  if (src->n != dst->n || src->k != dst->k || src->p != dst->p || src->seed != dst->seed ||
      src->opt.center != dst->opt.center || src->device != dst->device)
    return fail(s, SPCA_E_INVALID, "sessions differ in n, k, p, seed, centering or device");
  if (src->opt.math != dst->opt.math) return fail(s, SPCA_E_INVALID, "sessions differ in math form");
  if (src->omega_orth || dst->omega_orth)
    return fail(s, SPCA_E_STATE, "sessions after a power step have their own Omega and do not merge");
  CU(cudaSetDevice(dst->device));
  st = flush_tc(dst);
  if (st != SPCA_OK) return st;
  {
    // src's batched blocks belong to its sum too (flushing does not change what it represents)
    spca_session* ms = const_cast<spca_session*>(src);
    st = flush_tc(ms);
    if (st != SPCA_OK) return fail(s, st, "flushing src failed: %s", ms->err);
  }
  CU(cudaStreamSynchronize(src->stream));
  if (dst->opt.center && src->shift_set && !dst->shift_set) {
    // dst has seen no rows: it takes src's shift (and operand scale) with its sums
    CU(cudaMemcpyAsync(dst->shift, src->shift, sizeof(float) * dst->n, cudaMemcpyDeviceToDevice, dst->stream));
    dst->shift_set = true;
    if (dst->tc && dst->tcw.fmt == 1 && src->scale_set) {
      CU(cudaMemcpyAsync(dst->tcw.scale, src->tcw.scale, sizeof(float), cudaMemcpyDeviceToDevice, dst->stream));
      dst->scale_set = true;
    }
  }
  if (dst->opt.center && src->shift_set && src->m > 0) {
    // src's sums refer to its own shift: rebase them onto dst's while adding
    const int fmt = dst->tc ? (dst->tcw.fmt == 1 ? 2 : 1) : 0;
    CU(launch_merge_rebase(dst->state(), src->state(), dst->seed, fmt, src->m, dst->fin.lam, dst->stream));
  } else {
    CU(launch_merge(dst->state(), src->state(), dst->stream));
  }
  CU(cudaStreamSynchronize(dst->stream));
  dst->m += src->m;
  dst->u_ready = false;
  return SPCA_OK;
}

spca_status spca_reset(spca_session* s, uint64_t seed) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  CU(cudaSetDevice(s->device));
  const int L = s->L;
  CU(cudaMemsetAsync(s->H, 0, sizeof(double) * s->n * L, s->stream));
  CU(cudaMemsetAsync(s->shift, 0, sizeof(float) * s->n, s->stream));
  CU(cudaMemsetAsync(s->colsum, 0, sizeof(double) * s->n, s->stream));
  CU(cudaMemsetAsync(s->sG, 0, sizeof(double) * L, s->stream));
  CU(cudaMemsetAsync(s->gram, 0, sizeof(double) * L * L, s->stream));
  CU(cudaMemsetAsync(s->flags, 0, sizeof(int) * 4, s->stream));
  s->seed = seed;
  s->pend.nseg = 0;          // blocks batched for the previous pass are dropped with it
  s->pend.rows_total = 0;
  if (s->tc) {
    CU(launch_omega_op(s->tcw.fmt, seed, s->n, tc_npad(s->tcw), s->l, L, s->tcw.om16,
                         s->stream, &s->prof));
  } else {
    CU(launch_omega_f32(seed, s->n, s->l, L, s->omega32, L, s->stream, &s->prof));
  }
  s->m = 0;
  s->shift_set = false;
  s->scale_set = false;
  s->u_ready = false;
  s->omega_orth = false;
  return SPCA_OK;
}

spca_status spca_set_profiling(spca_session* s, int32_t on) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  s->prof.timing = (on != 0);
  return SPCA_OK;
}

spca_status spca_get_profile(spca_session* s, int32_t kernel, double* total_ms, int64_t* launches) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  if (kernel < 0 || kernel >= SPCA_K_COUNT) return fail(s, SPCA_E_INVALID, "unknown kernel class %d", kernel);
  CU(cudaStreamSynchronize(s->stream));
  double tot = 0.0;
  for (int i = 0; i < s->prof.nmarks; ++i) {
    if (s->prof.marks[i].id != kernel) continue;
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, s->prof.marks[i].a, s->prof.marks[i].b));
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = s->prof.launches[kernel];
  return SPCA_OK;
}

spca_status spca_clear_profile(spca_session* s) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  CU(cudaStreamSynchronize(s->stream));
  s->prof.clear();
  return SPCA_OK;
}

spca_status spca_sync(spca_session* s) {
  spca_status st = check_usable(s);
  if (st != SPCA_OK) return st;
  st = flush_tc(s);
  if (st != SPCA_OK) return st;
  CU(cudaStreamSynchronize(s->stream));
  return SPCA_OK;
}

spca_status spca_destroy(spca_session* s) {
  if (!s) return SPCA_OK;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
  free_all(s);
  delete s;
  return SPCA_OK;
}

const char* spca_last_error(const spca_session* s) { return s ? s->err : g_thread_err; }

int64_t spca_rows_seen(const spca_session* s) { return s ? s->m : -1; }

const char* spca_describe(spca_session* s) {
  if (!s) return "";
  if (s->tc && s->tcw.use_grp) {
    const GrpConfig& g = s->tcw.grp;
    snprintf(s->desc, sizeof(s->desc),
             "math=%s kernel=grouped n=%lld l=%d L=%d group=%d groups=%d ctas=%d blocks_per_cta=%d mtiles=%d "
             "stages=%d d1=%d fresh_h=%d smem=%u",
             s->tcw.fmt == 1 ? "fp16" : "bf16", (long long)s->n, s->l, s->L, g.S, g.NG, g.S * g.NG, g.nbmax, g.nu,
             g.ns1, g.nd1, g.nf, g.smem);
  } else if (s->tc) {
    snprintf(s->desc, sizeof(s->desc),
             "math=%s kernel=%s n=%lld l=%d L=%d cluster=%d w=%d clusters=%d ctas=%d smem=%u",
             s->tcw.fmt == 1 ? "fp16" : "bf16", s->tcw.v3 ? "pipelined" : "resident", (long long)s->n, s->l, s->L,
             s->tcw.v3 ? s->tcw.cfg3.CS : s->tcw.cfg.CS, s->tcw.v3 ? s->tcw.cfg3.w : s->tcw.cfg.w,
             s->tcw.v3 ? s->tcw.cfg3.nclusters : s->tcw.cfg.nclusters,
             s->tcw.v3 ? s->tcw.cfg3.nclusters * s->tcw.cfg3.CS : s->tcw.cfg.nclusters * s->tcw.cfg.CS,
             s->tcw.v3 ? s->tcw.cfg3.smem : s->tcw.cfg.smem);
  } else {
    snprintf(s->desc, sizeof(s->desc), "math=fp32 n=%lld l=%d L=%d max_block_rows=%lld row_splits<=%d",
             (long long)s->n, s->l, s->L, (long long)s->simt.mb, s->simt.T);
  }
  return s->desc;
}

spca_status spca_omega_words(uint64_t seed, int64_t n, int32_t l, uint32_t* out) {
  spca_session* s = nullptr;
  if (n < 1 || l < 1 || !out) return fail(nullptr, SPCA_E_INVALID, "bad arguments");
  CU(launch_omega_words(seed, n, l, out, 0));
  CU(cudaDeviceSynchronize());
  return SPCA_OK;
}

spca_status spca_shift_static(const void* rows, int64_t m, int64_t n, int64_t ld, int32_t dtype,
                              const float* block_scale, float* shift, void* cuda_stream) {
  spca_session* s = nullptr;
  if (!rows || !shift) return fail(nullptr, SPCA_E_INVALID, "spca_shift_static: NULL rows or shift");
  if (m < 1 || n < 1 || ld < n)
    return fail(nullptr, SPCA_E_INVALID, "spca_shift_static: need m >= 1, n >= 1, ld >= n (m=%lld n=%lld ld=%lld)",
                (long long)m, (long long)n, (long long)ld);
  if (n > SPCA_SHIFT_STATIC_MAX_N)
    return fail(nullptr, SPCA_E_INVALID,
                "spca_shift_static: n = %lld exceeds the fixed scratch (n <= %d); use a session instead",
                (long long)n, SPCA_SHIFT_STATIC_MAX_N);
  if (dtype_size(dtype) == 0) return fail(nullptr, SPCA_E_INVALID, "spca_shift_static: unknown dtype %d", dtype);
  float scale = 1.0f;
  if (dtype == SPCA_F8E4M3) {
    if (!block_scale) return fail(nullptr, SPCA_E_INVALID, "spca_shift_static: FP8 rows need a block_scale");
    scale = *block_scale;
    if (!(scale > 0.0f)) return fail(nullptr, SPCA_E_INVALID, "spca_shift_static: block_scale must be positive");
  }
  double* scratch = nullptr;
  CU(shift_static_scratch(&scratch));
  Prof quiet;   // counts only: records no events and allocates nothing
  CU(launch_shift(rows, dtype, m, n, ld, scale, shift, scratch, static_cast<cudaStream_t>(cuda_stream), &quiet));
  return SPCA_OK;
}

spca_status spca_omega(uint64_t seed, int64_t n, int32_t l, float* out) {
  spca_session* s = nullptr;
  if (n < 1 || l < 1 || !out) return fail(nullptr, SPCA_E_INVALID, "bad arguments");
  // FP32 Omega with ld = l: generate into a padded scratch then compact
  const int L = pad_l(l);
  float* tmp = nullptr;
  CU(cudaMalloc(&tmp, sizeof(float) * n * L));
  cudaError_t e = launch_omega_f32(seed, n, l, L, tmp, L, 0);
  if (e == cudaSuccess)
    e = cudaMemcpy2D(out, sizeof(float) * l, tmp, sizeof(float) * L, sizeof(float) * l, n, cudaMemcpyDeviceToDevice);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(nullptr, SPCA_E_CUDA, "omega: %s", cudaGetErrorString(e));
  CU(cudaDeviceSynchronize());
  return SPCA_OK;
}

}  // extern "C"
