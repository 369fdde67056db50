// Internal declarations shared by the translation units of the library.
// Not part of the public ABI (see include/spca.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "spca.h"

namespace spca {

// Runs f once per device (kernel attributes are per device), from any number of host
// threads: done holds one bit per device that has been set up (devices 0..63).
template <class F>
cudaError_t once_per_device(std::atomic<uint64_t>& done, std::mutex& mu, F f) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev >= 0 && dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = f();
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

constexpr int kMaxL = 256;          // largest l accepted
constexpr int kDefaultBlockRows = 8192;

// Round l up to the column padding of the device state.
inline int pad_l(int l) { return ((l + 15) / 16) * 16; }

// Launch accounting: every launcher calls begin/end around each kernel it enqueues.
// Counts are always kept; events are recorded only when timing is on.
struct Prof {
  int64_t launches[SPCA_K_COUNT] = {0};
  bool timing = false;
  struct Mark { int id; cudaEvent_t a, b; };
  Mark* marks = nullptr;   // recorded begin/end pairs (events reused after clear)
  int nmarks = 0, cap = 0;
  void begin(int id, cudaStream_t st);
  void end(int id, cudaStream_t st);
  void clear() { nmarks = 0; for (int i = 0; i < SPCA_K_COUNT; ++i) launches[i] = 0; }
  void release();
};

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `st` and returns the launch error (cudaGetLastError).

// a1: Omega as FP32 (n x L row-major, columns >= l zero) and raw Philox words.
cudaError_t launch_omega_f32(uint64_t seed, int64_t n, int l, int L, float* out, int64_t ld,
                             cudaStream_t st, Prof* prof = nullptr);
cudaError_t launch_omega_words(uint64_t seed, int64_t n, int l, uint32_t* out, cudaStream_t st);
// Omega from a matrix Q (n x L FP64, ld L), as FP32 / in the tensor-core operand layout
cudaError_t launch_omega_from_q_f32(const double* Q, int64_t n, int l, int L, float* out, cudaStream_t st);
cudaError_t launch_omega_from_q_op(int fmt, const double* Q, int64_t n, int64_t npad, int l, int L, uint16_t* out,
                                   cudaStream_t st);

// Shift c = FP32 of the FP64 column mean of the given rows; part: kShiftParts x n doubles.
constexpr int kShiftParts = 64;
cudaError_t launch_shift(const void* rows, int dtype, int64_t m, int64_t n, int64_t ld,
                         float scale, float* shift, double* part, cudaStream_t st, Prof* prof);

// Address of the fixed scratch of spca_shift_static on the current device (kShiftParts x
// SPCA_SHIFT_STATIC_MAX_N doubles); looked up once per device, then cached.
cudaError_t shift_static_scratch(double** out);

// FP32 SIMT pass over one piece of rows (a2-a5). Workspace pointers are owned by the session.
struct SimtWork {
  float* Gpart;       // gp_rows x L (split partials, S x rows_padded)
  float* G;           // mb x L
  double* gram_part;  // ceil(mb/32) x L x L (double-float group sums)
  double* sG_part;    // ceil(mb/32) x L
  float* Hpart;       // T x n x L
  float* cs_part;     // T x n
  int T;              // max row splits of the H contraction
  int64_t gp_rows;    // capacity of Gpart in rows (>= mb rounded up to 128)
  int64_t mb;         // max rows per piece
};

struct State {
  int64_t n;
  int l, L;
  const float* omega32;   // n x L
  double* H;              // n x L (FP64 state)
  const float* shift;     // n
  double* colsum;         // n
  double* sG;             // L
  double* gram;           // L x L
  int* flags;             // [0]: non-finite value seen
};

cudaError_t simt_pass(const State& s, const SimtWork& w, const void* rows, int dtype,
                      float scale, int64_t m, int64_t ld, float* G_out, cudaStream_t st, Prof* prof);

// Merge: dst += src (H, colsum, sG, gram).
cudaError_t launch_merge(const State& dst, const State& src, cudaStream_t st);
// Merge with the shift rebase from src's shift to dst's (fmt: 0 FP32, 1 BF16, 2 FP16 Omega);
// gamma: l doubles of scratch.
cudaError_t launch_merge_rebase(const State& dst, const State& src, uint64_t seed, int fmt, int64_t m_src,
                                double* gamma, cudaStream_t st);

// gram += sum of `parts` partial Gram matrices (fixed order), sG likewise.
cudaError_t launch_gram_accum(const double* gram_part, const double* sG_part, int parts, int L, double* gram,
                              double* sG, cudaStream_t st);

// ---------------------------------------------------------------- tensor-core pass (BF16)
struct TcConfig {
  int CS;             // cluster size (CTAs sharing one row tile, splitting the features)
  int w;              // features per CTA (multiple of 128)
  int nclusters;      // co-resident clusters launched
  uint32_t smem;      // dynamic shared memory per CTA
};

// the grouped kernel (sketch_grp.cu): NG groups of S CTAs; per CTA at most nbmax 64-feature
// blocks (nu 128-feature M-tiles of H), ns1 FP32 stages, nd1 D1 buffers; nf: per-tile fresh H
// buffers (1 or 2) added into a running H in TMEM (0: H drains to the partials every few tiles)
struct GrpConfig {
  int S, NG, nbt, nbmax, nu, ns1, nd1, nf;
  uint32_t smem;
  bool gram_in;          // the reducers accumulate the Gram matrix; else G' rows go to TcWork::gfull
};

struct TcWork {
  TcConfig cfg;          // the kernel holding each tile's operand (sketch_tc.cu); valid when cfg_ok
  bool cfg_ok;
  TcConfig cfg3;         // the pipelined kernel (sketch_tc3.cu), used when v3 is set
  bool v3;
  GrpConfig grp;         // the grouped kernel (sketch_grp.cu), preferred when use_grp is set
  bool use_grp;
  uint16_t* zero8k;      // grouped kernel: 8 KB of zeros
  float* part;           // grouped kernel: the groups' partial rings
  uint16_t* gbuf;        // grouped kernel: the groups' G' rings
  unsigned* cnt;         // grouped kernel: the groups' counters
  float* gfull;          // grouped kernel without in-kernel Gram: the launch's G' rows (tiles x 128 x L)
  int64_t gfull_rows;    // rows gfull holds
  uint64_t wait_ns = 500000000ull;   // grouped kernel: limit of each pipeline wait
  int fmt;               // 0: BF16 operands; 1: FP16 operands on values scaled by *scale
  float* scale;          // device scalar: power-of-two operand scale (FP16 form)
  unsigned int* scale_bits;   // device scratch for the largest row norm
  uint16_t* om16;        // Omega in the operand format, pre-swizzled 64-feature chunks (CS*w/64 x L x 64)
  float* Hpart;          // nclusters x (CS*w) x L; column l carries the column sums
  double* gram_part;     // nclusters*CS x L x L
  double* sG_part;       // nclusters*CS x L
  uint16_t* img;         // pipelined kernel: converted operand images, nclusters*CS x 2 tiles x 128 w
};

constexpr int kTcPendingMax = 48;       // row blocks batched into one launch
constexpr int64_t kTcPendingRows = 65536;

struct TcPending {
  int nseg = 0;
  int64_t rows_total = 0;
  int dtype = 0;                  // spca_dtype of every pending block (FP32 unless the grouped kernel runs)
  const void* rows[kTcPendingMax];
  int64_t m[kTcPendingMax];
  int64_t ld[kTcPendingMax];
  float* gout[kTcPendingMax];
  float dscale[kTcPendingMax];    // FP8 blocks: the block scale; else 1
};

// Whether (n, L) fits the fused kernel; fills the launch configuration.
bool tc_config(int64_t n, int L, int fmt, TcConfig* cfg);
const char* tc_config_reason();   // why the last tc_config call said no
cudaError_t launch_omega_op(int fmt, uint64_t seed, int64_t n, int64_t npad, int l, int L, uint16_t* out,
                            cudaStream_t st, Prof* prof);
// FP16 form: s = power of two from the largest shifted row norm of the given rows and a bound
// on the norm of Omega's columns
cudaError_t launch_op_scale(const void* rows, int dtype, float dscale, int64_t m, int64_t n, int64_t ld,
                            const float* shift, unsigned int* bits, float* scale, double omega_norm, cudaStream_t st,
                            Prof* prof);
cudaError_t tc_pass(const State& s, const TcWork& w, const TcPending& pend, cudaStream_t st, Prof* prof);
// H partials -> FP64 state and Gram partials -> state, for a launch of ncl clusters
cudaError_t launch_tc_finish(const State& s, const TcWork& w, int ncl, int64_t npad, int nctas, cudaStream_t st,
                             Prof* prof);
// the pipelined kernel: configuration, and one pass (sets *used = false, launching nothing,
// when a row block cannot be read through a tensor map)
bool tc3_config(int64_t n, int L, int fmt, TcConfig* cfg);
// the grouped kernel: configuration for (n, l, L), its buffer sizes (elements), and one pass
// (sets *used = false, launching nothing, when a row block cannot be read through a tensor map)
bool grp_config(int64_t n, int l, int L, int fmt, GrpConfig* cfg);
const char* grp_config_reason();
size_t grp_img_elems(const GrpConfig& c);
size_t grp_part_elems(const GrpConfig& c, int L);
size_t grp_gbuf_elems(const GrpConfig& c, int L, int fmt);
size_t grp_cnt_elems(const GrpConfig& c);
size_t grp_gfull_rows(const GrpConfig& c, int64_t max_block_rows);
// One thread polls a device counter that nothing writes with the pipeline's bounded wait;
// *ran_out = true when the wait gave up after limit_ns (the expected outcome).
cudaError_t grp_wait_selftest(uint64_t limit_ns, cudaStream_t st, bool* ran_out);
cudaError_t grp_pass(const State& s, const TcWork& w, const TcPending& pend, cudaStream_t st, Prof* prof,
                     bool* used);
const char* tc3_config_reason();
cudaError_t tc3_pass(const State& s, const TcWork& w, const TcPending& pend, cudaStream_t st, Prof* prof,
                     bool* used);

// FP64 finalisation (a7). Scratch is owned by the session.
struct FinalWork {
  double* Hbar;       // n x L
  double* gbar;       // L x L
  double* T;          // L x L
  double* X;          // L x L
  double* W;          // L x L
  double* lam;        // L
  double* Bt;         // n x L
  double* Cpart;      // nparts x L x L
  double* C;          // L x L
  double* sig;        // L
  double* Vtmp;       // n x k
  double* flip;       // L: the sign applied to each column of V
  double* Tu;         // L x L: T (= R^-T) of the last finalize
  double* M;          // l x k: sketch rows to left singular vectors (after a finalize)
  double* mrow;       // k: the centring term of that map
  int* info;          // [0]: rank kept, [1]: route (0 chol, 1 eigen), [2]-[4]: solver sweeps, [6]: power step failed
  int nparts;
};

// m: the row count used by the centering algebra (0 when centering is off);
// rows_seen / centered bound the rank of the Gram matrix (m - 1 when centred).
cudaError_t finalize_run(const State& s, const FinalWork& f, int64_t m, int k,
                         double* sigma_dev, double* V_dev, cudaStream_t st, Prof* prof,
                         int64_t rows_seen, bool centered);

cudaError_t centered_state(const State& s, const FinalWork& f, int64_t m, cudaStream_t st);

// the power scheme with P = 1: Q = orth(H_bar) (n x L FP64, in FinalWork scratch) by Cholesky
// QR twice; f.info[6] != 0 afterwards if H_bar was numerically rank deficient
cudaError_t power_omega_run(const State& s, const FinalWork& f, int64_t m, cudaStream_t st, const double** Q);

// the l x k map to U (and its centring term) from the last finalize's R^-T, eigenvectors and
// column signs; m: the rows of the centring (0 when centering is off)
cudaError_t launch_upass_w(const State& s, const double* V, const double* sigma, int k, float* W, cudaStream_t st);
cudaError_t launch_upass_corr(const State& s, const float* W, int64_t m_center, double* corr, cudaStream_t st);
cudaError_t launch_u_pass(const void* rows, int dtype, float scale, int64_t m, int64_t n, int64_t ld,
                          const float* shift, const float* W, int L, int k, const double* corr, float* Gpart,
                          int64_t gp_rows, double* U, int64_t ldu, cudaStream_t st);
cudaError_t launch_u_map(const State& s, const FinalWork& f, int k, int64_t m, cudaStream_t st);

// U rows [row0, row0 + mc) of the last finalize from kept sketch rows G (m x l, FP32), into
// column-major U with leading dimension ldu (device memory)
cudaError_t launch_left_vectors(const State& s, const FinalWork& f, int k, const float* G, int64_t row0, int64_t mc,
                                double* U, int64_t ldu, cudaStream_t st);

// ---------------------------------------------------------------- hooks for the serving loop
size_t session_footprint(int64_t n, int k, int p, int math, int64_t max_block_rows);   // 0: does not fit
cudaStream_t session_stream(spca_session* s);
spca_status session_flush(spca_session* s);
spca_status session_prepare_staging(spca_session* s);
spca_status session_finalize_async(spca_session* s, double* sigma_dev, double* V_dev, int* flags_host);
spca_status session_flags_status(spca_session* s, int flags);
int session_k(const spca_session* s);
int64_t session_n(const spca_session* s);

}  // namespace spca
