/*
 * spca.h - C ABI of the GB300 single-pass randomized PCA library.
 *
 * The method is Alg. 4 of Yu, Gu, Li, Liu, Li, "Single-Pass PCA of Large
 * High-Dimensional Data" (IJCAI 2017): one streaming pass over the rows of an
 * m x n data matrix A forms G = A Omega with an n x l Gaussian test matrix Omega
 * (Alg. 4 steps 3-6) and accumulates H = A^T G row block by row block (Alg. 4
 * step 7, Eq. 11); a small finalisation turns (G, H, Omega) into the leading k
 * singular values and right singular vectors (Alg. 4 steps 9-20). Here G is not
 * kept: the pass also accumulates the Gram matrix G^T G, the column sums of the
 * (shifted) data and of G, and the finalisation takes R from the Gram matrix
 * (Thm 1: Q = G R^-1 is orthonormal and B = Q^T A = R^-T H^T).
 *
 * Conventions for every call:
 *  - Every function returns an spca_status; none aborts or exits. On failure
 *    spca_last_error() describes the cause. A CUDA error puts the session in an
 *    error state; later calls on it return SPCA_E_STATE.
 *  - All matrices are row-major unless stated. "device" pointers are CUDA
 *    device addresses on the session's device; "host" pointers are ordinary
 *    (pageable or pinned) host memory.
 *  - The caller owns every buffer it passes in; the library owns the session
 *    and everything reachable from it.
 *  - Sizes: n >= 1, k >= 1, p >= 0, l = k + p with l <= min(n, 256).
 *  - Work is issued on the session's CUDA stream (the one given in the options,
 *    or a stream the library creates). Calls on one session must not overlap in
 *    time from several host threads.
 */
#ifndef SPCA_H_
#define SPCA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spca_session spca_session;

typedef enum {
  SPCA_OK = 0,
  SPCA_E_INVALID = 1,     /* bad argument (shape, dtype, pointer, size)        */
  SPCA_E_NOMEM = 2,       /* device or pinned-host allocation failed           */
  SPCA_E_CUDA = 3,        /* a CUDA runtime call or kernel launch failed       */
  SPCA_E_STATE = 4,       /* call not valid in the session's state             */
  SPCA_E_NUMERIC = 5,     /* NaN/Inf seen in the data, or no rows accumulated  */
  SPCA_E_TIMEOUT = 6,     /* a bounded device wait gave up                     */
  SPCA_E_UNSUPPORTED = 7  /* valid request this build or device cannot serve   */
} spca_status;

/* Storage type of the rows handed to spca_update. */
typedef enum {
  SPCA_F32 = 0,
  SPCA_BF16 = 1,
  SPCA_F8E4M3 = 2,        /* OCP E4M3 ("fn"): value = code * block_scale       */
  SPCA_F64 = 3
} spca_dtype;

/* Arithmetic of the two contractions of the pass (a3: G = A Omega, a4: H += A^T G). */
typedef enum {
  SPCA_MATH_FP32 = 0,     /* FP32 CUDA-core FMA, FP32 accumulate               */
  SPCA_MATH_BF16 = 1,     /* BF16 tensor-core operands, FP32 accumulate        */
  SPCA_MATH_BF16X2 = 2,   /* split BF16 (hi + lo) operands, FP32 accumulate    */
  SPCA_MATH_FP8 = 3,      /* FP8 E4M3 operands, FP32 accumulate                */
  SPCA_MATH_FP16 = 4      /* FP16 tensor-core operands on the shifted rows and G
                             scaled by one power of two per pass (chosen from the
                             first rows so that G stays below 2^14), FP32
                             accumulate: 8x finer rounding than BF16 at the same
                             operand size and rate. Later rows more than about
                             4x longer than the first ones overflow FP16 and
                             make spca_finalize return SPCA_E_NUMERIC.          */
} spca_math;

typedef struct {
  int32_t math;           /* spca_math; default SPCA_MATH_FP32                 */
  int32_t center;         /* 1 (default): principal components of the column-
                             centred data; 0: of the raw rows                   */
  int32_t max_block_rows; /* largest row count one internal launch handles;
                             0 = library default (8192). Bigger updates are
                             processed in pieces of this many rows.            */
  int32_t reserved;       /* must be 0                                         */
  void* cuda_stream;      /* cudaStream_t to work on; NULL = library-owned     */
} spca_options;

/* Fill *opt with the defaults. */
void spca_default_options(spca_options* opt);

/*
 * spca_create - start a streaming PCA session (Alg. 4 steps 1-3).
 *   n     number of features (columns of A)
 *   k     number of principal components wanted
 *   p     oversampling (the paper's s): l = k + p columns of Omega
 *   seed  64-bit key of the Philox4x32-10 stream that defines Omega:
 *         Omega[j, 4q + t] is normal t of the Box-Muller transform of the four
 *         words of Philox(counter = (j mod 2^32, j div 2^32, q, 0),
 *         key = (seed mod 2^32, seed div 2^32)), uniforms u = (x + 1/2) 2^-32
 *   opt   options or NULL for defaults
 *   out   receives the session handle (owned by the library; free it with
 *         spca_destroy)
 * Allocates the session's device state (H: n x l FP32, Omega, the Gram matrix,
 * the sums and a workspace of O((n + max_block_rows) l) floats): constant in m.
 * Errors: SPCA_E_INVALID (sizes), SPCA_E_NOMEM, SPCA_E_CUDA, SPCA_E_UNSUPPORTED
 * (math form not available on this device).
 */
spca_status spca_create(int64_t n, int32_t k, int32_t p, uint64_t seed,
                        const spca_options* opt, spca_session** out);

/*
 * spca_update - fold the next rows of A into the sketch (Alg. 4 steps 5-7,
 * Eq. 11; row order does not change the result in exact arithmetic).
 *   rows            m_i x n block, row-major with leading dimension ld >= n
 *                   elements, of type dtype
 *   block_scale     SPCA_F8E4M3 only: one FP32 scale for the whole block
 *                   (host pointer); ignored otherwise (may be NULL)
 *   rows_on_device  1: rows is a device pointer, read in place on the session
 *                   stream (the caller keeps it valid and unmodified until the
 *                   stream has passed this work, e.g. until spca_sync). The rows
 *                   must be ready when the call is made: a stream the library
 *                   created is not ordered after the caller's streams (give the
 *                   caller's stream in the options, or synchronise first);
 *                   0: rows is host memory, copied through the session's pinned
 *                   staging buffers; the call returns once the copy of the last
 *                   piece has been issued and the caller's buffer is no longer
 *                   read.
 *   G_out           optional device pointer (NULL = none) receiving the m_i x l
 *                   sketch rows G_i = (A_i - 1 c^T) Omega (row-major, ld = l)
 *                   as this pass computes them, c being the session's shift
 *                   (the FP32 column mean of the first rows seen when centering
 *                   is on, else 0).
 * Tensor-core sessions read BF16 and FP8 rows in their storage format when the
 * grouped kernel takes (n, l) (spca_describe says "kernel=grouped"): the operand is
 * (value - c) s rounded once to the operand format, value = code x block_scale for
 * FP8. A block of another format than the pending ones is launched separately.
 * Device rows whose start or row pitch is not a multiple of 16 bytes are copied to
 * the session's staging buffers first. Other tensor-core sessions read FP32 rows
 * only (SPCA_E_UNSUPPORTED otherwise).
 * m_i = 0 is a no-op. Errors: SPCA_E_INVALID, SPCA_E_CUDA, SPCA_E_STATE,
 * SPCA_E_UNSUPPORTED.
 */
spca_status spca_update(spca_session* s, const void* rows, int64_t m_i, int64_t ld,
                        int32_t dtype, const float* block_scale, int32_t rows_on_device,
                        float* G_out);

/*
 * spca_finalize - leading k singular values and right singular vectors of the
 * (centred) rows seen so far (Alg. 4 steps 9-20, FP64 on the device).
 *   sigma  k doubles, descending; entries beyond the numerical rank are 0
 *   V      n x k doubles, COLUMN-major (column i at V + i*n); column i is
 *          scaled by +-1 so that its entry of largest magnitude (lowest index
 *          on ties) is positive; columns for zero sigma are 0
 *   out_on_device  1: sigma and V are device pointers; 0: host pointers
 * Synchronises the session stream. Non-destructive: updates may continue.
 * Errors: SPCA_E_INVALID, SPCA_E_NUMERIC (no rows yet, or NaN/Inf in the
 * accumulated state), SPCA_E_CUDA, SPCA_E_STATE.
 */
spca_status spca_finalize(spca_session* s, double* sigma, double* V, int32_t out_on_device);

/*
 * spca_left_vectors - U, the leading k left singular vectors of the (centred)
 * rows, from the sketch rows G that spca_update returned in G_out (Alg. 4
 * steps 18-19: U = Q U~, with Q = G_bar R^-1 the orthonormal basis of the
 * sketch in the Gram reading of Thm 1 and U~ the left singular vectors of B).
 * Needs a spca_finalize after the last update, merge or reset; uses its R and
 * U~, so that A_bar ~ U diag(sigma) V^T with the V that call returned.
 *   G      device, m x l FP32, row-major with leading dimension l: the G_out
 *          rows of the rows seen (any subset or order: row r of U belongs to
 *          row r of G)
 *   m      rows of G (0 is a no-op)
 *   U      m x k doubles, COLUMN-major (column i at U + i*m); column i has the
 *          sign that makes U diag(sigma) V^T the approximation; columns for
 *          zero sigma are 0
 *   out_on_device  1: U is a device pointer; 0: host memory
 * With centering, G_bar = G - (1/m_seen) 1 sG^T uses the session's sums of G.
 * Synchronises the session stream.
 * Errors: SPCA_E_STATE (no finalize since the state last changed),
 * SPCA_E_INVALID (NULL pointers, G not in device memory), SPCA_E_CUDA.
 */
spca_status spca_left_vectors(spca_session* s, const float* G, int64_t m, double* U, int32_t out_on_device);

/*
 * spca_left_vectors_pass - U of given rows by a second pass over them, for callers
 * that kept no sketch rows (G_out): U = A_bar V Sigma^-1, the truncated SVD
 * A_bar ~ U diag(sigma) V^T solved for U with the sigma and V of the last
 * spca_finalize (Alg. 4 step 18 forms U from the stored sketch instead; with an
 * exactly rank-r matrix, r <= k, both give its left singular vectors).
 *   rows   device, m x n row-major with leading dimension ld >= n, of type dtype
 *          (block_scale as in spca_update for FP8 rows); any rows, e.g. the rows
 *          of the pass block by block: row r of U belongs to row r of rows
 *   U      device, m x k doubles, COLUMN-major with leading dimension ldu >= m
 *          (column i at U + i*ldu)
 * With centering, the column means mu = c + s_hat / m_seen of all rows seen are
 * subtracted: (a - mu) V Sigma^-1 = (a - c) W - (s_hat / m_seen)^T W, W = V Sigma^-1
 * in FP32 (products in FP32, sums of the slices and the centring term in FP64).
 * Columns for zero sigma are 0. Runs on the session stream and returns without
 * waiting: U is complete once the stream has passed the work (spca_sync). The
 * first call on a tensor-core session allocates a workspace of 65536 x L floats.
 * Errors: SPCA_E_STATE (no finalize since the state last changed),
 * SPCA_E_INVALID (NULL or host pointers, sizes), SPCA_E_NOMEM, SPCA_E_CUDA.
 */
spca_status spca_left_vectors_pass(spca_session* s, const void* rows, int64_t m, int64_t ld, int32_t dtype,
                                   const float* block_scale, double* U, int64_t ldu);

/*
 * spca_power_step - the power scheme with P = 1 (Sec. 3.2 and Sec. 4): for
 * Alg. 4, run the while loop once more with Omega replaced by H after "orth".
 * Replaces Omega by the orthonormal basis of the centred H_bar of the rows seen
 * so far (Cholesky QR twice, FP64 on the device; stored in the pass's operand
 * format) and clears H, the Gram matrix, the sums and the row count; the shift c
 * is kept. The caller then passes over the same rows again (spca_update) and
 * calls spca_finalize, which returns the result for (A A^T) A: the same
 * singular vectors with the tail's relative weight reduced.
 * A session after a power step does not merge (SPCA_E_STATE); spca_reset goes
 * back to the Gaussian Omega. Synchronises the session stream.
 * Errors: SPCA_E_NUMERIC (no rows yet, or H_bar numerically of rank < l; the
 * session is then unchanged), SPCA_E_CUDA, SPCA_E_STATE.
 */
spca_status spca_power_step(spca_session* s);

/*
 * Checkpoint and resume. The session's state is a sum over the rows seen (Eq. 11),
 * so a pass stopped after any block resumes from its accumulators: save them, and
 * load them into a session created with the same n, k, p, seed and options (in
 * this or another process), then continue with spca_update.
 *   spca_state_bytes  host bytes of a checkpoint of this session
 *   spca_save_state   write it into buf (host memory, >= spca_state_bytes);
 *                     flushes pending tensor-core blocks, synchronises
 *   spca_load_state   restore it (the session's own accumulators are replaced);
 *                     synchronises
 * A checkpoint holds H, the Gram matrix, the sums, the shift, the FP16 operand
 * scale, the row count and, after spca_power_step, Omega. Layout (native byte
 * order, host): a fixed header (magic "SPCAST1", n, m, k, p, l, L, math,
 * center, seed, flags, the size of the Omega part), then the arrays in that
 * order. Errors: SPCA_E_INVALID (NULL pointers, short buffer, a checkpoint of
 * a session with other n, k, p, seed, math or centering), SPCA_E_CUDA.
 */
spca_status spca_state_bytes(spca_session* s, size_t* bytes);
spca_status spca_save_state(spca_session* s, void* buf, size_t bytes);
spca_status spca_load_state(spca_session* s, const void* buf, size_t bytes);

/*
 * spca_get_state - the centred accumulators, for inspection and parity tests.
 *   H_bar    n x l doubles, row-major: A_bar^T G_bar (NULL = skip)
 *   gram_bar l x l doubles: G_bar^T G_bar (NULL = skip)
 *   colsum   n doubles: column sums of the shifted rows A - 1 c^T (NULL = skip)
 *   shift    n floats: the shift c (NULL = skip)
 *   m        receives the number of rows seen (NULL = skip)
 * with A_bar, G_bar the column-centred data and sketch (or the raw ones when
 * centering is off). All output pointers are host memory. Synchronises.
 */
spca_status spca_get_state(spca_session* s, double* H_bar, double* gram_bar,
                           double* colsum, float* shift, int64_t* m);

/*
 * spca_merge - dst += src for two sessions that saw disjoint row sets of the
 * same data (same n, k, p, seed, math form and centering). The sketch is a sum
 * over rows (Eq. 11), so the merged session equals one session that saw both
 * row sets. With centering, each session subtracts the shift c of its own first
 * rows; src's sums are rebased onto dst's shift while adding (delta = c_src -
 * c_dst, gamma = Omega^T delta: H += H_s + s_s gamma^T + delta sG_s^T +
 * m_s delta gamma^T, and likewise for the Gram matrix and the sums). A dst
 * without rows takes src's shift. Both sessions must be on the same device.
 * Synchronises both streams. src is not modified.
 * Errors: SPCA_E_INVALID (mismatch), SPCA_E_CUDA, SPCA_E_STATE.
 */
spca_status spca_merge(spca_session* dst, const spca_session* src);

/*
 * spca_wait_selftest - exercise the bounded wait that every cross-CTA and pipeline
 * wait of the tensor-core pass uses: one thread waits, with limit limit_ns, for a
 * device counter that nothing writes, gives up, and the call reports it. Returns
 * SPCA_E_TIMEOUT after about limit_ns (the expected outcome; the device stays
 * usable) and never SPCA_OK. The pass kernels' own limit is half a second, or
 * SPCA_WAIT_LIMIT_MS milliseconds (1 .. 60000) from the environment at
 * spca_create; a wait that runs out there ends the launch early and the next
 * synchronising call returns SPCA_E_TIMEOUT. Not part of the paper: an
 * operational check. cuda_stream may be NULL (the legacy default stream).
 * Errors: SPCA_E_INVALID (limit_ns outside [1, 6e10]), SPCA_E_CUDA.
 */
spca_status spca_wait_selftest(int64_t limit_ns, void* cuda_stream);

/* Wait until all work issued on the session's stream is done. */
spca_status spca_sync(spca_session* s);

/* Release the session and its device memory (after synchronising). NULL is ok. */
spca_status spca_destroy(spca_session* s);

/* Text of the last error on s (or of the calling thread when s is NULL). */
const char* spca_last_error(const spca_session* s);

/* Number of rows of A seen so far, or -1 for a NULL session. */
int64_t spca_rows_seen(const spca_session* s);

/*
 * spca_describe - one-line text describing the session's arithmetic and launch
 * configuration (math form, padded l, cluster size, features per CTA, clusters,
 * shared memory per CTA). The string is owned by the session and valid until the
 * next call on it; "" for a NULL session.
 */
const char* spca_describe(spca_session* s);

/*
 * spca_reset - start a new pass on the same session: zero H, the Gram matrix,
 * the sums and the row count, forget the shift, and regenerate Omega for
 * `seed` (Alg. 4 steps 1-3 again, without reallocating). Stream-ordered.
 */
spca_status spca_reset(spca_session* s, uint64_t seed);

/* Kernel classes reported by spca_get_profile. */
typedef enum {
  SPCA_K_OMEGA = 0,       /* a1: Omega generation                          */
  SPCA_K_SHIFT = 1,       /* a2: shift (column mean of the first rows)     */
  SPCA_K_G_PARTIAL = 2,   /* a3: G = A_hat Omega contraction               */
  SPCA_K_G_FINISH = 3,    /* a3/a5: split reduction, Gram and sum partials */
  SPCA_K_GRAM_ACCUM = 4,  /* a5: FP64 Gram and sum accumulation            */
  SPCA_K_H_PARTIAL = 5,   /* a4: H += A_hat^T G contraction (+ col sums)   */
  SPCA_K_H_FINISH = 6,    /* a4/a5: split reduction into H and col sums    */
  SPCA_K_FINALIZE = 7,    /* a7: all FP64 finalisation kernels together    */
  SPCA_K_TC_SKETCH = 8,   /* a2-a5 fused on the tensor cores (BF16 math)    */
  SPCA_K_COUNT = 9
} spca_kernel_id;

/*
 * spca_set_profiling - when on (1), every kernel launch of the session is
 * bracketed by CUDA events on the session stream, so that spca_get_profile can
 * report per-class device time. Launch counts are kept either way.
 */
spca_status spca_set_profiling(spca_session* s, int32_t on);

/*
 * spca_get_profile - for kernel class `kernel` (spca_kernel_id): total device
 * milliseconds of the launches timed since the last spca_clear_profile (0 when
 * profiling was off) and the number of launches. Synchronises the stream.
 */
spca_status spca_get_profile(spca_session* s, int32_t kernel, double* total_ms, int64_t* launches);

/* Forget the recorded launches and times. */
spca_status spca_clear_profile(spca_session* s);

/*
 * spca_omega_words - the raw Philox4x32-10 words behind Omega (a1), for
 * bit-exact checks: out (device, uint32) receives n x 4*ceil(l/4) words, row j
 * holding the words of counters (j, q = 0..ceil(l/4)-1) in order. Synchronous.
 */
spca_status spca_omega_words(uint64_t seed, int64_t n, int32_t l, uint32_t* out);

/*
 * spca_omega - Omega itself (a1) as FP32, n x l row-major, into device memory
 * out (ld = l): the FP64 Box-Muller normals rounded to FP32. Synchronous.
 */
spca_status spca_omega(uint64_t seed, int64_t n, int32_t l, float* out);

/*
 * spca_shift_static - the centering shift c exactly as a session computes it
 * from its first rows (FP32 of the FP64 column means of `rows`),
 * without allocating anything. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory at that moment, such
 * as a serving loop that has committed its device memory to admitted sessions,
 * or one that must not call cudaMalloc/cudaFree because those calls
 * synchronise the whole device and would stall every other session's work.
 * The 64 partial column sums it needs live in a fixed device array compiled
 * into the library (64 x SPCA_SHIFT_STATIC_MAX_N doubles, 8 MiB per device).
 *   rows        device, m x n row-major, leading dimension ld >= n (elements),
 *               element type dtype (spca_dtype)
 *   block_scale SPCA_F8E4M3 only: host pointer to the block's FP32 scale
 *   shift       device, n floats, overwritten
 *   cuda_stream cudaStream_t to enqueue on (NULL = the legacy default stream);
 *               the call returns once the two launches are enqueued
 * Nothing has to start at zero: each partial is written before it is read.
 * Errors: SPCA_E_INVALID (no CUDA call made) for m < 1, n < 1,
 * n > SPCA_SHIFT_STATIC_MAX_N, ld < n, a NULL pointer, an unknown dtype or a
 * missing or non-positive FP8 scale; SPCA_E_CUDA if the address lookup or a
 * launch fails. The first call on each device looks the array's address up
 * (cudaGetSymbolAddress with that device current), which may load the
 * library's device code: make that first call before any stream capture.
 * All calls on a device share the one array, so calls whose launches can
 * overlap (other streams, other host threads) race on it: serialise them.
 */
#define SPCA_SHIFT_STATIC_MAX_N 16384
spca_status spca_shift_static(const void* rows, int64_t m, int64_t n, int64_t ld, int32_t dtype,
                              const float* block_scale, float* shift, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SPCA_H_ */
