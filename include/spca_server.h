/*
 * spca_server.h - C ABI of the serving loop: many streaming-PCA sessions resident on one
 * device, fed row blocks concurrently.
 *
 * The paper has no serving loop; what makes one possible is its Eq. 11: a session's whole
 * state is the sum over rows of (H, the Gram matrix of G, the column sums) plus the shift,
 * the row count and the seed of Omega, so its memory is constant in m and sessions can stay
 * resident while their rows arrive. The server
 *  - admits sessions against a device-memory budget (a session whose state does not fit
 *    waits, with its requests, until closed sessions free enough memory),
 *  - runs each session on its own CUDA stream, so the work of different sessions overlaps on
 *    the device, and picks up requests that arrive while others run (continuous batching):
 *    the row blocks one session has waiting are folded into one launch of the fused
 *    tensor-core pass,
 *  - records the latency of every update and finalize request (submission to completion)
 *    and reports p50/p99,
 *  - keeps closed sessions, and sessions reserved ahead of time, in a pool with their device
 *    and pinned memory: an admission of the same (n, k, p) and math form takes one and
 *    resets its state for the new seed (as spca_reset), so it allocates nothing on the
 *    worker while other sessions run. Pooled sessions count against the budget and are
 *    freed, oldest first, when an admission of another shape needs their room.
 * A single worker thread owns all sessions and all CUDA work; the calls below only queue
 * requests and may come from any host thread. Rows must be device-resident FP32
 * (row-major, leading dimension ld); the caller keeps them valid and unmodified until the
 * request has completed (spca_server_wait).
 */
#ifndef SPCA_SERVER_H_
#define SPCA_SERVER_H_

#include <stddef.h>
#include <stdint.h>

#include "spca.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spca_server spca_server;

#define SPCA_SERVER_AUTO_MATH (-1)   /* FP16 tensor-core form where it fits, else FP32 */

typedef struct {
  size_t device_bytes;     /* budget for admitted session state; 0 = 80 % of the free device
                              memory when the server is created                          */
  int32_t math;            /* spca_math of every session, or SPCA_SERVER_AUTO_MATH (default) */
  int32_t max_sessions;    /* session slots, 1..4096 (default 1024)                          */
  int32_t max_block_rows;  /* largest update (rows) a session is sized for (default 4096)    */
  int32_t reserved;        /* must be 0                                                      */
} spca_server_options;

typedef struct {
  int64_t updates_done, finalizes_done;
  int64_t sessions_admitted, sessions_waiting;   /* now */
  double update_p50_ms, update_p99_ms;           /* over the most recent 2^20 completed updates */
  double finalize_p50_ms, finalize_p99_ms;       /* likewise for finalisations */
  double rows_bytes;                             /* bytes of rows folded in so far */
  double active_seconds;                         /* wall time with at least one request in flight */
  size_t device_bytes_in_use, device_bytes_budget;   /* admitted sessions; the budget */
  int64_t sessions_pooled;                       /* now */
  int64_t admissions_from_pool, sessions_created;  /* so far (created: admissions and reserves) */
  size_t device_bytes_pooled;                    /* now */
} spca_server_stats;

/* Fill *opt with the defaults. */
void spca_server_default_options(spca_server_options* opt);

/* Start the server and its worker thread on the current device.
 * Errors: SPCA_E_INVALID (options), SPCA_E_NOMEM, SPCA_E_CUDA. */
spca_status spca_server_create(const spca_server_options* opt, spca_server** out);

/*
 * spca_server_open - reserve a session slot for (n, k, p, seed) (the arguments of
 * spca_create). Returns at once with the slot id in *id; the session is created by the
 * worker when the budget allows, and requests queue behind that.
 * Errors: SPCA_E_INVALID (sizes, no free slot), SPCA_E_NOMEM (the session alone exceeds
 * the budget), SPCA_E_UNSUPPORTED (an explicit math form that does not fit).
 */
spca_status spca_server_open(spca_server* sv, int64_t n, int32_t k, int32_t p, uint64_t seed, int32_t* id);

/*
 * spca_server_reserve - queue the creation of `count` sessions of sizes (n, k, p) (math form
 * chosen as for spca_server_open) into the pool, so that later opens of that shape are
 * admitted without allocating. *ticket completes when they exist; its status is
 * SPCA_E_NOMEM if the budget (admitted plus pooled sessions) cannot hold all of them (those
 * made so far stay pooled) or the first failing spca_create's status.
 * Errors: SPCA_E_INVALID (sizes, count < 1, NULL ticket), SPCA_E_NOMEM (one session alone
 * exceeds the budget), SPCA_E_UNSUPPORTED (an explicit math form that does not fit),
 * SPCA_E_STATE (the server is stopping).
 */
spca_status spca_server_reserve(spca_server* sv, int64_t n, int32_t k, int32_t p, int32_t count, uint64_t* ticket);

/*
 * spca_server_update - queue m_i rows (device pointer, FP32, leading dimension ld >= n) for
 * session id; *ticket identifies the request. Errors: SPCA_E_INVALID.
 */
spca_status spca_server_update(spca_server* sv, int32_t id, const float* rows, int64_t m_i, int64_t ld,
                               uint64_t* ticket);

/*
 * spca_server_finalize - queue a finalisation of session id after its queued updates;
 * sigma (k doubles) and V (n x k doubles, column-major as in spca_finalize) are host
 * buffers written before the request completes. Errors: SPCA_E_INVALID.
 */
spca_status spca_server_finalize(spca_server* sv, int32_t id, double* sigma, double* V, uint64_t* ticket);

/* The status of every request that returned a ticket is kept until spca_server_wait has read
 * it: a caller that does not wait on its tickets should expect that record to grow.
 *
 * Wait until request `ticket` completes (timeout_s < 0: no limit) and return its status
 * (SPCA_E_TIMEOUT if the wait timed out; the request itself goes on). For a failed request,
 * spca_server_last_error on the same thread then gives its own reason (with the message of
 * the session that ran it). */
spca_status spca_server_wait(spca_server* sv, uint64_t ticket, double timeout_s);

/* Close session id after its queued requests; the session goes to the pool (its memory stays
 * allocated, counted as pooled) unless it had failed, in which case it is freed. */
spca_status spca_server_close(spca_server* sv, int32_t id);

/* Counters and latency percentiles so far. */
spca_status spca_server_get_stats(spca_server* sv, spca_server_stats* out);

/* Stop the worker after the queued requests and free every session; requests of sessions
 * never admitted complete with SPCA_E_STATE. NULL is ok. */
spca_status spca_server_destroy(spca_server* sv);

/* Text of the last error of a spca_server_* call on the calling thread. */
const char* spca_server_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPCA_SERVER_H_ */
