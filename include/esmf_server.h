/*
 * esmf_server.h -- C ABI of the build server: many concurrent ESMF
 * optimisations (different molecules, different numbers of densities) asking
 * for grouped J/K builds (Eq. J_and_K; one grouped pass per request as in
 * Sec. II.C) on one GPU.
 *
 * The server keeps each registered molecule's screening data and integral
 * store resident (a handle from esmf_fock_create) while they fit a device-
 * memory budget, evicting idle molecules least-recently-used first and
 * re-creating them on their next request.  Molecules that still have queued
 * requests are evicted last: while other builds are in flight, a request
 * whose molecule has no handle waits (up to 30 s) for room rather than
 * evict one of them, and when it must, the molecule whose next queued request
 * comes latest goes first.  A worker thread admits queued
 * requests whenever an execution slot, the molecule and enough memory are
 * free, so requests that arrive while others run start as soon as resources
 * allow and their work overlaps on the device (one non-blocking CUDA stream
 * per slot).  Builds of one molecule are serialised; different molecules run
 * concurrently.  Each build can be replayed from a captured CUDA graph, or,
 * with batched ticks, the builds admitted together on the tensor-core path
 * run as one esmf_fock_build_batch call: one persistent launch per pass of 16
 * densities for all of them.
 *
 * Conventions as in esmf_fock.h: 0 or a negative ESMF_ERR_* code; buffers are
 * row-major float64; the caller owns them.
 */
#ifndef ESMF_SERVER_H
#define ESMF_SERVER_H

#include <stdint.h>

#include "esmf_fock.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct esmf_server esmf_server_t;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t creates;            /* handles built (first use or after eviction)   */
    int64_t evictions;          /* idle handles released to fit the budget       */
    int64_t graph_launches;     /* builds replayed from a captured CUDA graph    */
    int64_t resident_bytes;     /* device bytes held by resident handles         */
    int64_t peak_inflight;      /* most requests on the device at once           */
    double p50_ms, p99_ms, mean_ms, max_ms;   /* submit-to-ready latency          */
    double span_s;              /* first submit to last completion               */
    int64_t batch_launches;     /* batched ticks issued (ESMF_SERVER_BATCH)      */
    int64_t batched_builds;     /* builds that ran inside a batched tick         */
    int64_t tick_graph_launches;/* batched ticks replayed from a captured graph  */
} esmf_server_stats_t;

/*
 * esmf_server_create -- start a server on `device`.
 *   budget_bytes  device memory the resident handles may hold (> 0)
 *   max_inflight  concurrent requests on the device, 1..64
 *   precision     ESMF_PREC_* used for every molecule's integral store
 *   flags         ESMF_SERVER_GRAPHS: capture each (molecule, m, slot) build
 *                 into a CUDA graph once and replay it;
 *                 ESMF_SERVER_BATCH: batched ticks -- every pass of the
 *                 worker collects the requests it admits whose molecule is on
 *                 the tensor-core path (stored FP16X2/BF16X2), copies their
 *                 inputs on their slots' streams and builds them together
 *                 with esmf_fock_build_batch (up to ESMF_MAX_BATCH per call)
 *                 on a stream of its own; with ESMF_SERVER_GRAPHS also set,
 *                 each tick composition (molecules, density counts, slots) is
 *                 captured into a CUDA graph once and the tick's persistent
 *                 launches are replayed from it (up to 128 compositions are
 *                 kept; graphs are dropped when a member's memory moves).
 *                 Other requests (molecules that fell back to integral-direct
 *                 FP32 under the budget, or FP64/FP32 servers) run as single
 *                 builds, replayed from graphs when ESMF_SERVER_GRAPHS is set.
 *                 The batching across molecules has no counterpart in the
 *                 paper.
 * Errors: INVALID_ARG (also for unknown flag bits), CUDA, OOM.
 */
#define ESMF_SERVER_GRAPHS 1
#define ESMF_SERVER_BATCH  2
/* ESMF_SERVER_EVICT_LARGEST: when memory must be freed, evict the largest
 * idle molecule first (among those with no queued request) instead of the
 * least recently used.  Re-creating a handle costs about the same per byte
 * of store, so freeing the room with fewer, larger evictions means fewer
 * re-creations when requests are spread evenly over the molecules. */
#define ESMF_SERVER_EVICT_LARGEST 4
int esmf_server_create(int device, int64_t budget_bytes, int max_inflight, int precision,
                       int flags, esmf_server_t **out);

/* Register a molecule (the basis is copied); returns its id in *basis_id.
 * The handle is created on the molecule's first request.  Errors: INVALID_ARG. */
int esmf_server_register(esmf_server_t *s, const esmf_basis_t *basis, double schwarz_tol,
                         int *basis_id);

/*
 * Queue one grouped build for molecule basis_id with m densities.
 *   D       host, m x N x N, read when the request is admitted
 *   J, K    host, m x N x N, written before the request completes
 *   traces  host, m doubles, or NULL
 * The buffers must stay valid until esmf_server_wait reports completion.
 * Errors: INVALID_ARG (unknown id, m out of range, NULL buffers).
 */
int esmf_server_submit(esmf_server_t *s, int basis_id, int m, const double *D, double *J,
                       double *K, double *traces, int64_t *ticket);

/* Wait up to timeout_ms (< 0: no limit) for a ticket.  Returns 0 when its
 * results are in the caller's buffers, ESMF_ERR_TIMEOUT if it has not
 * finished yet, or the error the build failed with. */
int esmf_server_wait(esmf_server_t *s, int64_t ticket, int timeout_ms);

/* Statistics since creation or the last reset. */
int esmf_server_stats(esmf_server_t *s, esmf_server_stats_t *out);
int esmf_server_reset_stats(esmf_server_t *s);

/* Stop the worker after the queued requests finish, free everything. */
void esmf_server_destroy(esmf_server_t *s);

#ifdef __cplusplus
}
#endif
#endif /* ESMF_SERVER_H */
