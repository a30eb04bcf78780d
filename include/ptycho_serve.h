/*
 * ptycho_serve.h — batching and serving of many reconstructions on one GPU.
 *
 * Each reconstruction is one context of include/ptycho.h running the
 * generalised divide-and-concur update x <- a P^b_C P^c_D x + (1 - a) x
 * (Introduction, the displayed equation) with its own (a, b, c).  Scans of
 * different sizes keep their exit waves, object and probe resident in HBM;
 * their iterations run concurrently on separate streams.
 *
 * Batch: a fixed set of loaded contexts advanced together; from the second
 * iteration on, one iteration of every context is captured into a single
 * CUDA graph and replayed, so a round of the whole batch is one graph launch.
 * In that graph the FP32 cluster-design contexts of one pattern side run as
 * one launch group: one divide launch over all their exit waves (a work list
 * of (scan, wave) items, however uneven the scans) and one launch per concur
 * kernel over all their scans; other contexts have a branch of their own.
 *
 * Server: a request queue with admission by an HBM budget, continuous
 * batching (requests join the active set as memory and slots free up, loaded
 * while the other requests' iterations run) and per-request latency.
 *
 * Same conventions as ptycho.h: status codes, host buffers copied, outputs to
 * caller-allocated host buffers; a batch or server is not thread-safe.
 */
#ifndef PTYCHO_SERVE_H
#define PTYCHO_SERVE_H

#include "ptycho.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ptycho_batch ptycho_batch;

/* Create an empty batch on device opts->device (opts may be NULL).
 * Errors: EINVAL, ECUDA. */
int ptycho_batch_create(ptycho_batch** out, const ptycho_opts* opts);

/* Add a context that has a scan loaded, with the (a, b, c) it iterates with.
 * The batch does not own the context.  Errors: EINVAL, ESTATE (no scan). */
int ptycho_batch_add(ptycho_batch* batch, ptycho_ctx* ctx, float a, float b, float c);

/* Advance every context of the batch by n_iter iterations.  The first
 * iteration (and any in which a context holds its probe fixed) is launched
 * directly; the others replay one captured graph.  Results are those of
 * ptycho_iterate(ctx, a, b, c, n_iter) on each context alone, bit for bit
 * (a launch group may pin its contexts' concur launch shapes to a common
 * choice, which changes no result).  Synchronises.
 * Errors: EINVAL (n_iter < 0), ESTATE (empty), ENOMEM, ECUDA. */
int ptycho_batch_run(ptycho_batch* batch, int32_t n_iter);

/* How a batch replays its iterations: PTYCHO_BATCH_GROUPS (launch groups, as
 * above), PTYCHO_BATCH_BRANCHES (a graph branch per context: scans overlap
 * across streams but each launches its own kernels), or PTYCHO_BATCH_AUTO
 * (the default: with at least three replays, one timed replay of each and
 * then the faster).  Both compute the same iterations, bit for bit. */
enum { PTYCHO_BATCH_AUTO = 0, PTYCHO_BATCH_GROUPS = 1, PTYCHO_BATCH_BRANCHES = 2 };
int ptycho_batch_set_mode(ptycho_batch* batch, int mode);  /* Errors: EINVAL. */

typedef struct {
    int32_t groups;       /* launch groups of the last run (0: none used) */
    int32_t in_groups;    /* contexts that ran in them */
    int32_t used;         /* the graph replayed: PTYCHO_BATCH_GROUPS or _BRANCHES */
    float groups_ms;      /* auto mode: one timed replay of each graph (else 0) */
    float branches_ms;
} ptycho_batch_info_t;

/* What the last ptycho_batch_run did.  Errors: EINVAL. */
int ptycho_batch_info(const ptycho_batch* batch, ptycho_batch_info_t* out);

/* Release the batch (not its contexts).  NULL is a no-op. */
void ptycho_batch_destroy(ptycho_batch* batch);

typedef struct ptycho_server ptycho_server;

/* One reconstruction request: a scan in host memory, with the same layout and
 * rules as ptycho_load_scan. */
typedef struct {
    int32_t J, N, M_rows, M_cols;
    const int32_t* pos_rc;   /* [J][2] */
    const float* intensity;  /* [J][N][N] */
    const float* obj0;       /* [M_rows][M_cols][2] */
    const float* probe0;     /* [N][N][2] */
} ptycho_scan_desc;

/* Create a server on opts->device that keeps at most max_active
 * reconstructions resident and admits a request only while the device bytes
 * of the active ones plus the request's (ptycho_scan_bytes) stay within
 * hbm_budget_bytes and within the device's free memory.  Errors: EINVAL, ECUDA. */
int ptycho_server_create(ptycho_server** out, size_t hbm_budget_bytes, int32_t max_active,
                         const ptycho_opts* opts);

/* Queue a request: n_iter iterations of (a, b, c) on the scan.  The scan is
 * copied (the caller may free its buffers on return).  *req_id receives the
 * request's id.  Errors: EINVAL (bad sizes or values, a scan that could
 * never fit the budget). */
int ptycho_server_submit(ptycho_server* srv, const ptycho_scan_desc* scan, float a, float b,
                         float c, int32_t n_iter, uint64_t* req_id);

/* One scheduling step, which does not wait for the device to drain: retire
 * requests whose iterations have all finished (results copied to host,
 * device memory freed), admit queued requests in arrival order while they fit
 * (their scans loaded while the other requests' work runs; a request that
 * does not fit the device's free memory while nothing else is active fails,
 * state PTYCHO_REQ_FAILED), and enqueue the
 * next iters_per_round iterations of every active request whose previous
 * round has finished, each on its own stream.  When none of these can be
 * done it first waits (at most 2 s) for some round to finish.  Call it until
 * n_active and n_queued are 0.  n_active / n_queued (either may be NULL)
 * receive the counts after the step.  Errors: EINVAL, ECUDA. */
int ptycho_server_step(ptycho_server* srv, int32_t iters_per_round, int32_t* n_active,
                       int32_t* n_queued);

/* Request states reported by ptycho_server_poll. */
enum { PTYCHO_REQ_QUEUED = 0, PTYCHO_REQ_ACTIVE = 1, PTYCHO_REQ_DONE = 2, PTYCHO_REQ_FAILED = 3 };

/* State of a request; when done, copy its object and probe (either may be
 * NULL) and times[0..3] = seconds from submission to admission, seconds from
 * submission to completion, seconds of service per 100 iterations, and the
 * final model Fourier error E_F(P * O_j) (times may be NULL).
 * Errors: EINVAL (unknown id). */
int ptycho_server_poll(ptycho_server* srv, uint64_t req_id, int32_t* state, float* obj_out,
                       float* probe_out, double* times);

/* Release every request and context of the server.  NULL is a no-op. */
void ptycho_server_destroy(ptycho_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* PTYCHO_SERVE_H */
