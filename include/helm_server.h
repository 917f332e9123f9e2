/*
 * helm_server.h -- solve server of libhelm: batched Helmholtz solve requests of different
 * grids, frequencies, precisions and right-hand-side counts, with the factors kept resident
 * on the device.  The paper has no counterpart (it solves one problem family at a time); the
 * server reuses helm_assemble / helm_factor / helm_solve / helm_adjoint_solve of helm.h
 * unchanged, so each request's result is the one those calls give.
 *
 * Model:
 *   - A model is a squared-slowness field on a grid (helm_server_add_model); the server
 *     keeps a device copy of m.
 *   - A request asks for X = A(m, w)^{-1} B (or A^H) for one model, one frequency w, one
 *     precision and nrhs right-hand sides.  B and X are host arrays [nrhs][N] of helm_c128
 *     owned by the caller; they must stay valid (B unchanged) until helm_server_wait returns
 *     for the request.  Pinned host memory makes the copies asynchronous.
 *   - Factor cache: one entry per (model, w, precision) holds the operator and its factor
 *     (with its refinement scratch) and a CUDA stream of its own.  Entries are evicted least
 *     recently used first, never while a batch uses them.
 *   - HBM admission: every device byte of the server is accounted (entries and the working
 *     memory of batches in flight) against hbm_budget_bytes.  A request whose own footprint
 *     (its factor plus its working memory) exceeds the budget is refused at submission
 *     (HELM_ENOMEM); otherwise it waits until evictions make room.  Footprints are computed
 *     from the documented sizes: factor nx*nz^2*(8 mixed | 16 FP64) + 96 B per node,
 *     working memory 32 B per node and right-hand side (device B and X) plus 64 B (mixed
 *     refinement), plus 1 MiB per entry.
 *   - Batching: a worker takes the oldest queued request whose entry is not in use by
 *     another worker, adds the later queued requests with the same (model, w, precision,
 *     adjoint) key up to max_batch_rhs right-hand sides, and solves them as one block with
 *     the smallest rtol of the batch.
 *   - Latency of a request: submission (arrival) to the end of the copy of its X to the host.
 *
 * Threading: submit, wait and stats may be called from any host threads concurrently.
 * No entry point aborts, exits or throws; each returns a helm_status (helm.h).
 */
#ifndef HELM_SERVER_H
#define HELM_SERVER_H

#include <stddef.h>
#include <stdint.h>
#include "helm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_server helm_server_t;

typedef struct {
    uint64_t hbm_budget_bytes;   /* device bytes the server may hold; 0: 180 GiB */
    int32_t max_batch_rhs;       /* right-hand sides per batched solve; <= 0: 128 */
    int32_t workers;             /* host worker threads (batches in flight); <= 0: 8 */
    int32_t max_iter;            /* refinement cap of mixed solves; <= 0: 10 */
} helm_server_opts;

typedef struct {
    int32_t model;          /* id from helm_server_add_model */
    double omega;           /* angular frequency */
    int32_t prec;           /* helm_prec */
    int32_t adjoint;        /* nonzero: solve with A^H */
    int32_t nrhs;           /* >= 1 */
    const helm_c128 *B;     /* host [nrhs][N] */
    helm_c128 *X;           /* host [nrhs][N] */
    double rtol;            /* residual tolerance of mixed solves */
} helm_request;

typedef struct {
    int32_t status;         /* helm_status of the request's solve */
    int32_t cache_hit;      /* 1 if the factor was resident when the batch started */
    int32_t batch_rhs;      /* right-hand sides of the batch it ran in */
    int32_t iters;          /* refinement sweeps of the batch (1 for FP64) */
    double max_relres;      /* of the batch, as helm_solve_info */
    double queue_ms;        /* arrival -> batch start */
    double total_ms;        /* arrival -> X on the host */
} helm_request_info;

typedef struct {
    int64_t submitted, completed, refused;
    int64_t rhs_solved;
    int64_t batches;
    int64_t factor_builds, cache_hits, evictions;
    int64_t entries;                    /* resident factors */
    uint64_t bytes_used, bytes_peak;    /* accounted device bytes now and at most */
    uint64_t bytes_budget;
} helm_server_counters;

/* helm_server_create -- start the server and its workers.  opts may be NULL (defaults).
 * Errors: EINVAL (budget below 1 MiB), ECUDA. */
helm_status helm_server_create(const helm_server_opts *opts, helm_server_t **out);

/* helm_server_add_model -- register m (host [N] squared slowness > 0) on grid; *model_id
 * receives the id.  Errors: EINVAL, ENOMEM, ECUDA. */
helm_status helm_server_add_model(helm_server_t *s, const helm_grid *grid, const double *m_host,
                                  int32_t *model_id);

/* helm_server_footprint -- device bytes a request of nrhs right-hand sides for this model
 * and precision needs (its factor plus its working memory), as admission counts them. */
uint64_t helm_server_footprint(const helm_server_t *s, int32_t model_id, int32_t prec, int32_t nrhs);

/* helm_server_submit -- queue a request; *ticket identifies it for helm_server_wait.
 * Errors: EINVAL (unknown model, nrhs < 1, NULL arrays, omega <= 0, bad precision),
 * ENOMEM (footprint above the budget: refused, not queued). */
helm_status helm_server_submit(helm_server_t *s, const helm_request *req, int64_t *ticket);

/* helm_server_wait -- block until the request is done; fills info (may be NULL) and
 * returns the request's status.  Each ticket can be waited for once.  EINVAL for an
 * unknown ticket. */
helm_status helm_server_wait(helm_server_t *s, int64_t ticket, helm_request_info *info);

/* helm_server_stats -- counters (any time). */
helm_status helm_server_stats(const helm_server_t *s, helm_server_counters *out);

/* helm_server_destroy -- finish queued requests, stop the workers, free every device
 * byte of the server.  Requests not yet waited for are dropped with their results written. */
void helm_server_destroy(helm_server_t *s);

#ifdef __cplusplus
}
#endif

#endif /* HELM_SERVER_H */
