/*
 * soptx_serve.h -- request server for many concurrent topology-optimisation
 * design jobs on one GPU (continuous batching of the per-iteration hot path
 * of include/soptx.h).
 *
 * Each design job (a `job` id) keeps its mesh, CSR pattern and element data
 * resident on the device between its iterations (Sec. 3.2.2: the invariant
 * parts are computed once and reused).  A request asks for one iteration's
 * K(rho) and sensitivities (Sec. 2.2, Appendix D) of one job.  Requests are
 * admitted in arrival order whenever a slot is free and the job's mesh fits
 * under the HBM cap -- evicting meshes of jobs with no request in flight,
 * least recently used first -- so requests that arrive while others run are
 * started as capacity frees up, and their kernels overlap on a pool of
 * streams.  Requests of one job run in order on that job's stream.
 *
 * The paper has no server; this is the serving pattern built around its
 * assembly path.  All entry points are thread-safe.
 */
#ifndef SOPTX_SERVE_H
#define SOPTX_SERVE_H

#include <stdint.h>

#include "soptx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct soptx_server_s *soptx_server;

typedef struct {
    int64_t hbm_cap_bytes;   /* budget for resident meshes (device bytes)      */
    int32_t max_slots;       /* requests in flight at once (>= 1)             */
    int32_t n_streams;       /* stream pool size (>= 1)                       */
    int32_t max_queue;       /* pending requests accepted before SOPTX_EBUSY  */
    int32_t device;          /* CUDA device ordinal the server runs on        */
    int32_t group_small;     /* 1: requests on small box lattices (see
                              * soptx_assemble_and_sensitivity_group) are
                              * launched together, one kernel for all of
                              * them that are admitted in one scheduler pass;
                              * such a job's requests always take that kernel
                              * and start once its previous one completed  */
} soptx_server_opts;

/*
 * One iteration of one design job.  The mesh description (host arrays) is
 * read only when the job's mesh is not resident -- on the job's first request
 * or after an eviction -- so it must stay valid until the request completes.
 * The device buffers are caller-owned and must stay valid until completion:
 *   d_rho [n_cells], d_u [ndof] in; d_vals [nnz], d_dc [n_cells], d_c [1] out
 * (d_vals may be NULL for a sensitivity-only request, d_c may be NULL).
 */
typedef struct {
    uint64_t job;
    int32_t dim;
    soptx_cell cell;
    int32_t order;
    int64_t n_vertices;
    const double *coords;
    int64_t n_cells;
    const int32_t *cell_vertices;
    soptx_material mat;
    soptx_elem_prec prec;
    const double *d_rho;
    const double *d_u;
    double *d_vals;
    double *d_dc;
    double *d_c;
} soptx_request;

typedef struct {
    soptx_status status;     /* SOPTX_OK, or why the request failed           */
    double queue_us;         /* submit -> admitted                            */
    double latency_us;       /* submit -> completion observed                 */
    double gpu_us;           /* device time of the request's kernels          */
    int64_t nnz;             /* CSR nonzeros of the job's mesh                */
    int32_t mesh_was_resident; /* 1 if no mesh setup was needed              */
    /* device timeline of the request, in microseconds from an event the server
     * records at creation: when its stream reached the request's first
     * operation and when its last operation completed (gpu_end_us -
     * gpu_start_us = gpu_us).  Intervals of different requests that intersect
     * were in flight on the device at the same time. */
    double gpu_start_us, gpu_end_us;
} soptx_result;

typedef struct {
    int64_t submitted, completed, failed, evictions, mesh_setups;
    int64_t resident_bytes, peak_resident_bytes;
    int32_t resident_meshes, in_flight, queued;
    int64_t groups;          /* grouped launches of small lattice requests */
} soptx_server_stats;

/* Starts the scheduler thread.  Errors: EINVAL (bad options), ECUDA. */
soptx_status soptx_server_create(const soptx_server_opts *opts, soptx_server *out);

/* Queues a request and returns its ticket.  EBUSY when max_queue requests are
 * pending; EINVAL for a malformed request (the mesh itself is validated at
 * admission and reported through the result). */
soptx_status soptx_serve_submit(soptx_server srv, const soptx_request *req, uint64_t *ticket);

/* Host only (no device work, usable without a GPU): an upper bound of the
 * device bytes soptx_mesh_create allocates for the request's mesh, from its
 * description alone (the device buffers are not read).  The server makes this
 * much room under hbm_cap_bytes (evicting idle meshes) before it builds a
 * job's mesh, then accounts the mesh's actual bytes: a job whose bound exceeds
 * the cap is still built once nothing else is resident, and fails with ENOMEM
 * only if its actual bytes do.  One pass over the cell array (the most cells
 * at a vertex bounds the padding of the pair kernel's tables).  Errors: EINVAL
 * for a NULL argument or a malformed mesh description, ENOMEM. */
soptx_status soptx_serve_mesh_bytes_bound(const soptx_request *req, int64_t *bytes);

/* Waits up to timeout_us (< 0: forever) for the ticket; on success fills *res
 * and forgets the ticket.  ETIMEOUT if it did not complete in time (the ticket
 * stays valid), ENOTFOUND for an unknown or already collected ticket. */
soptx_status soptx_serve_wait(soptx_server srv, uint64_t ticket, int64_t timeout_us, soptx_result *res);

/* *done = 1 when the ticket has completed (its result is then ready). */
soptx_status soptx_serve_poll(soptx_server srv, uint64_t ticket, int32_t *done);

soptx_status soptx_server_stats_get(soptx_server srv, soptx_server_stats *stats);

/* Finishes the requests in flight, fails the queued ones, frees every mesh. */
soptx_status soptx_server_destroy(soptx_server srv);

#ifdef __cplusplus
}
#endif

#endif /* SOPTX_SERVE_H */
