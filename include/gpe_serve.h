/*
 * gpe_serve.h - batches of independent GPE instances and a request server
 * (C ABI), built on the plans of gpe.h.
 *
 * The paper runs one simulation at a time; these entry points advance many
 * independent solves of the same method (TSSP steps, Numerical Scheme; ground
 * states by imaginary time) together.  Instances that share grid, box, time
 * step, precision and trapped axes advance in one kernel launch per pass;
 * other groups run concurrently on their own streams.  Running N steps in
 * chunks is exact: each chunk is a complete gpe_step_real sequence.
 */
#ifndef GPE_SERVE_H
#define GPE_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "gpe.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- batches */
typedef struct gpe_batch gpe_batch;

/* count instance descriptions (each with batch == 1 and no per-instance
 * arrays; V_host is rejected with GPE_EUNSUPPORTED, here and by
 * gpe_serve_submit).  Instances are grouped; each group owns one plan, whose tile
 * shapes are chosen by gpe_plan_autotune on the group's grid (per-thread
 * staging; two scratch arrays of the group's size while the call runs).  The
 * batch enqueues on cuda_stream (NULL: legacy default stream). */
gpe_status gpe_batch_create(const gpe_plan_desc *descs, int count, void *cuda_stream, gpe_batch **out);
gpe_status gpe_batch_destroy(gpe_batch *batch);

/* Advance every instance by nsteps real-time steps in place.  psi_dev is a
 * HOST array of count device pointers (instance i's state, layout of gpe.h,
 * 16-byte aligned).  use_graph != 0 captures the launch sequence of this nsteps
 * value once into a CUDA graph and replays it on later calls. */
gpe_status gpe_batch_step_real(gpe_batch *batch, void *const *psi_dev, int64_t nsteps, int use_graph);

/* out_host[6*i + k]: the six values of gpe_norm_energy for instance i.
 * Synchronises the batch stream. */
gpe_status gpe_batch_norm_energy(gpe_batch *batch, void *const *psi_dev, double *out_host);

/* number of groups (plans) the batch formed, or -1 */
int gpe_batch_groups(const gpe_batch *batch);

/* ---------------------------------------------------------------- server */
typedef struct gpe_server gpe_server;

typedef struct gpe_request {
    gpe_plan_desc desc;     /* one instance: batch == 1, no per-instance arrays      */
    int imag;               /* 0: nsteps real-time steps; 1: imaginary time          */
    int64_t nsteps;         /* real: steps; imaginary: maximum steps                 */
    double etol;            /* imaginary: stop once |E - E_previous_check| < etol    */
    int check_every;        /* imaginary: steps between energy checks (>= 1)         */
    double target_norm;     /* imaginary: renormalisation target (> 0)              */
    const void *psi0_host;  /* initial state on the host; copied by gpe_serve_submit */
} gpe_request;

typedef struct gpe_result {
    gpe_status status;      /* GPE_OK, or why the request failed (GPE_EBUSY: larger than the budget) */
    int64_t steps_done;
    double norm, energy;    /* of the final state                                    */
    double t_submit, t_admit, t_done;   /* seconds on the server's clock             */
} gpe_result;

/* A server with one worker thread on the current device.  Requests are
 * admitted in arrival order while at most max_active are resident and their
 * device memory (states plus group plans, estimated) fits in
 * hbm_budget_bytes; resident requests of the same group advance together in
 * chunks of at most chunk_steps steps (0: 64), and requests that finish leave
 * between chunks so that queued ones can enter.  max_active <= 0 derives it
 * from the budget: budget / 64 MiB, clamped to 16..256 (it also sizes every
 * group plan: one parameter slot per resident request).
 * Each scheduling round enqueues every group's work on its own stream before
 * waiting for any: request states come from a server-owned stream-ordered
 * memory pool (no device-wide synchronisation on admission or release), and
 * imaginary-time sets copy their energies into pinned buffers that are read
 * after the round's streams have been waited for. */
gpe_status gpe_server_create(size_t hbm_budget_bytes, int max_active, int chunk_steps, gpe_server **out);
gpe_status gpe_server_destroy(gpe_server *server);

/* Queue a request (its initial state is copied); *ticket identifies it. */
gpe_status gpe_serve_submit(gpe_server *server, const gpe_request *req, uint64_t *ticket);

/* Wait up to timeout_ms (negative: forever, 0: no wait) for a request.
 * GPE_ENOTREADY if it has not finished; otherwise fills *res, copies the final
 * state to psi_out_host (may be NULL) and forgets the ticket. */
gpe_status gpe_serve_poll(gpe_server *server, uint64_t ticket, int timeout_ms, gpe_result *res, void *psi_out_host);

/* queued and resident requests and the device bytes accounted to the budget */
gpe_status gpe_server_stats(gpe_server *server, int *queued, int *active, size_t *hbm_used);

#ifdef __cplusplus
}
#endif

#endif /* GPE_SERVE_H */
