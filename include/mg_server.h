/* Serving engine for the adaptive multigrid solver: solve requests on several
 * gauge configurations, continuous batching, resident set-ups under an HBM
 * budget.
 *
 * The paper has no counterpart; it motivates the design: a set-up made at the
 * lightest mass is reused for the other masses (Sec. 4), and its cost is
 * amortised over many right-hand sides.  The server keeps each
 * configuration's hierarchy (null vectors, P, the Galerkin operators, the
 * coarsest inverse) resident on the device while it fits in the budget and
 * solves the requests of one configuration and mass together.
 *
 * Hierarchies.  Each (configuration, mass) pair that has requests is served
 * by its own resident hierarchy with its own CUDA stream: the first one of a
 * configuration by mg_setup at its set-up mass (then mg_set_mass), the others
 * by mg_clone of a resident one (the set-up's vectors are shared by every
 * mass, Sec. 4), so that requests at different masses neither re-mass nor
 * wait for each other.
 *
 * Scheduling.  A pool of host worker threads.  A worker takes the (configuration,
 * mass) group whose oldest pending request is the oldest overall among those
 * whose hierarchy no other worker holds, and packs that request and every
 * other pending request of the group with the same solver and tolerance (up
 * to max_rhs right-hand sides) into one batched mg_solve.  Requests that
 * arrive while a batch is on the GPU join the next batch of their group
 * (continuous batching); batches of different groups run concurrently.
 *
 * Admission.  A new hierarchy is made only if its memory (mg_setup_bytes peak
 * for a set-up, resident bytes for a clone, plus the batch buffers) fits the
 * budget together with the resident ones, after destroying idle hierarchies
 * (not held, no pending request at their mass), least recently used first.
 * Otherwise an idle hierarchy of the same configuration is re-massed
 * (mg_set_mass), or the group waits while the workers serve others (a waiting
 * worker holds nothing, so the pool cannot deadlock).  A configuration whose
 * set-up is larger than the whole budget fails its requests with
 * MG_ERR_NOMEM.
 *
 * Results.  A request's solution is the same as a solve of it alone with
 * the same solver, within the solver's tolerance (batched right-hand sides
 * share the Krylov loop, not their arithmetic: each has its own scalars and
 * stopping test).
 *
 * Threads: all calls are thread-safe.  Device memory passed to submit must
 * stay valid until wait returns for that request.
 */
#ifndef MG_SERVER_H
#define MG_SERVER_H

#include "mg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_server mg_server;

typedef struct {
  long long submitted, completed, failed;
  long long batches, batched_rhs;    /* batched_rhs / batches = mean batch size   */
  long long builds, clones, evictions, remasses;
  long long resident_bytes, peak_resident_bytes, budget_bytes;
  double p50_ms, p99_ms, max_ms;     /* submit-to-completion latency, completed   */
} mg_server_stats;

/* budget_bytes: device memory for resident hierarchies and their batch
 * buffers (> 0).  max_rhs: right-hand sides per batch (1..64); requests may
 * have at most this many.  workers: host threads (1..16).  The CUDA device
 * current at creation is used by every worker. */
mg_status mg_server_create(long long budget_bytes, int max_rhs, int workers, mg_server** out);

/* Registers a gauge configuration: gauge is a device complex128 [2][Lt][Lx]
 * array and params->setup_noise a device buffer of mg_setup_noise_len
 * complex128; both are copied (the caller may free them on return).
 * params->max_rhs is replaced by the server's max_rhs.  setup_mass: the mass
 * of the set-up (Sec. 4: the lightest mass of interest).  No device work
 * beyond the copies; *config_id receives the id (0, 1, ...). */
mg_status mg_server_add_config(mg_server* s, const void* gauge, const mg_params* params,
                               double setup_mass, int* config_id);

/* Queues a solve of A(mass) x = b for nrhs right-hand sides (device
 * complex128 [nrhs][Lt][Lx][2], b read and x written by a worker on the
 * server's own stream; 1 <= nrhs <= max_rhs), tolerance tol on the true FP64
 * relative residual, solver MG_SOLVER_*.  b must hold its final values when
 * submit is called (its producer synchronised).  Returns at once with
 * *request_id. */
mg_status mg_server_submit(mg_server* s, int config_id, double mass, const void* b, void* x,
                           int nrhs, double tol, int solver, long long* request_id);

/* Waits for a request; info receives nrhs records (may be NULL), latency_ms
 * the time from submit to completion (may be NULL).  Returns the request's
 * status (the solve's, or MG_ERR_NOMEM when its configuration cannot fit the
 * budget).  Each request is waited for once. */
mg_status mg_server_wait(mg_server* s, long long request_id, mg_solve_info* info,
                         double* latency_ms);

mg_status mg_server_get_stats(mg_server* s, mg_server_stats* out);

/* Failure injection on the host, for tests of the failure path: the next
 * `count` hierarchy builds or clones report MG_ERR_CUDA (after 50 ms, without
 * touching the device) instead of running.  A failed build or clone fails
 * the queued requests of its own (configuration, mass) group only; requests
 * at other masses, and builds of other groups in flight meanwhile, go on. */
mg_status mg_server_inject_build_failures(mg_server* s, int count);

/* Waits for every queued request, then frees everything.  NULL is allowed. */
void mg_server_destroy(mg_server* s);

#ifdef __cplusplus
}
#endif

#endif /* MG_SERVER_H */
