/*
 * px_serve.h -- continuous-batching request loop on top of px.h.
 *
 * A server owns up to max_slots px handles, each with its own CUDA stream and host
 * worker thread.  Requests (a structure plus its frequency sweep, Sec. "Running and
 * Input Configuration": geometry, atom types, field, frequency grid) are queued by
 * px_submit and admitted, in arrival order with small requests allowed to pass a head
 * that does not fit, whenever a slot is free and the request's estimated device
 * footprint fits the server's HBM budget.  Admitted requests run concurrently on
 * their slots' streams, so their kernels overlap on the GPU.  A slot whose previous
 * request had the same structure and options keeps its device-resident operators
 * (CSR of K, T) and skips the structure set-up.
 *
 * Conventions are those of px.h: status codes, caller-owned buffers, inputs copied at
 * the call, complex numbers as interleaved doubles.  The server's functions may be
 * called from any host thread.
 */
#ifndef PX_SERVE_H
#define PX_SERVE_H

#include "px.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct px_server px_server;

/* One request: a structure (as in px_set_structure) and a sweep (as in px_solve).
 * Every array is copied by px_submit. */
typedef struct {
  int model;                  /* px_model */
  int n_atoms;
  const double* xyz_ang;      /* [n_atoms][3] */
  const int* type_idx;        /* [n_atoms] */
  const px_atom_type* types;  /* [n_types] */
  int n_types;
  int n_freq;
  const double* omega_ev;     /* [n_freq] */
  const double* alpha_ib;     /* [n_types][n_freq] complex, PX_WFQFMU only */
  int n_pol;
  const double* pol_dir;      /* [n_pol][3] */
  double e0;
} px_request;

typedef struct {
  long long submitted, completed, failed;
  long long running, queued;
  double p50_latency_ms, p99_latency_ms, max_latency_ms;  /* submit -> result ready */
  double busy_points;         /* spectrum points (converged columns) delivered */
  double wall_s;              /* server lifetime so far */
  long long structure_reuses; /* admissions that kept a slot's resident operators */
  size_t peak_reserved_bytes; /* largest sum of admitted footprint estimates */
  long long merged_requests;  /* requests solved as extra columns of another request's
                                 block (same structure, model, field directions, E0) */
} px_server_stats;

/* Create a server.  opt: solver options for every request (NULL = defaults); with
 * solver = PX_SOLVER_SHIFTED the PX_WFQ requests use the shifted solver (PX_WFQFMU ones
 * stay batched) and an automatic shift_krylov_max becomes 1500, so that admission can
 * count the shifted work space.  max_slots in [1, 32]; hbm_budget_bytes = 0 means 80% of
 * the free device memory.  PX_EINVAL, PX_ECUDA. */
px_status px_server_create(px_server** s, const px_options* opt, int max_slots,
                           size_t hbm_budget_bytes);

/* Queue a request; *req_id receives its id.  PX_EINVAL for a malformed request,
 * PX_ENOMEM if its footprint can never fit the budget, PX_EBUSY if 100000 requests are
 * already waiting. */
px_status px_submit(px_server* s, const px_request* r, uint64_t* req_id);

/* Non-blocking: *done = 1 and results copied to out (see px_result in px.h; the
 * request's n_freq, n_pol and n_atoms size the buffers) when finished, else *done = 0.
 * Returns the request's solve status once done (PX_OK, PX_ENOTCONV, ...), PX_OK while
 * pending, PX_ENOTFOUND for an unknown or already collected id.  A finished request
 * is forgotten after its results were copied. */
px_status px_poll(px_server* s, uint64_t req_id, px_result* out, int* done);

/* Block until the request finishes or timeout_s passes (PX_ETIMEOUT), then as
 * px_poll. */
px_status px_wait(px_server* s, uint64_t req_id, px_result* out, double timeout_s);

px_status px_server_get_stats(px_server* s, px_server_stats* st);

/* Finish every admitted request, drop the queued ones, release all slots. */
px_status px_server_destroy(px_server* s);

#ifdef __cplusplus
}
#endif
#endif /* PX_SERVE_H */
