/*
 * adsgb.h -- C ABI of the GB300 (sm_103a) IGA-ADS + CRVPINN hybrid time step.
 *
 * The library computes, on one GPU, the hybrid CO2-sequestration time step:
 *   - the IGA-ADS explicit saturation update: Gauss-quadrature assembly of the
 *     right-hand side of the L2 projection (Sec. 4, Eqs. 10b-13, i.e. the weak
 *     form Eq. 10a of Eq. 6) followed by the Kronecker-factored mass solve
 *     M = Mx (x) My (x) Mz (Eq. 14) as banded LDL^T line sweeps along x, y, z;
 *   - the CRVPINN pressure update: MLP over the collocation grid (Eq. 21),
 *     the discrete residual (Eqs. 23b-25), the robust loss RES^T G^-1 RES
 *     (Eqs. 26-28), its hand-written gradient and Adam (Sec. 8.3);
 *   - the hybrid loop of Sec. 6 (projection of the network pressure into the
 *     B-spline space, 10 saturation steps, 100 Adam iterations);
 *   - the plain method of Sec. 7: the Galerkin B-spline pressure (Sec. 4,
 *     Eqs. 15-20) solved directly, in place of the network (2D).
 *
 * Conventions (every entry point):
 *   - Every call returns an ads_status; no exception crosses the ABI.
 *   - A context owns all its device memory and enqueues all work on the
 *     stream given at ads_init (NULL = the legacy default stream).  Calls
 *     return after enqueueing, except those that return host data (ads_get,
 *     a non-NULL loss/stat output), which wait for the stream with a deadline
 *     (ADS_ERR_TIMEOUT if it passes).
 *   - Host arrays passed in are copied; the caller keeps ownership.  Device
 *     pointers handed out by ads_device_ptr are borrowed and valid until
 *     ads_destroy.
 *   - A CUDA error makes the context's status sticky (ADS_ERR_CUDA); later
 *     calls on it return that status.  ads_last_error gives the message.
 *   - One context is used by one host thread at a time.
 *   - Array layout: row-major with x fastest: [y][x] in 2D, [z][y][x] in 3D.
 *     B-spline coefficient arrays have (n+2)^dim entries (quadratic, C1);
 *     nodal arrays (n+1)^dim; interior collocation arrays (n-1)^dim.
 *   - Non-dimensional parameters: the viscosity and density ratios of the
 *     paper's Sec. 8.1 table; gravity acts along -vertical (y in 2D, z in 3D).
 */
#ifndef ADSGB_H
#define ADSGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ads_ctx ads_ctx;

typedef enum {
  ADS_OK = 0,
  ADS_ERR_INVALID_ARG = 1,  /* a pointer, size or parameter is out of range */
  ADS_ERR_OOM = 2,          /* device allocation failed                      */
  ADS_ERR_CUDA = 3,         /* a CUDA call failed (sticky)                   */
  ADS_ERR_NONFINITE = 4,    /* a loss, step size or field became non-finite  */
  ADS_ERR_TIMEOUT = 5,      /* waiting for the stream exceeded the deadline  */
  ADS_ERR_STATE = 6,        /* call not valid in this state (e.g. no network)*/
  ADS_ERR_UNSUPPORTED = 7,  /* valid request the library does not implement  */
  ADS_ERR_IO = 8            /* a checkpoint file could not be written or read */
} ads_status;

/* arithmetic types */
typedef enum { ADS_F64 = 0, ADS_F32 = 1, ADS_BF16 = 2 } ads_dtype;

#define ADS_MAX_SOURCES 8
typedef struct {
  double center[3];  /* (x, y, z) in [0,1]^dim                                */
  double sigma;      /* width of the normalised Gaussian                      */
  double rate;       /* Q >= 0                                                */
  int kind;          /* 0: gas injector q_g += Q G; 1: producer, total Q G
                        removed, gas share = fractional flow f_g(S)           */
} ads_source;

typedef struct {
  int dim;           /* 2 (or 3 where supported)                              */
  int n;             /* elements per axis (>= 2); collocation intervals N = n  */
  double phi;        /* porosity when no porosity map is given (> 0)          */
  double mu_w, mu_g, rho_w, rho_g;
  double grav;       /* |g| >= 0                                              */
  double grav_sign;  /* +1: gravity term derived from Eq. 2; -1: as printed in
                        Eq. 9 (saturation equation only)                      */
  double kz_ratio;   /* 3D vertical permeability ratio (1 = isotropic)        */
  int n_src;         /* 0..ADS_MAX_SOURCES                                    */
  ads_source src[ADS_MAX_SOURCES];
  int ads_dtype;     /* ADS_F64 or ADS_F32: saturation-step arithmetic        */
} ads_params;

typedef struct {
  int width;         /* hidden width: 64 or 128 (ADS_F64: 64)                 */
  int hidden_layers; /* 4                                                     */
  int dtype;         /* ADS_F64 or ADS_F32: network, residual, Gram and Adam
                        in that precision on the CUDA cores.  ADS_BF16: the
                        network's layer products on the tcgen05 tensor cores
                        with BF16 operands and FP32 accumulation, stored
                        activations in BF16, everything else (residual, Gram,
                        Adam, master parameters) in FP32.                     */
  int act_chunks;    /* ADS_BF16: stored activations.  1: all points' at once.
                        k > 1: activation recomputation -- the forward of an
                        iteration stores none; the backward runs over k chunks
                        of the 128-point tiles, each preceded by a forward of
                        that chunk that stores its activations, so the buffer
                        holds one chunk.  0: 1 unless all points' activations
                        would take more than a quarter of the free device
                        memory, then the fewest chunks that fit.  Ignored for
                        ADS_F32 / ADS_F64.                                   */
} crvpinn_params;

typedef struct {
  int n_sub;         /* saturation steps per hybrid step (Sec. 6 uses 10)     */
  double dt;         /* fixed step (dt_policy 0) or upper bound (policy 1)    */
  int dt_policy;     /* 0 fixed, 1 CFL: min(cfl*h/v_max, src_frac/s_max, dt)  */
  double cfl;        /* e.g. 0.1                                              */
  double src_frac;   /* e.g. 0.05                                             */
  int adam_iters;    /* Adam iterations per pressure update (100)             */
  double lr;         /* Adam learning rate                                    */
} hybrid_params;

typedef struct {
  double dt_used;    /* step size of the last saturation steps                */
  double loss_last;  /* robust loss at the last Adam iteration                */
  double mass_err;   /* sum over the last saturation steps of
                        int S_{k+1} - int S_k - dt int q_g/phi                */
  double mass_total; /* int S after the step                                  */
} hybrid_stats;

/* fields for ads_get / ads_device_ptr */
typedef enum {
  ADS_FIELD_S = 0,        /* saturation coefficients (n+2)^dim            */
  ADS_FIELD_P = 1,        /* pressure coefficients   (n+2)^dim            */
  ADS_FIELD_K = 2,        /* nodal permeability      (n+1)^dim            */
  ADS_FIELD_ALPHA = 3,    /* nodal alpha = lambda K  (n+1)^dim (Eq. 23b)  */
  ADS_FIELD_F = 4,        /* interior RHS            (n-1)^dim (Eq. 23b)  */
  ADS_FIELD_U = 5,        /* network at interior nodes (n-1)^dim          */
  ADS_FIELD_RES = 6,      /* residual RES            (n-1)^dim (Eq. 25)   */
  ADS_FIELD_Z = 7,        /* G^-1 RES                (n-1)^dim (Eq. 28)   */
  ADS_FIELD_GU = 8,       /* dLOSS/du                (n-1)^dim            */
  ADS_FIELD_THETA = 9,    /* network parameters      nparams              */
  ADS_FIELD_GRAD = 10,    /* dLOSS/dtheta            nparams              */
  ADS_FIELD_LOSS = 11,    /* loss of the last Adam iteration (1 value)    */
  ADS_FIELD_DT = 12,      /* current step size (1 value)                  */
  ADS_FIELD_MASS = 13,    /* [int S, accumulated mass error, source int.] */
  ADS_FIELD_LOSS_LOG = 14 /* ring of the last 4096 losses                 */
} ads_field;

/* ---- lifetime ------------------------------------------------------------
 * ads_init: create a context on the current CUDA device.
 *   K_nodal   (n+1)^dim permeability, > 0, finite (required)
 *   phi_nodal (n+1)^dim porosity > 0 or NULL (constant params->phi)
 *   S0        (n+2)^dim initial saturation coefficients or NULL (zero)
 *   crv       network description, or NULL for a saturation-only context
 *   stream    cudaStream_t to enqueue on (NULL: legacy default stream)
 * Builds the basis tables, the 1D mass matrices and their LDL^T factors
 * (Eq. 14, factored once in FP64), the sine transform and shifted
 * tridiagonal factors of the Gram matrix (Eq. 28, factored once in FP64).
 * Errors: ADS_ERR_INVALID_ARG (bad sizes/values, NULL K or out),
 * ADS_ERR_NONFINITE (non-finite K/phi/S0), ADS_ERR_OOM, ADS_ERR_CUDA. */
ads_status ads_init(const ads_params* params, const crvpinn_params* crv,
                    const double* K_nodal, const double* phi_nodal,
                    const double* S0, void* stream, ads_ctx** out);
/* ads_destroy: waits for the context's stream, frees every device buffer
 * (through the caller's allocator when one was given), the pinned staging
 * buffer, a stream the context created, and the context.  NULL: no-op. */
void ads_destroy(ads_ctx* ctx);

/* ads_init_with_allocator: ads_init whose context buffers come from the
 * caller's allocator (e.g. a serving process's own pool).  alloc(bytes, user)
 * returns device memory of this context's device, 256-byte aligned, or NULL
 * (-> ADS_ERR_OOM); a misaligned block is handed back to free() and
 * ads_init fails with ADS_ERR_INVALID_ARG.  free(ptr, user) is called for
 * every block, by ads_destroy after the context's stream has finished or by
 * a failing ads_init.  The short-lived staging buffers of ads_get and of the
 * host uploads stay stream-ordered cudaMallocAsync blocks.  allocator NULL or
 * with a NULL function: ads_init. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} ads_allocator;
ads_status ads_init_with_allocator(const ads_params* params, const crvpinn_params* crv,
                                   const double* K_nodal, const double* phi_nodal,
                                   const double* S0, void* stream, const ads_allocator* allocator,
                                   ads_ctx** out);

/* ads_hbm_estimate (no counterpart in the paper; admission control): bytes of
 * device memory ads_init would allocate for these parameters (crv NULL: a
 * saturation-only context); 0 when ads_init would refuse them.  Host-only: no
 * CUDA call.  Not counted: the Galerkin-pressure workspace, which
 * ads_galerkin_pressure allocates on first use. */
size_t ads_hbm_estimate(const ads_params* params, const crvpinn_params* crv);

/* ads_set_concurrency: the number of contexts expected to run on the GPU at
 * the same time as this one (default 1).  Above 1, the tensor-core network
 * kernels launch fewer CTAs that each take more 128-point tiles (at least 4
 * per forward CTA and 64 per backward CTA): the context's own iterations take
 * longer, the GPU's total throughput over the concurrent contexts rises.
 * Results agree within rounding (the gradient partials are summed in another
 * grouping).  Drops the context's cached graphs; waits for its stream.
 * Errors: ADS_ERR_INVALID_ARG (contexts < 1). */
ads_status ads_set_concurrency(ads_ctx* ctx, int contexts);

/* ---- saturation (Secs. 2-4) -----------------------------------------------
 * ads_saturation_step: n_sub explicit steps S_{k+1} = M^-1 R(S_k, p) of Eq. 6
 * in the weak form Eq. 10a/10b with the current pressure coefficients and a
 * fixed step dt > 0.  Each step is one fused quadrature + x-sweep kernel and
 * one y-sweep kernel (which also accumulates the mass balance).  dt <= 0
 * uses the step size currently held on the device (e.g. from ads_cfl_dt).
 * Errors: ADS_ERR_INVALID_ARG (n_sub < 0). */
ads_status ads_saturation_step(ads_ctx* ctx, double dt, int n_sub);

/* ads_cfl_dt: device step size min(cfl*h/v_max, src_frac/s_max, dt_cap),
 * v_max = max over Gauss points of |K (grad p + s rho_g g e)|/(mu_g phi),
 * s_max = max q_inj/phi (the paper fixes tau; this is the CFL reading).  The
 * result stays on the device for the next ads_saturation_step(dt <= 0);
 * dt_out (nullable) receives it after a synchronisation. */
ads_status ads_cfl_dt(ads_ctx* ctx, double cfl, double src_frac, double dt_cap,
                      double* dt_out);

/* ---- Galerkin pressure: the plain method (Sec. 7; system of Sec. 4) ---------
 * ads_galerkin_pressure: sets the pressure coefficients to the solution of the
 * B-spline Galerkin pressure system for the current saturation -- the weak
 * form Eq. 12a in the space of Eqs. 15-20:
 *   (lambda K grad p, grad v) = (q_w + q_g, v) - (g K rho lambda, dv/dy)
 * for every interior tensor B-spline v, p = 0 on the boundary (Sec. 8.1),
 * lambda = lambda_w + lambda_g and rho lambda = rho_w lambda_w + rho_g lambda_g
 * of the clamped saturation, K the bilinear nodal map.  This is the pressure
 * the IGA-ADS + direct solver baseline uses instead of the network.  It is
 * assembled by 3-point Gauss quadrature and solved by a banded Cholesky
 * factorisation, all in FP64 whatever ads_dtype is (the result is stored in
 * ads_dtype).  The factorisation and the two triangular sweeps run in one
 * thread block each: n^2 sequential pivots, meant for the baseline's sizes.
 * 2D with n <= 512 only (else ADS_ERR_UNSUPPORTED).  The first call allocates
 * the workspace, n^2 (2n + 32) doubles (2.2 GB at n = 512; 0.8 MB at n = 32),
 * through the context's allocator and keeps it (ADS_ERR_OOM if it cannot);
 * ads_hbm_estimate does not count it.  Work is enqueued on the context's
 * stream; the call returns after enqueueing.  A pivot that is not positive
 * and finite (non-finite or negative inputs) sets every coefficient to NaN and
 * the context's non-finite flag, which hybrid_step then reports. */
ads_status ads_galerkin_pressure(ads_ctx* ctx);

/* ads_set_pressure_coeffs / ads_set_saturation: replace the B-spline
 * coefficients of p or S (the unknowns of Eq. 10a; (n+2)^dim host doubles,
 * copied; the call waits for the stream).  ads_set_saturation also makes the
 * new int S the reference of the mass balance.
 * Errors: ADS_ERR_INVALID_ARG (NULL), ADS_ERR_NONFINITE (a non-finite value). */
ads_status ads_set_pressure_coeffs(ads_ctx* ctx, const double* host_p);
ads_status ads_set_saturation(ads_ctx* ctx, const double* host_s);

/* ---- CRVPINN pressure (Sec. 5) ---------------------------------------------
 * crvpinn_set_theta: load network parameters (nparams host doubles, layout
 * [W_1 (out x in, row-major), b_1, ..., W_5, b_5]) and reset Adam (m=v=0,t=0).
 * crvpinn_num_params: nparams for this context's network.
 * Errors: ADS_ERR_STATE (a context without a network), ADS_ERR_INVALID_ARG
 * (NULL), ADS_ERR_NONFINITE (a non-finite parameter). */
ads_status crvpinn_set_theta(ads_ctx* ctx, const double* theta);
ads_status crvpinn_num_params(const ads_ctx* ctx, int* nparams);

/* crvpinn_update_coefficients: alpha = lambda(S) K and RHS (Eq. 23b) at the
 * collocation nodes from the current saturation coefficients.
 * Errors: ADS_ERR_STATE (no network). */
ads_status crvpinn_update_coefficients(ads_ctx* ctx);

/* crvpinn_loss_grad: one evaluation of the robust loss (Eq. 27) and its
 * gradient dLOSS/dtheta at the current parameters, without an update:
 * MLP forward, residual (Eq. 25), G^-1 RES through the sine transform along x
 * and shifted tridiagonal line solves along y (Eq. 28), loss, adjoint
 * 2 A G^-1 RES, MLP backward.  loss_out (nullable) is filled after a
 * synchronisation; the gradient is kept on the device (ADS_FIELD_GRAD).
 * Errors: ADS_ERR_STATE (no network), ADS_ERR_NONFINITE (non-finite loss). */
ads_status crvpinn_loss_grad(ads_ctx* ctx, double* loss_out);
/* crvpinn_vjp: the network's vector-Jacobian product at the current
 * parameters, g_theta = (du/dtheta)^T g_u, with u the network's values on
 * the interior collocation nodes (Eq. 21, the boundary is 0) in the layout of
 * ADS_FIELD_U.  It chains a gradient with respect to the network pressure
 * (e.g. from ads_degree_project_vjp and ads_degree_step_vjp, the inverse
 * problem of Sec. 9) back to the parameters, through the hand-written forward
 * and backward kernels.  g_u: (N-1)^dim host doubles (copied in; they replace
 * dLOSS/du in ADS_FIELD_GU); g_theta: nparams host doubles (written, in the
 * crvpinn_set_theta layout; ADS_FIELD_GRAD holds them too).  In the network's
 * precision.  Waits for the stream (bounded).
 * Errors: ADS_ERR_INVALID_ARG (NULL pointers), ADS_ERR_STATE (no network),
 * ADS_ERR_UNSUPPORTED (activation recomputation, act_chunks > 1). */
ads_status crvpinn_vjp(ads_ctx* ctx, const double* g_u, double* g_theta);

/* crvpinn_pretrain: coefficients from the current saturation, reset Adam,
 * then `iters` Adam iterations at learning rate lr (Sec. 6 step 2).
 * crvpinn_pressure_update: same without the Adam reset (Sec. 6 step 7; Adam
 * moments persist across updates).  loss_out (nullable): loss of the last
 * iteration, after a synchronisation.
 * Errors: ADS_ERR_STATE (no network), ADS_ERR_INVALID_ARG (iters < 0, lr not
 * positive and finite), ADS_ERR_NONFINITE (non-finite loss). */
ads_status crvpinn_pretrain(ads_ctx* ctx, int iters, double lr, double* loss_out);
ads_status crvpinn_pressure_update(ads_ctx* ctx, int iters, double lr, double* loss_out);

/* ads_project_pressure: network at the interior nodes (boundary 0), L2
 * projection of its piecewise-(bi)linear interpolant into the B-spline space
 * (Sec. 6 step 4) -> pressure coefficients.  Errors: ADS_ERR_STATE (no
 * network). */
ads_status ads_project_pressure(ads_ctx* ctx);

/* ---- hybrid step (Sec. 6) ---------------------------------------------------
 * hybrid_step: project the network pressure; step size (fixed or CFL); n_sub
 * saturation steps; coefficients from the new saturation; adam_iters Adam
 * iterations.  The whole step is replayed from a CUDA graph.  stats (nullable)
 * is filled after a synchronisation; ADS_ERR_NONFINITE if the loss or dt is
 * not finite.
 * Errors: ADS_ERR_INVALID_ARG (hp NULL, n_sub or adam_iters < 0, dt, lr, cfl
 * or src_frac out of range), ADS_ERR_STATE (no network), ADS_ERR_NONFINITE,
 * ADS_ERR_TIMEOUT (a kernel's bounded device wait gave up). */
ads_status hybrid_step(ads_ctx* ctx, const hybrid_params* hp, hybrid_stats* stats);

/* hybrid_step_batch (no counterpart in the paper: it steps one scenario at a
 * time): hybrid_step for n independent contexts, every step enqueued before
 * any statistics are read, so that contexts on different streams overlap on
 * the device.
 * Grouped training: when n >= 2 distinct contexts share the grouped shape
 * (2D; width-64 tensor-core network with FP32 network arithmetic and stored
 * activations; N a power of two, so the Gram solve takes the FFT route, in
 * its three-pass form, i.e. not the one-cluster form that a context alone at
 * N <= 128 takes: ads_set_concurrency > 1), each kernel of an Adam
 * iteration runs once for the whole batch.  It is a grouped launch over
 * per-context argument tables, on a stream of the batch's own, after each
 * context's saturation part (on the context's stream), which then waits for
 * it.  Every context's results are bit-identical to its own hybrid_step's.
 * The batch's tables, stream and graphs are made on the first call with this
 * list of contexts and kept (up to 16 lists; made again when a member's
 * concurrency changes; released when a member is destroyed).  They come from
 * cudaMalloc, not from a context's allocator.  The list of plans is shared
 * by the process and locked while a call enqueues a batch's work, so host
 * threads that step batches of their own contexts may call at once.  Other
 * batches are stepped context by context.  The grouped Adam iterations count in the first
 * context's kernel launches (ads_kernel_launches).
 * stats: NULL or n entries.  Errors: ADS_ERR_INVALID_ARG (ctxs or hp NULL, a
 * NULL context, n < 0), else the first failing context's status (the
 * contexts after it are not stepped, or not read); a failed grouped launch
 * marks every context of the batch ADS_ERR_CUDA. */
ads_status hybrid_step_batch(ads_ctx* const* ctxs, int n, const hybrid_params* hp,
                             hybrid_stats* stats);
/* hybrid_step_batch_profile (diagnostic): for n >= 2 contexts of the grouped
 * shape (see hybrid_step_batch), one grouped Adam iteration with event records
 * between its 8 kernels is captured into a graph and replayed `iters` times on
 * the batch's stream (each replay waited for, bounded), after the contexts'
 * streams have been waited for.  The iterations train the networks as
 * hybrid_step_batch's do.  ms_out[8] receives the average durations of: the
 * weight images, the forward, the Gram rows pass with the residual, the Gram
 * columns pass, the Gram rows pass with the loss partials, the adjoint with
 * the loss, the backward, the gradient sum with Adam.
 * Errors: ADS_ERR_INVALID_ARG (ctxs or ms_out NULL, a NULL context, n < 2,
 * iters < 1), ADS_ERR_UNSUPPORTED (not of the grouped shape), ADS_ERR_TIMEOUT,
 * ADS_ERR_CUDA (then set on every context of the batch). */
ads_status hybrid_step_batch_profile(ads_ctx* const* ctxs, int n, int iters, double* ms_out);

/* ---- serving: continuous batching of many scenarios (the paper steps one
 * scenario at a time) ----------------------------------------------------------
 * A server owns a worker thread and n_streams CUDA streams on the current
 * device.  ads_server_submit copies a scenario (parameters, network, hybrid
 * step parameters, number of hybrid steps, pretraining at admission, and its
 * host arrays) into the arrival queue and returns at once.  Between rounds the
 * worker admits the oldest waiting scenarios while the sum of their
 * ads_hbm_estimate stays within hbm_budget and at most max_active are
 * resident; each round enqueues one hybrid step of every resident scenario
 * (streams round-robin, so their kernels overlap) and records each step's
 * latency from enqueue to completion.  A scenario that has run n_steps copies
 * its saturation and pressure coefficients out and frees its memory, which
 * admits the next arrivals.  Results depend only on the scenario's inputs:
 * alone or in any mix they are identical.
 * ads_server_wait blocks until request `id` finished (or timeout_s passed:
 * ADS_ERR_TIMEOUT), copies S and P ((n+2)^dim doubles each, nullable) and its
 * statistics, and forgets the request.  A scenario whose estimate exceeds the
 * whole budget is refused at submission (ADS_ERR_OOM).
 * ads_server_destroy stops the worker, releases resident scenarios and drops
 * waiting ones.
 * Errors: create: ADS_ERR_INVALID_ARG (NULL, hbm_budget 0, n_streams outside
 * 1..64 or max_active < 1), ADS_ERR_CUDA.  submit: ADS_ERR_INVALID_ARG (NULL
 * spec, K or id_out, n_steps < 0, parameters ads_init would refuse),
 * ADS_ERR_OOM (more than the whole budget).  wait: ADS_ERR_INVALID_ARG
 * (unknown id), ADS_ERR_TIMEOUT, else the request's own status.  stats:
 * ADS_ERR_INVALID_ARG (NULL). */
typedef struct ads_server ads_server;
typedef struct {
  size_t hbm_budget;   /* bytes of device memory for resident scenarios      */
  int max_active;      /* cap on resident scenarios                           */
  int n_streams;       /* CUDA streams the resident scenarios share (1..64)   */
} ads_server_config;
typedef struct {
  ads_params params;
  crvpinn_params crv;
  hybrid_params hp;
  int n_steps;         /* hybrid steps to run                                 */
  int pretrain_iters;  /* Adam iterations at admission (0: none)              */
  double pretrain_lr;
} ads_request_spec;
typedef struct {
  int status;          /* ads_status of the request                           */
  int steps;
  double queue_ms;     /* submission to admission                             */
  double total_ms;     /* submission to completion                            */
  double p50_step_ms, p99_step_ms;
  hybrid_stats last;
} ads_request_result;
typedef struct {
  int64_t completed, rejected, steps, pending, active;
  int peak_active;
  size_t bytes_in_use, peak_bytes;
  double p50_step_ms, p99_step_ms;  /* over all completed scenarios' steps     */
} ads_server_stats_t;
ads_status ads_server_create(const ads_server_config* cfg, ads_server** out);
ads_status ads_server_submit(ads_server* s, const ads_request_spec* spec, const double* K_nodal,
                             const double* phi_nodal, const double* S0, const double* theta0,
                             int64_t* id_out);
ads_status ads_server_wait(ads_server* s, int64_t id, double timeout_s, double* S_out,
                           double* P_out, ads_request_result* result);
ads_status ads_server_stats(ads_server* s, ads_server_stats_t* out);
void ads_server_destroy(ads_server* s);

/* ---- data access -------------------------------------------------------------
 * ads_get: copy a field to host doubles (count = number of values expected
 * for the field; ADS_ERR_INVALID_ARG if it differs).  Waits for the stream;
 * ADS_ERR_TIMEOUT also when a kernel's bounded wait on its own bulk copies or
 * tensor-core work has given up on this context (the flag is sticky; the
 * field may be incomplete).
 * ads_device_ptr: borrowed device pointer, its element count and dtype. */
ads_status ads_get(ads_ctx* ctx, int field, double* host_dst, size_t count);
ads_status ads_field_count(const ads_ctx* ctx, int field, size_t* count);
ads_status ads_device_ptr(ads_ctx* ctx, int field, void** dptr, size_t* count, int* dtype);
ads_status ads_sync(ads_ctx* ctx, double timeout_s);

/* ---- checkpoint / resume -----------------------------------------------------
 * ads_save: wait for the stream, then write the context's evolving state to
 * `path` (created or truncated): the current saturation, the pressure
 * coefficients, K and phi, the step size and mass statistics, and with a
 * network the coefficients alpha and f, the network values, theta, the Adam
 * moments, step counter and bias-correction state, the learning rate and the
 * loss log.  Tables and scratch that follow from the parameters are not
 * written.  Binary, host byte order: an 8-byte magic, a version, the shape
 * fields below, then (id, byte count, bytes) sections.
 * ads_load: read such a file into a context made by ads_init with the same
 * dim, n, saturation precision, phi map presence and network (width, layers,
 * precision, parameter count); the next calls continue bit for bit as the
 * saved context would have with the same launch settings (ads_set_concurrency
 * and act_chunks are settings of the context, not part of the checkpoint).
 * Drops cached graphs.
 * Errors: ADS_ERR_INVALID_ARG (NULL path; a file of another shape or not a
 * checkpoint), ADS_ERR_IO (open, write or short read), ADS_ERR_CUDA. */
ads_status ads_save(ads_ctx* ctx, const char* path);
ads_status ads_load(ads_ctx* ctx, const char* path);

/* ---- saturation step without allocation (no counterpart in the paper) -------
 * For callers that cannot call cudaMalloc -- e.g. a serving process whose own
 * allocator owns the whole device memory budget, or a latency-critical loop
 * that must not risk the device synchronisation cudaMalloc/cudaFree can imply.
 * One explicit saturation step S_out = M^-1 R(S, p) (the same kernels as
 * ads_saturation_step), with no context and no allocation: the caller passes
 * device pointers to its inputs and output (FP64, layouts as above:
 * d_K (n+1)^2, d_phi (n+1)^2 or NULL for params->phi, d_S, d_P and d_S_out
 * (n+2)^2; d_S_out must not be d_S) and a step size dt > 0.  All working
 * memory lives in one fixed 4 MiB device array inside the library, reserved on
 * every GPU that loads the library until the process exits; meshes up to
 * n = 512 fit, larger n returns ADS_ERR_INVALID_ARG.  2D, ads_dtype = ADS_F64
 * only (else ADS_ERR_UNSUPPORTED).  The parameters pass the same check as
 * ads_init (same statuses), before any CUDA call.  The first call on a device looks up that
 * array's device address (set-up), so make the first call before any stream
 * capture.  Every call shares the one array: calls that may overlap on the
 * GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  Nothing in the array needs to start at zero;
 * each call rewrites what it reads.  Work is enqueued on `stream` (cudaStream_t,
 * NULL = legacy default stream); the call returns after enqueueing. */
ads_status ads_saturation_step_noalloc(const ads_params* params, const double* d_K,
                                       const double* d_phi, const double* d_S,
                                       const double* d_P, double dt, double* d_S_out,
                                       void* stream);
/* The step above reports problems in a status word inside the same array,
 * since it returns before its kernels run.  The word is sticky: every step
 * ORs into it and none clears it.  ads_saturation_step_noalloc_status waits
 * for `stream` (10 s deadline -> ADS_ERR_TIMEOUT), reads the word into
 * *flags_out (nullable) and clears it.  It returns ADS_ERR_TIMEOUT when a
 * bounded device wait of a step gave up (bit 8: that step's d_S_out is
 * incomplete), ADS_ERR_NONFINITE when a step's int S_out was not finite
 * (bit 0), else ADS_OK.  Call it on the stream of the steps it should cover.
 * The array's device address is looked up once per device and kept, so
 * neither call may be used after cudaDeviceReset in the same process. */
ads_status ads_saturation_step_noalloc_status(void* stream, int* flags_out);

/* ---- saturation step for B-splines of degree 2, 3 or 4 ---------------------
 * Sec. 4 writes the basis for a general order r with continuity C^{r-1}
 * (Eq. 11); Sec. 8 runs r = 2, which is what the context path implements.
 * These calls take the explicit step of Eqs. 10b-13 with the Kronecker mass
 * solve of Eq. 14 for degree p in {2, 3, 4} on an open uniform knot vector,
 * 2D, FP64 (same readings as ads_saturation_step: clamped mobility, phi inside
 * the integrand, nodal K and phi interpolated bilinearly, normalised Gaussian
 * sources with the producer's gas share f_g(S), no-flux boundary).  Written for
 * any p and for correctness first: (p+1)^2 Gauss points per element, one
 * thread per element, per degree of freedom and per line; not the quadratic
 * path's tuned kernels.
 *   ads_degree_plan_create: builds the tables for params (the same check as
 *     ads_init; dim 2 and ads_dtype ADS_F64 only, else ADS_ERR_UNSUPPORTED;
 *     degree outside 2..4 or n > 4096: ADS_ERR_INVALID_ARG) and allocates
 *     the device memory of the plan (about n^2 (p+1)^2 doubles), which the
 *     plan owns; *plan = NULL on failure.  Synchronous.
 *   ads_degree_coeffs: coefficients per axis, n + p (0 for NULL).
 *   ads_degree_step: S_out = M^-1 R(S, P) with the step size dt (> 0,
 *     finite).  Device pointers, row-major with x fastest: d_K and d_phi
 *     (NULL: params->phi) (n+1)^2 nodal values; d_S, d_P, d_S_out (n+p)^2
 *     coefficients; d_S_out must differ from d_S and d_P.  Enqueued on
 *     `stream` (cudaStream_t; NULL = legacy default stream), returns after
 *     enqueueing.  One plan's calls must not overlap on the GPU (they share
 *     its working memory).
 *   ads_degree_mass: int S over the unit square for the (n+p)^2 coefficients
 *     d_S; waits (bounded: ADS_ERR_TIMEOUT after 10 s) for `stream` and
 *     writes *mass.
 *   ads_degree_plan_destroy: frees the plan (NULL: no-op); call it after the
 *     plan's work has completed. */
typedef struct ads_degree_plan ads_degree_plan;
ads_status ads_degree_plan_create(const ads_params* params, int degree, ads_degree_plan** plan);
int ads_degree_coeffs(const ads_degree_plan* plan);
ads_status ads_degree_step(ads_degree_plan* plan, const double* d_K, const double* d_phi, const double* d_S,
                           const double* d_P, double dt, double* d_S_out, void* stream);
ads_status ads_degree_mass(ads_degree_plan* plan, const double* d_S, double* mass, void* stream);
/* ads_degree_project: the L2 projection (Sec. 6, step 4) of nodal values
 *   d_nodal ((n+1)^2, device; their bilinear interpolant) into the degree-p
 *   splines: d_out ((n+p)^2, device) = M^-1 F with F = int I_h u v.
 *   Enqueued on `stream`.
 * ads_degree_cfl_dt: the step size min(dt_cap, cfl h / v_max, src_frac / s_max)
 *   with v_max = max |K (grad p + s rho_g g e_y)| / (mu_g phi) and
 *   s_max = max q_inj / phi over the Gauss points, for pressure coefficients
 *   d_P ((n+p)^2) and the nodal d_K, d_phi (NULL: params->phi); a term is left
 *   out when its maximum is 0.  cfl, src_frac > 0, finite; dt_cap > 0 (may be
 *   +inf).  Waits (bounded: ADS_ERR_TIMEOUT) for `stream` and writes *dt;
 *   ADS_ERR_NONFINITE for a non-finite maximum. */
ads_status ads_degree_project(ads_degree_plan* plan, const double* d_nodal, double* d_out, void* stream);
/* ads_degree_project_vjp: the adjoint of ads_degree_project.  For
 * J = g . P with P the projection of the nodal values, d_gnodal ((n+1)^2,
 * device) = dJ/d(nodal) = A^T M^-1 g, A the assembly of int I_h u v; d_g
 * ((n+p)^2, device), distinct from d_gnodal.  Enqueued on `stream`. */
ads_status ads_degree_project_vjp(ads_degree_plan* plan, const double* d_g, double* d_gnodal, void* stream);
ads_status ads_degree_cfl_dt(ads_degree_plan* plan, const double* d_K, const double* d_phi, const double* d_P,
                             double cfl, double src_frac, double dt_cap, double* dt, void* stream);
/* Vector-Jacobian product of ads_degree_step (a building block of gradients
 * through the explicit steps, e.g. for placing wells: Sec. 9 names the inverse
 * problem as future work).  For J = lambda . S_out with S_out the step of the
 * same arguments (d_K, d_phi, d_S, d_P, dt), it writes
 *   d_gS = dJ/dS and d_gP = dJ/dP ((n+p)^2 each, device), and, when h_gsrc is
 *   not NULL, h_gsrc[3k + 0, 1, 2] = dJ/d(rate, centre x, centre y) of
 *   source k (host, 3 n_src doubles; the call then waits, bounded, for
 *   `stream`).
 * d_lambda: (n+p)^2 (device).  Through mu = M^-1 lambda (M symmetric):
 * J = mu . R(S, P, sources), differentiated at the Gauss points; the clamp
 * of the mobility is differentiated inside (0, 1) and flat outside, so
 * gradients are exact away from S = 0 and S = 1 at the Gauss points.
 * d_gS and d_gP must differ from each other and from the inputs.
 * ADS_ERR_INVALID_ARG for NULL pointers, aliasing or dt not > 0. */
ads_status ads_degree_step_vjp(ads_degree_plan* plan, const double* d_K, const double* d_phi, const double* d_S,
                               const double* d_P, double dt, const double* d_lambda, double* d_gS, double* d_gP,
                               double* h_gsrc, void* stream);
void ads_degree_plan_destroy(ads_degree_plan* plan);

/* ---- maps given as images (Sec. 8.1) -----------------------------------------
 * Sec. 8.1 gives each reservoir's porosity (0 to 1) and permeability (mDarcy,
 * used in SI units) as a picture of the domain.  The method takes K and phi as
 * nodal values on the (n+1)^d vertex grid (K_nodal / phi_nodal of ads_init,
 * d_K / d_phi of ads_degree_step); ads_map_from_image brings a picture there.
 *   d_img: device pixels, ADS_PIXEL_F32 (float, 4-byte aligned) or
 *     ADS_PIXEL_U8 (unsigned char); img_shape[0..dim-1] = {W, H(, D)}: W
 *     columns along x, H rows along y, D slices along z; layout
 *     [slice][row][column], columns fastest.  Row 0 is the picture's top edge
 *     (y = 1) when flip_y != 0, its bottom edge (y = 0) otherwise; slice 0
 *     lies at z = 0.  The caller keeps ownership.
 *   A pixel holds offset + scale * pixel over its square (cube) of the unit
 *     domain.  The nodal value is that field's average over the node's dual
 *     cell, [x_i - h/2, x_i + h/2] per axis clipped to [0, 1]: the arithmetic
 *     mean (ADS_MAP_ARITHMETIC; keeps the map's integral) or the geometric
 *     mean exp(avg log) (ADS_MAP_GEOMETRIC; the usual upscaling of a
 *     log-normal permeability; a zero pixel gives 0 to the cells that see it).
 *     Overlaps are exact (integers in units of 1/(2 n W)) and the sums FP64,
 *     so a picture finer or coarser than the mesh, in any ratio, is accepted.
 *   n[0..dim-1]: elements per axis, 1 to 65536; at most 2^31 - 1 nodes.
 *   d_nodal: device, prod(n_a + 1) doubles, [z][y][x] with x fastest,
 *     8-byte aligned, not overlapping d_img.
 * Enqueued on `stream`; the call then waits (bounded: ADS_ERR_TIMEOUT after
 * 10 s) and returns ADS_ERR_NONFINITE if a nodal value is not finite (a NaN or
 * infinite pixel, or a negative one under the geometric mean; every value is
 * written all the same).  ADS_ERR_INVALID_ARG: a NULL pointer, dim not 2 or 3,
 * an extent or count out of range, an unknown pixel type or mean, a
 * non-finite scale or offset, misalignment or overlapping buffers.
 * ADS_ERR_OOM / ADS_ERR_CUDA: the 4-byte counter could not be allocated / a
 * CUDA call failed. */
typedef enum { ADS_PIXEL_F32 = 0, ADS_PIXEL_U8 = 1 } ads_pixel_type;
typedef enum { ADS_MAP_ARITHMETIC = 0, ADS_MAP_GEOMETRIC = 1 } ads_map_mean;
ads_status ads_map_from_image(const void* d_img, int pixel_type, int dim, const int* img_shape, int flip_y,
                              const int* n, int mean, double scale, double offset, double* d_nodal,
                              void* stream);

/* ---- diagnostics (no counterpart in the paper) ------------------------------
 * ads_kernel_launches: number of library kernels enqueued on this context so
 * far (a graph replay counts the kernels it contains).
 * ads_profile_train: one Adam iteration with CUDA event records between its
 * kernels is captured into a graph, which is launched `iters` times on the
 * context's stream (the kernels run back to back, as in the hybrid step's
 * graphs); ms_out[8] receives the
 * average duration of: network forward, residual, sine transform, tridiagonal
 * sweeps, inverse transform (+ loss partials), adjoint stencil (+ loss
 * finalise), network backward, gradient sum + Adam.  Updates the parameters like
 * crvpinn_pressure_update at the learning rate last set.
 * ads_profile_saturation: one saturation step (current dt) captured likewise
 * and launched `steps` times (each launch repeats the same step from the same
 * state; afterwards the state is one step on); ms_out[3]: quadrature + x
 * sweep, y sweep, mass bookkeeping. */
ads_status ads_kernel_launches(const ads_ctx* ctx, unsigned long long* count);
/* ads_probe_wait_expiry: runs, on the context's stream, one kernel that waits
 * on an mbarrier the way every kernel here does -- bounded, with tensor
 * memory held and a bulk copy of its own in flight -- but that nobody
 * completes (arrive = 0) or that a second thread completes (arrive != 0).
 * After `limit_s` seconds (0 < limit_s <= 10) without completion the kernel
 * records bit 8 (the same bit the real kernels set on a timed-out wait), lets
 * its copy land, frees its tensor memory and returns.  Waits for the stream;
 * *bits_out (nullable) receives the probe's status word.  The context's own
 * status word is not touched, so the context carries on.  Returns
 * ADS_ERR_TIMEOUT when the wait expired, else ADS_OK.  No counterpart in the
 * paper.  Errors: ADS_ERR_INVALID_ARG (NULL context, limit out of range). */
ads_status ads_probe_wait_expiry(ads_ctx* ctx, double limit_s, int arrive, int* bits_out);
/* ads_measure_unit_rates: measured peak rates of the arithmetic units the
 * rooflines use, on the current device (no counterpart in the paper).  One
 * wave of CTAs runs 8 independent chains per thread of one operation;
 * out[0..4] = results per second of ex2.approx.f32, rcp.approx.f32, the
 * tanh pair (one ex2 + one rcp, counted as one result), scalar FP32 fma and
 * packed fma.rn.f32x2 (two results per instruction); out[5..9] = the same per
 * SM per clock; out[10] = the SM clock (MHz) the chains ran at.  nout >= 11.
 * Allocates a few MB of device memory for the run and frees it; synchronous.
 * Errors: ADS_ERR_INVALID_ARG (NULL or nout < 11), ADS_ERR_CUDA. */
ads_status ads_measure_unit_rates(double* out, int nout);
ads_status ads_profile_train(ads_ctx* ctx, int iters, double* ms_out);
ads_status ads_profile_saturation(ads_ctx* ctx, int steps, double* ms_out);

/* ads_last_error: the message of the context's last failure ("" if none;
 * "null context" for NULL), owned by the context and valid until its next
 * call or ads_destroy.  ads_status_str: a static name for a status ("unknown"
 * for other values).  Neither touches the GPU. */
const char* ads_last_error(const ads_ctx* ctx);
const char* ads_status_str(ads_status st);

#ifdef __cplusplus
}
#endif
#endif /* ADSGB_H */
