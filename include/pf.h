/*
 * pf.h -- C ABI of libpf, a GB300 (sm_103a) solver for the staggered phase-field model
 * of brittle fracture with the fixed-stress schemes of Luo, "Fast staggered schemes for
 * the phase-field model of brittle fracture based on the fixed-stress concept"
 * (arXiv 2209.07969).
 *
 * The model (Sec. 2): energy split into an active part
 *     Psi+ = mu eps_dev:eps_dev + K/2 <tr eps>_+^2
 * and an inactive part K/2 <tr eps>_-^2, degraded stress
 *     sigma = g(d) [2 mu eps_dev + K <tr eps>_+ I] + K <tr eps>_- I,
 * AT2 functions g(d) = (1-d)^2 + eta, w(d) = d^2, c_w = 2 (Table 1), and the history
 * field H = max over time of Psi+ driving the evolution equation
 *     [G_c/l + 2H] d - G_c l lap d = 2H.
 * Discretisation: bilinear (Q1) elements on a structured nx-by-ny grid, 2x2 Gauss.
 * Staggered schemes (Sec. 3.1, Fig. 1; Sec. 3.3-3.5, Table 2): standard (ST, d-u
 * order) and fixed-stress S1 (first stress invariant held), S2 (deviatoric relation),
 * S3 (both).
 *
 * Layouts (all arrays dense, C order):
 *   node (i, j), 0 <= i <= nx, 0 <= j <= ny : id j*(nx+1) + i, at (i*Lx/nx, j*Ly/ny)
 *   element (i, j), 0 <= i < nx, 0 <= j < ny: id j*nx + i, nodes (i,j),(i+1,j),(i,j+1),(i+1,j+1)
 *   u   : 2*N doubles, interleaved (u_x, u_y) per node, N = (nx+1)*(ny+1)
 *   d   : N doubles
 *   H   : 4*nx*ny doubles, element-major, Gauss points (-,-),(+,-),(-,+),(+,+)
 *
 * Errors: every call returns a pf_status; PF_OK is 0.  Calls on a context set a
 * message readable with pf_last_error.  Nothing in the library aborts the process.
 * Thread safety: one context must not be used from two host threads at once.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PF_API_VERSION 1

typedef enum {
  PF_OK = 0,
  PF_EINVAL = 1,     /* bad argument (sizes, flags, NULL pointer, material out of range) */
  PF_ENOMEM = 2,     /* device or host allocation failed */
  PF_ENOTCONV = 3,   /* a solver hit its iteration cap; state is kept, see pf_step_result */
  PF_ECUDA = 4,      /* a CUDA runtime call failed (message has the CUDA error string) */
  PF_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
  PF_EBUSY = 6       /* resource in use (e.g. server slots full) */
} pf_status;

/* Staggered schemes of Table 2. */
typedef enum { PF_ST = 0, PF_S1 = 1, PF_S2 = 2, PF_S3 = 3 } pf_scheme;

/* Node flag bits (one byte per node). */
enum {
  PF_FIX_X = 1,   /* u_x held at 0 */
  PF_FIX_Y = 2,   /* u_y held at 0 */
  PF_LOAD_X = 4,  /* u_x held at the prescribed displacement ubar */
  PF_LOAD_Y = 8,  /* u_y held at ubar */
  PF_D_FIX1 = 16, /* d held at 1 (initial slit) */
  PF_D_FIX0 = 32  /* d held at 0 (protected region) */
};
/* A node with no active element has all its DOFs held at 0. */

enum { PF_PLANE_STRAIN = 0, PF_PLANE_STRESS = 1 };
enum { PF_FP64 = 0, PF_FP32_IR = 1 };          /* linear-solve precision */
enum { PF_PRECOND_JACOBI = 0, PF_PRECOND_GMG = 1 };
enum { PF_F64 = 0, PF_F32 = 1 };                /* element type of operator-level arrays */
/* Energy split (Sec. 2).  VD: Psi+ = mu e.e + K/2 <tr>_+^2, the split the paper runs.
 * SPECTRAL: the alternative split Sec. 2 names, Psi+ = lam/2 <tr>_+^2 + mu sum <e_i>_+^2
 * over the in-plane principal strains e_i, lam = K - 2 mu cdim.  The fixed-stress schemes
 * act on the trace part (S1), the second part (S2) or both (S3) of Psi+ for either split;
 * with VD these are the forms of Sec. 3.4.  The spectral split's Newton tangent depends
 * on the strain, not on a sign bit: its u-solves run on an assembled nodal stencil of the
 * per-point tangents (FP64 and FP32 copies) instead of the matrix-free operator. */
enum { PF_SPLIT_VD = 0, PF_SPLIT_SPECTRAL = 1 };

/* Structured Q1 mesh; host pointers, copied by pf_create. */
typedef struct {
  int nx, ny;                  /* elements per side, >= 1 */
  double Lx, Ly;               /* side lengths (mm), > 0 */
  const uint8_t *elem_active;  /* nx*ny bytes (0 = masked out) or NULL = all active */
  const uint8_t *node_flags;   /* N bytes of PF_* flag bits; must not be NULL */
  int plane;                   /* PF_PLANE_STRAIN (3D invariants, eps_zz = 0) or
                                  PF_PLANE_STRESS (2D invariants, K = E/(2(1-nu))) */
  int precision;               /* PF_FP64 or PF_FP32_IR */
  int reaction_dir;            /* 0: x, 1: y -- component summed over LOAD nodes */
  int precond;                 /* PF_PRECOND_JACOBI or PF_PRECOND_GMG */
  int model;                   /* PF_AT2_HISTORY (0): AT2, w = d^2, c_w = 2, history field
                                  H = max Psi+ drives the (linear) evolution equation;
                                  PF_AT1_PENALTY (1): AT1, w = d, c_w = 8/3, current Psi+ and
                                  the penalty gamma <d - d_{n-1}>_- (Sec. 2, Table 1),
                                  semismooth Newton per d-solve */
  double tol_ir;               /* AT1 irreversibility tolerance: gamma = 27 G_c / (64 l
                                  tol_ir^2) (Sec. 2); <= 0 selects 0.01 */
  int split;                   /* PF_SPLIT_VD (0) or PF_SPLIT_SPECTRAL (1) */
} pf_mesh;

#define PF_AT2_HISTORY 0
#define PF_AT1_PENALTY 1

/* Solver controls.  pf_default_options fills the defaults given in brackets. */
typedef struct {
  double tol_nr;     /* [1e-7] Newton stop: ||R_free|| <= tol_nr*max(||R0_free||, ||F_constr||)
                        (TOL_NR of Sec. 4) */
  double tol_lin;    /* [1e-10] relative residual of every linear solve (d-solves; u-solves
                        when newton_forcing is 0) */
  double tol_inner;  /* [1e-3] relative residual of one FP32 inner solve (PF_FP32_IR) */
  int max_newton;    /* [50] Newton iterations per u-solve */
  int max_stag;      /* [1000] staggered iterations per load step */
  int max_lin;       /* [200000] Krylov iterations per linear solve */
  int max_refine;    /* [30] FP64 refinement sweeps per linear solve (PF_FP32_IR) */
  double psi_crit;   /* [-1] < 0: G_c/(c_w l) of Sec. 3.5; else the given threshold */
  int project;       /* [0] 1: clamp d into [d_{n-1}, 1] after every d-solve */
  int check_every;   /* [8] Krylov iterations between host convergence reads when
                        device_loop is 0 or the device-side loop is unavailable */
  double newton_forcing; /* [1e-3] inexact Newton for u: the correction at residual R_k is
                        solved to the relative residual max(tol_lin, min(1e-2,
                        newton_forcing * tol_nr * max(||R0||, ||F_constr||) / ||R_k||)), so
                        that the linear residual stays below the Newton tolerance; 0 solves
                        every correction to tol_lin */
  int device_loop;   /* [1] 1: each Krylov solve is one CUDA graph whose iterations loop on
                        the device (conditional WHILE node, one host synchronisation per
                        solve); 0: host-checked batches of check_every iterations (same
                        kernels; for profilers that cannot see inside conditional nodes) */
} pf_options;

typedef struct {
  double ubar;          /* prescribed displacement after the step */
  double reaction;      /* sum of the internal force over LOAD nodes (force / thickness) */
  double stag_residual; /* max_i |R_d,i / K_dd,ii| at the last check (free d DOFs) */
  int stag_iters;       /* d-u passes of this step */
  int newton_u;         /* Newton linear solves for u */
  int lin_u;            /* Krylov iterations in u-solves (inner iterations in FP32_IR) */
  int lin_d;            /* Krylov iterations in d-solves, incl. the augmented S-solve */
  int d_solves;         /* d linear solves (ST: 1 per pass, S1/S2/S3: 2 per pass) */
  int refine_steps;     /* FP64 refinement sweeps (PF_FP32_IR) */
  int converged;        /* 1 if the staggered residual met tol */
  double ms;            /* device time of the step (CUDA events), milliseconds */
} pf_step_result;

typedef struct pf_ctx pf_ctx;

void pf_default_options(pf_options *opt);
/* Environment: PF_PDL=0 launches the kernels of the Krylov iteration without programmatic
 * dependent launch (by default each is dispatched while its predecessor drains and waits
 * for it on the device; results are the same either way). */

/* Create a simulation (Sec. 2 model with E, nu, G_c, l and residual stiffness k_res,
 * the eta of g(d) = (1-d)^2 + eta).  Allocates all device memory for the mesh; the
 * state starts at u = 0, H = 0, d = Dirichlet values (1 on PF_D_FIX1 nodes, else 0),
 * ubar = 0.  Uses the calling thread's current CUDA device and a new stream.
 * Errors: PF_EINVAL (nx, ny < 1; L <= 0; nu outside (-1, 0.5); E, Gc, l <= 0;
 * k_res < 0; NULL pointers), PF_ENOMEM, PF_ECUDA.  *out is NULL on error. */
pf_status pf_create(const pf_mesh *mesh, double E, double nu, double Gc, double l,
                    double k_res, pf_ctx **out);
/* Device bytes pf_create allocates for this mesh (0 for an invalid mesh); a scheduler
 * admits simulations by this footprint.  Exact: pf_create takes every array of the
 * context from one allocation of this size (each array 256-byte aligned); the driver's
 * page rounding (up to 2 MiB) and pf_batch_attach's few hundred bytes come on top. */
size_t pf_footprint_bytes(const pf_mesh *mesh);
pf_status pf_set_options(pf_ctx *ctx, const pf_options *opt);
pf_status pf_get_options(const pf_ctx *ctx, pf_options *opt);

/* One load step (Sec. 3.1 and 3.3-3.5): ubar += d_ubar, Dirichlet lift, u-solve with
 * d_{n-1}, then staggered passes {d-step by `scheme`; u-solve; residual check} until
 * stag_residual <= tol or max_stag passes; H_n = max(H_{n-1}, Psi+(u_n)).
 * `out` may be NULL.  Returns PF_ENOTCONV (state advanced, out->converged = 0) when a
 * cap was hit.  Synchronises the context's stream before returning. */
pf_status pf_load_step(pf_ctx *ctx, double d_ubar, int scheme, double tol,
                       pf_step_result *out);

/* Copy the committed state to caller-owned host arrays (any may be NULL):
 * u: 2N doubles, d: N doubles, H: 4*nx*ny doubles. */
pf_status pf_get_fields(pf_ctx *ctx, double *u, double *d, double *H);
/* Overwrite the committed state from host arrays (any may be NULL = keep). */
pf_status pf_set_fields(pf_ctx *ctx, const double *u, const double *d, const double *H,
                        double ubar);

/* Serialised state (u, d, H, ubar, step count) for checkpoint/resume. */
size_t pf_state_size(const pf_ctx *ctx);
pf_status pf_get_state(pf_ctx *ctx, void *buf, size_t size);
pf_status pf_set_state(pf_ctx *ctx, const void *buf, size_t size);

/* Counts of the mesh: nodes N, elements, quadrature points. */
pf_status pf_sizes(const pf_ctx *ctx, int64_t *n_nodes, int64_t *n_elems, int64_t *n_qp);
/* Kernel launches issued by this context since creation (for accounting). */
int64_t pf_launch_count(const pf_ctx *ctx);

/* Host milliseconds accumulated per phase of pf_load_step since creation or the last
 * reset: each phase ends in a stream synchronisation, so these are device-bound times
 * plus launch gaps.  ms[i] for i < n (n <= PF_PROF_PHASES); reset != 0 zeroes them. */
enum {
  PF_PROF_U_SETUP = 0,  /* multigrid hierarchy builds for u */
  PF_PROF_U_SOLVE = 1,  /* Newton corrections for u (Krylov + refinement), incl. setups */
  PF_PROF_U_RESID = 2,  /* internal-force residual + norms per Newton iterate */
  PF_PROF_D_SETUP = 3,  /* multigrid hierarchy builds for d */
  PF_PROF_D_SOLVE = 4,  /* d linear solves (ST, augmented and frozen S-solves), incl. setups */
  PF_PROF_STAG = 5,     /* staggered residual checks */
  PF_PROF_TOTAL = 6,    /* whole load steps */
  PF_PROF_PHASES = 8
};
pf_status pf_profile(pf_ctx *ctx, double *ms, int n, int reset);

const char *pf_last_error(const pf_ctx *ctx);
const char *pf_status_string(pf_status s);
void pf_destroy(pf_ctx *ctx);

/* ------------------------------------------------------------------------------------
 * Autotuning.  Launch shapes of the FP32 multigrid solve timed on the context's own grid
 * (CUDA events on its stream, 3 untimed and 10 timed launches each) and fixed for its
 * later load steps: the node rows per warp of the strip kernel that applies the FP32
 * elasticity tangent (2, 4 or 8) and the largest level, in nodes, that the single-CTA
 * coarse cycle takes (300, 1100 or 4300; larger levels run as grid-wide kernels).  Both
 * change only how the work is split into launches and CTAs, not the method; reductions
 * are grouped differently, so results can change in the last bits.  The paper has no
 * counterpart (it names no hardware mapping).
 * ------------------------------------------------------------------------------------ */
typedef struct {
  int strip_rows;          /* chosen rows per warp; 0 = grid-size rule (not tuned) */
  int coarse_nodes;        /* chosen single-CTA coarse-cycle limit; 0 = built-in 1100 */
  double apply_us[3];      /* FP32 tangent apply, strip rows 2, 4, 8 (0: not timed) */
  double vcycle_us[3];     /* V-cycle below the fine level, coarse limits 300, 1100, 4300 */
} pf_tuning;
/* Time the candidates and keep the fastest.  Only before the first load step of ctx and
 * while ctx is not attached to a batch (PF_EBUSY otherwise); PF_EINVAL unless ctx uses
 * PF_FP32_IR with PF_PRECOND_GMG and the VD split.  out (may be NULL) receives the choice
 * and the timings. */
pf_status pf_autotune(pf_ctx *ctx, pf_tuning *out);
/* The current choice (zeros where pf_autotune has not run). */
pf_status pf_get_tuning(const pf_ctx *ctx, pf_tuning *out);

/* ------------------------------------------------------------------------------------
 * Batches.  Several simulations advanced together so that their Krylov solves share
 * kernel launches.  Each attached context runs its load steps on its own host thread (or
 * through pf_batch_load_step); whenever every attached context that is inside a load
 * step waits for an FP32 multigrid solve (the inner solves of PF_FP32_IR with
 * PF_PRECOND_GMG and the VD split; Sec. 3.1-3.5 are unchanged), those solves run as one
 * captured CUDA graph in which each fused PCG stage, multigrid level and coarse cycle is
 * one launch for all of them, on the batch's own stream, with a device-side loop that
 * stops every simulation's iteration on its own convergence test.  A simulation's
 * arithmetic does not depend on the others: its results are bit-identical alone and in
 * any batch.  Other solves (FP64, Jacobi, spectral split, grids too small for the fused
 * multigrid) run per context as without a batch.  The paper has no batching layer; this
 * is the lock-step executor of the batched workloads.
 * ------------------------------------------------------------------------------------ */
typedef struct pf_batch pf_batch;
/* A batch on the calling thread's CUDA device.  Errors: PF_EINVAL, PF_ENOMEM, PF_ECUDA. */
pf_status pf_batch_create(pf_batch **out);
/* Attach ctx (same device, not attached elsewhere: PF_EBUSY).  Allocates a few hundred
 * bytes of device memory per multigrid hierarchy.  Not while ctx is in a load step. */
pf_status pf_batch_attach(pf_batch *b, pf_ctx *ctx);
/* Detach ctx; PF_EBUSY while ctx is inside a load step.  pf_destroy detaches too. */
pf_status pf_batch_detach(pf_batch *b, pf_ctx *ctx);
/* One load step of each of the n distinct attached contexts ctx[i] (increment d_ubar[i],
 * scheme[i], tolerance tol[i]), run concurrently on n host threads; returns when all are
 * done.  res[i] / status[i] (each n long or NULL) receive what pf_load_step returns for
 * ctx[i].  Returns PF_OK, PF_ENOTCONV if some step did not converge, or the first hard
 * error; PF_EINVAL for a context not attached to b or listed twice. */
pf_status pf_batch_load_step(pf_batch *b, int n, pf_ctx *const *ctx, const double *d_ubar,
                             const int *scheme, const double *tol, pf_step_result *res,
                             pf_status *status);
/* Kernel launches of the batched solves, solves and launch groups run, largest group. */
pf_status pf_batch_stats(const pf_batch *b, int64_t *launches, int64_t *solves,
                         int64_t *groups, int *max_group);
/* Detach every context and free the batch.  No load step of an attached context may be
 * running. */
void pf_batch_destroy(pf_batch *b);

/* ------------------------------------------------------------------------------------
 * Serving.  A continuous-batching request server on the calling thread's CUDA device:
 * `slots` host worker threads each run one simulation at a time (pf_create, one
 * pf_load_step per load increment, pf_destroy), so up to `slots` simulations are resident
 * and their kernels overlap on the device, each on its own stream.  Requests are admitted
 * first come, first served when a slot is free and their device footprint
 * (pf_footprint_bytes) fits in `hbm_budget` minus the footprints of the running
 * simulations; the queue head blocks the requests behind it.  The kernels are
 * deterministic, so a request gives the same results alone and in the mix.  The paper has
 * no serving layer; this is the request loop of the served-batch workload.
 * ------------------------------------------------------------------------------------ */
typedef struct pf_server pf_server;

typedef struct {
  pf_mesh mesh;                 /* as for pf_create; node_flags / elem_active copied */
  double E, nu, Gc, l, k_res;   /* as for pf_create */
  const double *increments;     /* host, n_steps load increments (copied at submit) */
  int n_steps;                  /* >= 1 */
  int scheme;                   /* PF_ST .. PF_S3 */
  double tol;                   /* staggered tolerance of every step, > 0 */
  const pf_options *options;    /* NULL: pf_default_options (copied at submit) */
} pf_request;

enum {
  PF_REQ_QUEUED = 0,
  PF_REQ_RUNNING = 1,
  PF_REQ_DONE = 2,
  PF_REQ_FAILED = 3,
  PF_REQ_CANCELLED = 4   /* withdrawn while queued, or stopped between load steps */
};

typedef struct {
  int state;           /* PF_REQ_* */
  int status;          /* PF_OK, or the status of the call that failed (PF_REQ_FAILED);
                          a step that hit a cap (PF_ENOTCONV) does not fail the request */
  int steps_done;      /* load steps completed */
  int steps_converged; /* of those, steps whose staggered residual met tol */
  int64_t admit_seq;   /* 0-based admission order, -1 while queued */
  size_t footprint;    /* device bytes reserved for the request */
  double queue_ms;     /* submit -> admission (host clock) */
  double path_ms;      /* submit -> completion (host clock), 0 until done */
  double step_ms_p50;  /* device time per load step (pf_step_result.ms), over done steps */
  double step_ms_p99;
} pf_request_info;

/* hbm_budget > 0 bytes, slots >= 1.  Errors: PF_EINVAL, PF_ENOMEM. */
pf_status pf_server_create(size_t hbm_budget, int slots, pf_server **out);
/* Queue a request; *id receives its id (>= 1).  PF_EINVAL for an invalid request or one
 * whose footprint exceeds the whole budget; PF_EBUSY after pf_server_destroy began. */
pf_status pf_server_submit(pf_server *s, const pf_request *req, int64_t *id);
/* State of request `id`.  reactions (double) and stag_iters (int), each n_steps long or
 * NULL, receive the per-step reaction force and staggered passes of the steps done so
 * far.  PF_EINVAL for an unknown id. */
pf_status pf_server_poll(pf_server *s, int64_t id, pf_request_info *info, double *reactions,
                         int *stag_iters);
/* Wait until no request is queued or running; PF_ETIMEOUT after timeout_s seconds
 * (timeout_s < 0 waits without limit). */
pf_status pf_server_drain(pf_server *s, double timeout_s);
/* Peaks since creation: device bytes reserved and simulations running at once. */
pf_status pf_server_stats(pf_server *s, size_t *peak_bytes, int *peak_running);
/* Cancel request `id`: a queued request is withdrawn without being started; a running
 * one stops after its current load step (its results so far stay readable).  PF_EINVAL
 * for an unknown id; a finished request is left as it is. */
pf_status pf_server_cancel(pf_server *s, int64_t id);
/* Forget a finished (done, failed or cancelled) request and free its results; later
 * calls with `id` return PF_EINVAL.  PF_EBUSY while it is queued or running. */
pf_status pf_server_release(pf_server *s, int64_t id);
/* paused != 0: admit no further requests (running ones continue); 0: resume admission. */
pf_status pf_server_pause(pf_server *s, int paused);
/* Stop: requests still queued are not started; running ones finish their load path;
 * the worker threads are joined and all memory freed.  No other pf_server_* call on `s`
 * may be in progress or follow. */
void pf_server_destroy(pf_server *s);

/* ------------------------------------------------------------------------------------
 * Operator level.  Stateless single operations on caller-owned DEVICE arrays, enqueued
 * on `stream` (a cudaStream_t, NULL = legacy default stream) and not synchronised
 * unless stated.  These are the building blocks of pf_load_step, exposed for checking
 * and for callers with their own drivers.
 * ------------------------------------------------------------------------------------ */

/* Grid descriptor: device pointers may be NULL where stated. */
typedef struct {
  int nx, ny;
  double hx, hy;                /* element sizes Lx/nx, Ly/ny */
  const uint8_t *elem_active;   /* device, nx*ny bytes, or NULL = all active */
  const uint8_t *dof_mask;      /* device, N bytes from pf_op_dof_mask, or NULL: no DOF
                                   constrained (operators return plain K x) */
} pf_grid;

/* Material in the notation of Sec. 2: shear modulus mu, bulk modulus K, deviatoric
 * factor cdim (1/3 plane strain, 1/2 plane stress), eta, G_c, l, and the energy split
 * (PF_SPLIT_VD or PF_SPLIT_SPECTRAL; pf_material_make sets PF_SPLIT_VD). */
typedef struct {
  double mu, K, cdim, eta, Gc, l;
  int split;
} pf_material;

pf_status pf_material_make(double E, double nu, double Gc, double l, double k_res,
                           int plane, pf_material *out);

/* dof_mask[n] bit0: u_x constrained, bit1: u_y constrained, bit2: d constrained,
 * bit3: node without active element (then all DOFs constrained at 0), from node flags
 * and the element mask.  node_flags, elem_active (may be NULL), dof_mask: device arrays. */
pf_status pf_op_dof_mask(int nx, int ny, const uint8_t *node_flags,
                         const uint8_t *elem_active, uint8_t *dof_mask, void *stream);

/* Internal force of the momentum balance, F = sum_e sum_q w B^T sigma(eps(u), d)
 * (weak form F_u of Sec. 3.2 without the boundary term), over all 2N DOFs, FP64, for the
 * material's split.  VD: `tension` (may be NULL) receives one byte per element, bit q set
 * where tr eps > 0 at Gauss point q (the indicator I_+ of Sec. 3.3).  SPECTRAL: `tension`
 * is not written; the call allocates and frees device scratch (12 doubles per element)
 * and synchronises `stream`.  dof_mask ignored. */
pf_status pf_op_elas_residual(const pf_grid *g, const pf_material *m, const double *u,
                              const double *d, double *F, uint8_t *tension, void *stream);

/* y = K_uu x, the tangent of F for a frozen indicator `tension` (stress increment of
 * Sec. 3.3 at fixed d), VD split (the material's split is not read).  Rows/columns of
 * constrained DOFs (dof_mask) are zeroed. dtype PF_F64 or PF_F32 for d, x, y. */
pf_status pf_op_elas_apply(const pf_grid *g, const pf_material *m, int dtype, const void *d,
                           const uint8_t *tension, const void *x, void *y, void *stream);
/* diag[i] = (K_uu)_ii for free DOFs, 0 for constrained ones. */
pf_status pf_op_elas_diag(const pf_grid *g, const pf_material *m, int dtype, const void *d,
                          const uint8_t *tension, void *diag, void *stream);

/* Newton tangent of the stress at every Gauss point for the material's split, FP64:
 * Dq[k * 4 ne + 4 e + q], k = 0..5 the entries D00, D01, D02, D11, D12, D22 of the
 * symmetric 3 x 3 Voigt matrix (xx, yy, engineering xy) mapping a strain increment to a
 * stress increment.  VD: the frozen-indicator form at the sign of tr eps(u); SPECTRAL: the
 * consistent tangent (principal-frame derivative of eps+).  Masked elements get 0. */
pf_status pf_op_elas_tangent_qp(const pf_grid *g, const pf_material *m, const double *u,
                                const double *d, double *Dq, void *stream);
/* y = K(Dq) x = sum_e sum_q w B^T D_q B x with Dq as written by pf_op_elas_tangent_qp,
 * through the assembled nodal stencil (9 neighbours x 2 x 2 blocks per node) that the
 * spectral-split u-solves use.  Rows/columns of constrained DOFs (dof_mask) zeroed.
 * dtype PF_F64 or PF_F32 for x and y (and the stencil); allocates and frees the stencil
 * (36 values per node) and synchronises `stream`. */
pf_status pf_op_elas_apply_qp(const pf_grid *g, int dtype, const double *Dq, const void *x,
                              void *y, void *stream);

/* y = K_dd x = sum_q w [c_q N N^T + kappa grad N . grad N^T] x (evolution equation
 * tangent, Sec. 3.2; AT2: c_q = G_c/l + 2 H_q (+ K~_q), kappa = G_c l).  c: 4*ne per
 * Gauss point.  Constrained rows/columns (dof_mask bit2) zeroed. */
pf_status pf_op_damage_apply(const pf_grid *g, int dtype, const void *c, double kappa,
                             const void *x, void *y, void *stream);
pf_status pf_op_damage_diag(const pf_grid *g, int dtype, const void *c, double kappa,
                            void *diag, void *stream);
/* b = sum_q w 2 H_q N (AT2 driving term), all N DOFs, FP64. */
pf_status pf_op_damage_rhs(const pf_grid *g, const double *H, double *b, void *stream);

/* Per Gauss point (FP64): psi = Psi+(eps(u)) (Sec. 2, the material's split) and
 * Hout = max(Hprev, psi) (history update).  psi may be NULL. */
pf_status pf_op_qp_energy(const pf_grid *g, const pf_material *m, const double *u,
                          const double *Hprev, double *psi, double *Hout, void *stream);

/* Fixed-stress coefficient (Sec. 3.4-3.5), per Gauss point, FP64:
 *   active = Psi+ > psi_crit && Psi+ > Hprev && d_q < 0.95 (strict),
 *   c_aug  = G_c/l + 2 max(Hprev, Psi+) + (active ? -4 (1-d_q)^2/g(d_q) Q_S : 0),
 * Q_S1 = K<tr>_+^2, Q_S2 = 2 mu e.e, Q_S3 = sum (VD; SPECTRAL: Q_S1 = lam <tr>_+^2,
 * Q_S2 = 2 mu sum <e_i>_+^2, Q_S3 = sum).  active: one byte per Gauss point. */
pf_status pf_op_fs_coeff(const pf_grid *g, const pf_material *m, int scheme,
                         double psi_crit, const double *u, const double *d,
                         const double *Hprev, double *c_aug, uint8_t *active,
                         void *stream);
/* Predicted history (Sec. 3.3 with the Delta d > 0 rule of Sec. 3.5), FP64:
 *   s = 1 + 2(1-d_q)/g(d_q) max(Delta d_q, 0); S1: <tr>_+ -> s<tr>_+; S2: e.e -> s^2 e.e;
 *   S3: both (SPECTRAL: S1 scales the trace part, S2 the part mu sum <e_i>_+^2, by s^2);
 *   Hhalf = max(Hprev, active ? Psi_hat : Psi+). */
pf_status pf_op_fs_predict(const pf_grid *g, const pf_material *m, int scheme,
                           const double *u, const double *d, const double *dd,
                           const double *Hprev, const uint8_t *active, double *Hhalf,
                           void *stream);

/* Reaction: sum of F component `dir` over nodes with PF_LOAD_X (dir 0) / PF_LOAD_Y
 * (dir 1) that have an active element.  Result written to *out (host), synchronises
 * `stream`.  Uses a device scratch buffer allocated by the call. */
pf_status pf_op_reaction(const pf_grid *g, const uint8_t *node_flags, const double *F,
                         int dir, double *out, void *stream);

/* Staggered residual (reading of Sec. 3.1): with H = max(Hprev, Psi+(u)),
 *   out = max over free d DOFs of |(K_dd(H) d - b(H))_i / (K_dd(H))_ii|.
 * FP64.  Synchronises `stream`; allocates device scratch for the call. */
pf_status pf_op_stag_residual(const pf_grid *g, const pf_material *m, const double *u,
                              const double *d, const double *Hprev, double *out,
                              void *stream);

/* Allocation-free variant of pf_op_stag_residual (the paper has no counterpart; this is
 * an interface convenience).  pf_op_stag_residual allocates and frees device scratch on
 * every call, which some callers cannot do: code whose device memory is owned by another
 * allocator (a framework's caching pool with a fixed budget), and code that must not
 * stall the device, since cudaMalloc and cudaFree can synchronise it.  This variant takes
 * the same inputs and gives the same result, but keeps its scratch in a static device
 * array of PF_NOALLOC_MAX_DOUBLES doubles (about 12 MiB) that every GPU which loads the
 * library holds until the process exits.  It calls no allocation routine.
 *   Size limit: 2*Q + 3*N <= PF_NOALLOC_MAX_DOUBLES (Q = 4*nx*ny Gauss points, N nodes),
 *   about 136,000 elements (e.g. 368 x 368); larger grids return PF_EINVAL before any
 *   GPU work.
 *   First call on a device: resolves the scratch address with cudaGetSymbolAddress while
 *   that device is current; make that first call before any stream capture.
 *   Sharing: every call on a device uses the same scratch, and the last call's contents
 *   stay there; calls whose work overlaps on the GPU (different streams or threads at the
 *   same time) race and must be serialised by the caller.
 * Synchronises `stream`; the result goes to *out (host). */
#define PF_NOALLOC_MAX_DOUBLES 1500000
pf_status pf_op_stag_residual_noalloc(const pf_grid *g, const pf_material *m, const double *u,
                                      const double *d, const double *Hprev, double *out,
                                      void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
