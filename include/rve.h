/*
 * rve.h -- C ABI of the GB300 ADMM solver for periodic micromechanics cells.
 *
 * Method: Zhou & Bhattacharya, "Accelerated computational micromechanics",
 * Section 2.1 (augmented Lagrangian, eq. al; ADMM Steps 1-4, eqs. eq, helm,
 * update, check; penalty update eq. rho-update) on the periodic unit cell of
 * Section 2.3 (strain control <F> = Fbar, central-difference symbols).
 *
 * Conventions shared by every call
 *   - The cell is the unit cube [0,1)^d, d = 2 (plane strain) or 3, on an
 *     N^d grid, h = 1/N.  N is even, of the form 2^a 3^b, 4 <= N <= 512.
 *   - A scalar field is N^d values, x fastest: index (z*N + y)*N + x.
 *   - A tensor field (F, Lambda) is d*d scalar fields, component-major,
 *     component (i, j) at offset (i*d + j) * N^d.  A vector field (u~, n) is
 *     d (or 3 for n) scalar fields.
 *   - 3x3 host matrices (Fbar, stress) are row-major double[9]; in 2D only the
 *     upper-left 2x2 block is read or written (the rest of stress is zero).
 *   - The multiplier Lambda has the paper's sign: the Lagrangian term is
 *     Lambda : (grad u - F), so Lambda converges to the first Piola-Kirchhoff
 *     stress (Section 2.1, "Connection to physics").
 *   - All calls return an int status: RVE_OK (0) or a negative RVE_E_* code.
 *     No exception crosses the ABI and device code never traps; device-side
 *     failures come back as status codes.  rve_strerror() names a code.
 *   - A handle is used by one host thread at a time.
 *   - Host pointers passed in are read during the call only; the caller keeps
 *     ownership.  Device memory is owned by the handle (or by the caller when a
 *     workspace is supplied to rve_create_in).
 */
#ifndef RVE_H
#define RVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define RVE_OK 0
#define RVE_E_INVALID_ARG (-1)   /* bad size, pointer, enum or value          */
#define RVE_E_OOM (-2)           /* device allocation or workspace too small */
#define RVE_E_NOT_CONVERGED (-3) /* max_iter reached; state valid, info set  */
#define RVE_E_NUMERICAL (-4)     /* NaN/Inf residual or J <= 0 in the state  */
#define RVE_E_CUDA (-5)          /* a CUDA runtime call failed               */
#define RVE_E_BUSY (-6)          /* server: no slot / queue full             */
#define RVE_E_STATE (-7)         /* call out of order (e.g. no material set) */
#define RVE_E_NOT_FOUND (-8)     /* server: unknown or finished ticket       */

/* ------------------------------------------------------------------ enums */
enum rve_model {
    RVE_NEOHOOKE = 0, /* W = mu/2(|F|^2 - d - 2 ln J) + lam/2 (J-1)^2, Section 4.1
                         params per phase: {mu, lam}                           */
    RVE_LINEAR = 1,   /* W = mu|sym(F-I)|^2 + lam/2 tr(F-I)^2, params {mu, lam} */
    RVE_LCE = 2       /* liquid crystal elastomer, Section 5.1 (3D only); params
                         per phase {mu, lam, r, alpha, kappa_F}; needs n0      */
};
enum rve_precision {
    RVE_FP64 = 0,  /* every field, FFT and local solve in double                 */
    RVE_MIXED = 1, /* float bulk (fields, FFT, Newton) with double residuals and
                      stress; promoted to double for the final iterations        */
    RVE_FP32 = 2   /* float bulk only, double residuals (stops at its floor)     */
};
enum rve_rho_policy { RVE_RHO_FIXED = 0, RVE_RHO_ADAPTIVE = 1 };
enum rve_lambda0 { RVE_LAMBDA0_STRESS = 0, RVE_LAMBDA0_ZERO = 1 };
enum rve_field { RVE_FIELD_F = 0, RVE_FIELD_LAMBDA = 1, RVE_FIELD_U = 2, RVE_FIELD_N = 3 };

/* ------------------------------------------------------------------ options */
typedef struct rve_options {
    int precision;      /* enum rve_precision, default RVE_FP64                    */
    int rho_policy;     /* enum rve_rho_policy, default fixed                      */
    int lambda0;        /* initial multiplier of a fresh state: W_F(Fbar) or 0     */
    int max_iter;       /* ADMM iteration cap per solve, default 1000              */
    int newton_max;     /* per-voxel Newton iteration cap, default 30              */
    double newton_tol;  /* Newton stops after a full step with max|dF| <= this;
                           0 selects 1e-10 (double) / 1e-5 (float)                 */
    double rho_kappa;   /* adaptive rho factor (eq. rho-update), default 1.3       */
    double rho_tau;     /* adaptive rho balance threshold, default 10              */
    double rho_min;     /* adaptive rho lower bound; 0 selects mu_ref              */
    double mu_ref;      /* modulus in r_d (eq. check); 0 selects the volume average
                           of the per-voxel shear modulus                          */
    double mixed_switch;/* RVE_MIXED: promote to double once max(r_p, r_d) <= this
                           or float stagnates; default 3e-7 (float r_p levels off
                           near 1.3e-7 on O(1) deformation gradients, and float
                           iterations below about 3e-7 no longer track the
                           double iteration)                                       */
    int check_every;    /* host reads the device status every this many iterations */
    int use_graph;      /* 1: replay iteration chunks as a CUDA graph (default 1)  */
    double local_ratio; /* f > 0: inexact local steps (Section 2.1, "Approximate
                           solution of the local problem"; Section 4.2 adopts
                           r_l <= f r_d with f = 0.3).  Each voxel's Newton stops
                           once |grad phi|_F <= f mu_ref r_d, r_d of the last
                           check complete when the local step starts (two checks
                           back: the device fuses Step 1 with the previous check);
                           the first two local steps of a solve are exact.  The
                           pointwise bound implies r_l <= f r_d.  Not applied to the
                           increment-form steps of the RVE_MIXED polish.  Default 0
                           (exact local solves).                                   */
    double local_fraction; /* p in (0, 1], elastic laws: fraction-converged local steps (Section
                           4.2's first strategy: proceed once a fraction p of the
                           voxels met the pointwise Newton test, checked every two
                           local iterations).  Built without a grid-wide barrier:
                           each voxel's Newton is capped at K, the smallest even
                           count by which a fraction p converged in the previous
                           pass (K + 2 if fewer converged within K, at most
                           newton_max); the first two local steps of a solve use
                           newton_max.  Not applied to the increment-form steps of
                           the RVE_MIXED polish.  Default 0 (off).                 */
} rve_options;

/* Fill *opt with the defaults listed above. */
void rve_default_options(rve_options* opt);

/* ------------------------------------------------------------------ solve info */
typedef struct rve_solve_info {
    int iterations;        /* ADMM iterations done by this solve (all precisions) */
    int fp64_iterations;   /* of which in double (RVE_MIXED polish)               */
    int converged;         /* 1 if r_p <= tol and r_d <= tol                      */
    int status;            /* same code the call returned                         */
    double r_p, r_d;       /* residuals of the last iteration (eq. check)         */
    double rho;            /* penalty used in the last iteration                  */
    double mu_ref;         /* modulus used in r_d                                 */
    int newton_max_iters;  /* largest per-voxel Newton count in the last pass     */
    long long newton_fail; /* voxels that hit newton_max in the last pass         */
    double time_ms;        /* device time of the iteration loop (CUDA events)    */
    long long launches;    /* kernel launches this solve issued (graph nodes too) */
    double r_l;            /* local residual (Section 2.1) of the last fused
                              pass's local step, |grad phi| at the step's result in
                              the unit-cell L2 norm over mu_ref; 0 unless
                              local_ratio > 0                                      */
} rve_solve_info;

typedef struct rve* rve_t;

/* ------------------------------------------------------------------ lifetime */
/* Create a solver for a d-dimensional N^d cell (d = 2 or 3).  All device state
 * is allocated here with cudaMalloc and stays resident until rve_destroy.
 * opt may be NULL (defaults).  cuda_stream is a cudaStream_t (NULL = legacy
 * default stream); all device work of the handle is ordered after prior work
 * on that stream and each call returns with its work finished.
 * Errors: RVE_E_INVALID_ARG (bad d, N, options), RVE_E_OOM, RVE_E_CUDA. */
int rve_create(rve_t* out, int dim, int n, int model, const rve_options* opt, void* cuda_stream);

/* Same as rve_create but carves all device state out of a caller-owned device
 * buffer of `bytes` bytes (>= rve_workspace_bytes(...), 256-byte aligned), which
 * must outlive the handle.  Nothing is allocated on the device.  RVE_E_INVALID_ARG
 * for a NULL or misaligned buffer, RVE_E_OOM when `bytes` is too small. */
int rve_create_in(rve_t* out, int dim, int n, int model, const rve_options* opt, void* cuda_stream,
                  void* device_workspace, size_t bytes);

/* Device bytes a handle of this shape and these options needs (fields, tables,
 * control block, residual history); opt may be NULL (defaults).  0 if invalid. */
size_t rve_workspace_bytes(int dim, int n, int model, const rve_options* opt);

/* Release the handle and, unless the workspace was supplied, its device memory. */
void rve_destroy(rve_t h);

/* ------------------------------------------------------------------ material */
/* Set the microstructure: phase[N^d] (host, values < nphase), params[nphase *
 * nparam] per-phase constants of the model (see enum rve_model), n0[3 * N^d]
 * (host, unit vectors, component-major) for RVE_LCE, else NULL.  Marks the
 * state fresh: the next solve starts from F = Fbar, u~ = 0, Lambda_0.
 * Errors: RVE_E_INVALID_ARG (phase id out of range, non-positive modulus,
 * nparam too small, missing n0), RVE_E_CUDA. */
int rve_set_material(rve_t h, const uint8_t* phase, int nphase, const double* params, int nparam,
                     const double* n0);
/* RVE_LCE parameters per phase: mu, lambda, r, alpha, kappa_F (Section 5.1 with the
 * readings of the build), optionally nu_F/dt and nu_n/dt: the dissipation weights of
 * one implicit time step, dt D((F - F^n)/dt, (n - n^n)/dt) = nu_F/(2 dt) |F - F^n|^2 +
 * nu_n/(2 dt) |n - n^n|^2, with (F^n, n^n) the state the solve starts from (default 0:
 * the equilibrium problem).  <S> then includes the viscous part nu_F/dt (F - F^n).
 * An eighth entry 1 (0: default) makes the network incompressible: W loses its
 * volumetric terms (-mu ln J, lambda is ignored) and det F = 1 is enforced in the
 * local step by a Lagrange multiplier (Section 5.1), always solved to the step
 * tolerance (opt.local_ratio does not apply to it).  Every phase must give the same
 * value.  The reaction pressure is not part of the state: rve_stress then returns
 * <Lambda>, which equals <W_F - p cof F> (+ the viscous part) once converged. */

/* ------------------------------------------------------------------ solve */
/* Run ADMM iterations (Section 2.1, Steps 1-4) at macroscopic gradient Fbar
 * until r_p <= tol and r_d <= tol or opt.max_iter iterations.  A fresh state is
 * initialised from Fbar; otherwise the resident state (F, Lambda, u~) of the
 * previous solve is the warm start (the previous load step, Algorithm 1).  rho
 * is the penalty (the starting value under the adaptive policy).  tol < 0 runs
 * exactly max_iter iterations.  info may be NULL.
 * Returns RVE_OK, RVE_E_NOT_CONVERGED (state valid), RVE_E_NUMERICAL,
 * RVE_E_STATE (no material), RVE_E_INVALID_ARG (rho <= 0, det Fbar <= 0),
 * RVE_E_CUDA. */
int rve_solve(rve_t h, const double Fbar[9], double rho, double tol, rve_solve_info* info);

/* Mixed macroscopic control (Section 2.3: some components of <F> prescribed, the
 * complementary components of <S> zero; Section 5.3's UNI, PE and EB loadings).
 * free_mask bit 3i+j set: <F_ij> is free, Fbar[3i+j] is only its starting value,
 * and the solve drives <W_F(F)>_ij to 0 (to the residual tolerance); the other
 * components of Fbar are prescribed.  The free components join Step 2: each
 * iteration sets them to the mean of F - Lambda/rho (Du~ has zero mean), after
 * which <Lambda>_ij = 0.  Bits outside the d x d block are RVE_E_INVALID_ARG.  A
 * mask leaving both <F_ij> and <F_ji> free leaves a rigid rotation to the start
 * value (W is frame-indifferent).  rve_solve is rve_solve_mixed with mask 0.
 * Returns as rve_solve; rve_macro_gradient gives the resulting <F>. */
int rve_solve_mixed(rve_t h, const double Fbar[9], unsigned free_mask, double rho, double tol,
                    rve_solve_info* info);

/* Current macroscopic gradient <F> (row-major 3x3; prescribed and free parts). */
int rve_macro_gradient(rve_t h, double F[9]);

/* A loading path (Section 5.3: quasi-static steps along UNI, PE or EB with the
 * implicit time discretisation of Section 5.1): `steps` solves in order, each warm
 * started from the previous state, which is also the previous time step of the LCE
 * dissipation terms.  Fbars[9 s ...] gives step s's prescribed <F> (row-major);
 * components in free_mask (as in rve_solve_mixed) start from the previous step's
 * result.  Per step: S_out[9 s ...] = <S> after the step, Fbar_out[9 s ...] = <F>
 * (either may be NULL), infos[s] (may be NULL).  Returns RVE_OK, or
 * RVE_E_NOT_CONVERGED if some step stopped at max_iter (all steps still run), or
 * the first other error. */
int rve_solve_path(rve_t h, const double* Fbars, int steps, unsigned free_mask, double rho, double tol,
                   double* S_out, double* Fbar_out, rve_solve_info* infos);

/* ------------------------------------------------------------------ Bloch waves */
/* Result of rve_bloch. */
typedef struct rve_bloch_info {
    int iterations;      /* Steps 1'-4' run                                        */
    int converged;       /* r_p <= tol and r_d <= tol                              */
    double beta;         /* sigma of the last Step 2' (the multiplier of ||p|| = 1):
                            beta_k once converged                                  */
    double rayleigh;     /* <D p, L D p> of the final p (||p|| = 1)                */
    double r_p, r_d;     /* residuals of the last iteration                        */
    double time_ms;      /* device time of the iterations                          */
    long long launches;  /* kernel launches issued                                 */
    int fail;            /* RVE_E_NUMERICAL causes, bits: 1 L + rho I not positive
                            definite, 2 b^ has no weight at the lowest kappa (Step 2'
                            hard case), 4 Step 2' root not found in its passes     */
    double rho;          /* penalty of the last iteration                          */
    int float_iterations; /* of which in the float phase (RVE_MIXED, RVE_FP32)     */
} rve_bloch_info;

/* Modulus of stability beta_k (Section 2.4): the minimum over unit Bloch waves
 * v = p(x) exp(i omega.x), omega_j = 2 pi / k_j, of <grad v, L grad v> with
 * L(x) = W_FF(F(x)) of the handle's material at its resident state F (the
 * solution of the last solve, or a field set with rve_set_field), computed by the
 * Bloch-wave ADMM (Steps 1'-4') with the unit-norm constraint inside Step 2' (its
 * secular equation) and the grid's central differences applied to v, so that beta_k
 * is the smallest eigenvalue of the discrete D^* L D.  k: k[0..d-1] non-zero
 * integers, at least one with |k_j| >= 2 (otherwise the Bloch operator has null
 * modes).  p0: host, 2 d N^d doubles, the start p_0 as (re, im) pairs,
 * component-major like the fields (normalised by the call; not all zero).  rho:
 * penalty, L + rho I must be positive definite everywhere; the iteration count grows
 * about linearly with rho, and a rho too close to the most negative eigenvalue of L
 * lets the iteration diverge (measured on a compressed two-phase cell: stable and
 * fastest near twice that eigenvalue's magnitude).  tol: bound on r_p and
 * r_d (r_d scaled by rho / mu_ref as for rve_solve); max_iter > 0.  The handle's
 * opt.rho_policy applies: RVE_RHO_ADAPTIVE balances the residuals as for rve_solve
 * (Section 2.1: rho times opt.rho_kappa when r_p > opt.rho_tau r_d, divided by it when
 * r_d > opt.rho_tau r_p) with the floor max(opt.rho_min or mu_ref, 2 s*), s* the
 * smallest shift making L + s* I positive definite everywhere (found by bisection,
 * once per call); rho is then the starting penalty, and a large one is fine.  p_out
 * (host, same layout as p0) receives the final p and hist (host, 4 doubles per
 * iteration: r_p, r_d, sigma, rho) the history; either may be NULL.  Precision follows
 * opt.precision: RVE_FP64 runs every step in double; RVE_MIXED runs a float bulk
 * (fields, factor, FFTs and the fused step in float; spectrum weights, the Step 2'
 * root and the residual sums in double) until both residuals are within a few hundred
 * float roundings of their scale or stop improving, then converts p and g to double,
 * redoes the factor and Step 1' in double and continues in FP64 to tol; RVE_FP32 stops
 * after the float phase.  Models
 * RVE_NEOHOOKE and RVE_LINEAR.  The call keeps a device workspace of about
 * (48 d^2 + 8 d^2 (d^2 + 1) + 64 d) N^d bytes on the handle until rve_destroy.
 * Returns RVE_OK, RVE_E_NOT_CONVERGED (results valid), RVE_E_INVALID_ARG (k, rho,
 * p0, max_iter, model), RVE_E_STATE (no material, or no state yet),
 * RVE_E_NUMERICAL (L + rho I not positive definite somewhere, or Step 2' found no
 * root), RVE_E_OOM, RVE_E_CUDA. */
int rve_bloch(rve_t h, const int k[3], const double* p0, double rho, double tol, int max_iter, double* p_out,
              double* hist, rve_bloch_info* info);

/* Homogenised first Piola-Kirchhoff stress <W_F(F)> of the current state,
 * summed in double on the device (Section 2.3: <S> is the macroscopic stress);
 * <Lambda> for the incompressible LCE network. */
int rve_stress(rve_t h, double S[9]);

/* Mean of the multiplier field <Lambda> (equals <W_F(F)> at an exact local solve). */
int rve_mean_lambda(rve_t h, double L[9]);

/* Copy a field of the current state to/from host doubles in the layout above:
 * F, LAMBDA: d*d*N^d; U: d*N^d (the periodic part u~); N: 3*N^d (RVE_LCE).
 * rve_set_field makes the state non-fresh (it is the warm start of the next solve). */
int rve_get_field(rve_t h, int which, double* host_out);
int rve_set_field(rve_t h, int which, const double* host_in);

/* Mark the state fresh (the next solve starts from F = Fbar, u~ = 0). */
int rve_reset(rve_t h);

/* Residual history of the last solve: r_p, r_d and the rho used, per iteration
 * (up to cap entries).  Returns the number of entries written (>= 0) or an error. */
int rve_history(rve_t h, double* r_p, double* r_d, double* rho, int cap);

/* Local residual r_l of the same passes (local_ratio > 0, else zeros): entry i is
 * the local step fused with check i, i.e. Step 1 of iteration i + 2 (iterations
 * counted from 1).  Returns the number of entries written or an error. */
int rve_history_local(rve_t h, double* r_l, int cap);

/* ------------------------------------------------------------------ batches */
typedef struct rve_batch* rve_batch_t;

/* Group existing handles (each with its material set) for batched solves of
 * uneven RVEs.  Every per-iteration pass of all members runs as ONE persistent
 * kernel launch over a tile table spanning the members (per group of members
 * with the same model and dimension), and chunks of iterations are replayed as
 * CUDA graphs.  Members keep their own state, options and sizes; they must share
 * the precision mode and the rho policy.  A member's result is bitwise the same
 * as solving it alone with rve_solve (its blocks, partial sums and reductions
 * depend on its own size only).  The handles must outlive the batch and must not
 * be used by other calls during rve_batch_solve.  cuda_stream as in rve_create.
 * Allocates descriptors and tile tables with cudaMalloc.
 * Errors: RVE_E_INVALID_ARG (count < 1, null handle, duplicate handle, mixed
 * precision or rho policy), RVE_E_STATE (a member without material), RVE_E_OOM,
 * RVE_E_CUDA. */
int rve_batch_create(rve_batch_t* out, rve_t* handles, int count, void* cuda_stream);

/* Solve every member at its own Fbars[9*i .. 9*i+8] (row-major) and rhos[i] to
 * tol, as rve_solve does for one handle (same initialisation, warm start, stop
 * rule and precision phases).  Members finish independently; a finished member
 * leaves the tile tables.  infos (count entries, may be NULL) gets each member's
 * result.  Returns RVE_OK if every member converged, else the status of the first
 * member (in handle order) that did not. */
int rve_batch_solve(rve_batch_t b, const double* Fbars, const double* rhos, double tol, rve_solve_info* infos);

/* Release the batch (not its handles). */
void rve_batch_destroy(rve_batch_t b);

/* ------------------------------------------------------------------ serving */
typedef struct rve_server* rve_server_t;

/* A continuous-batching server for RVE solve requests of any size and model.
 * Requests are admitted, in arrival order, whenever the device workspaces of the
 * admitted requests fit mem_budget_bytes (rve_workspace_bytes with opt); idle
 * workspaces are kept by shape for reuse and released when memory is needed.
 * Admitted requests iterate together: each rve_server_step runs one chunk of
 * opt->check_every iterations of every admitted request as batched launches
 * (see rve_batch_create), retires the finished ones (homogenised stress and info
 * kept for rve_server_poll) and admits waiting requests into the freed memory,
 * so requests that arrive while others run join the running set.  A request's
 * result is bitwise the same as rve_solve of the same input on a fresh handle.
 * opt applies to every request (NULL = defaults).  The server is driven by one
 * host thread. */
int rve_server_create(rve_server_t* out, size_t mem_budget_bytes, const rve_options* opt, void* cuda_stream);

/* Queue a solve: a fresh state on an N^d cell (inputs as rve_create /
 * rve_set_material / rve_solve; host arrays are copied).  *ticket identifies it.
 * Errors: RVE_E_INVALID_ARG (shape, phase ids, rho, tol, or a non-finite Fbar or
 * det Fbar <= 0, checked here as rve_solve does), RVE_E_OOM (its workspace
 * exceeds the budget).  Material parameters are checked when the request is
 * admitted: a request rve_set_material rejects ends by itself with
 * RVE_E_INVALID_ARG (NaN stress) and the server carries on. */
int rve_server_submit(rve_server_t s, int dim, int n, int model, const uint8_t* phase, int nphase,
                      const double* params, int nparam, const double* n0, const double Fbar[9], double rho,
                      double tol, long long* ticket);

/* One scheduler tick (admit, iterate one chunk, retire); active/queued counts out. */
int rve_server_step(rve_server_t s, int* active_out, int* queued_out);

/* Result of a finished request: RVE_OK (or its non-OK solve status) with S (3x3,
 * row-major), info (info.time_ms = admission to completion), latency (submit to
 * completion) and queue wait in milliseconds; the result is then forgotten.
 * RVE_E_BUSY while queued or running, RVE_E_NOT_FOUND for unknown tickets. */
int rve_server_poll(rve_server_t s, long long ticket, double S[9], rve_solve_info* info, double* latency_ms,
                    double* queue_ms);

/* Drop a queued or running request (its workspace returns to the pool). */
int rve_server_cancel(rve_server_t s, long long ticket);

/* Queue length, running requests, completed requests, workspace bytes held. */
int rve_server_stats(rve_server_t s, long long* queued, long long* active, long long* completed, size_t* bytes_used);

/* Release the server, its pooled and running workspaces. */
void rve_server_destroy(rve_server_t s);

/* ------------------------------------------------------------------ FFT autotuner */
/* Time candidate FFT geometries for N^d grids on the current device -- x-pass
 * lines per block with the order of the half-length radices, y/z tile width with
 * the order of the full-length radices -- in the arithmetic of the given precision
 * mode (double for RVE_FP64, float otherwise), and keep the fastest: every later
 * rve_create of that shape in this process uses it (handles created before keep
 * theirs).  If cache_path is not NULL, one JSON object is appended as a line
 * (JSON Lines): {"kind": "rve-fft-geometry", "dim", "n", "precision", "lpb", "tk64",
 * "tk32", "rad_half": [...], "rad_full": [...], "ms"}.
 * *best_ms (may be NULL) gets the tuned FFT time of one iteration.  Allocates a
 * scratch handle.  Returns RVE_OK or an error. */
int rve_autotune(int dim, int n, int precision, const char* cache_path, double* best_ms);

/* Register the geometries stored in a cache file written by rve_autotune (later
 * lines win; lines that are not valid geometries are skipped).  Returns the number
 * of lines loaded, or RVE_E_NOT_FOUND. */
int rve_autotune_load(const char* cache_path);

/* ------------------------------------------------------------------ profiling */
/* Kernel classes of the iteration (index into rve_kernel_times' arrays). */
enum rve_kernel_class {
    RVE_KCLASS_LOCAL = 0,       /* fused Step 3 + Step 4 partials + Step 1 (per iteration)   */
    RVE_KCLASS_LOCAL_FIRST = 1, /* Step 1 alone (start of a solve / precision phase)         */
    RVE_KCLASS_XFWD = 2,        /* divergence of F - Lambda/rho + forward x FFT (Step 2)     */
    RVE_KCLASS_FWD_Y = 3,       /* forward y FFT (3D)                                        */
    RVE_KCLASS_SOLVE = 4,       /* last-axis forward FFT, multiply by 1/|k|^2, inverse       */
    RVE_KCLASS_INV_Y = 5,       /* inverse y FFT (3D)                                        */
    RVE_KCLASS_XINV = 6,        /* inverse x FFT -> u~ (Step 2 result)                       */
    RVE_KCLASS_LOCAL_R = 7,     /* double polish (RVE_MIXED): fused local + float increment R */
    RVE_KCLASS_XFWD_INCR = 8,   /* divergence of R + forward x FFT (float)                   */
    RVE_KCLASS_XINV_INCR = 9,   /* inverse x FFT, u~_{k+1} = u~_k + P(R) in double           */
    RVE_KCLASS_COUNT = 10
};

/* on != 0: every kernel launch of later solves is bracketed by CUDA events on
 * the handle's stream (CUDA graphs are not used meanwhile) and its device time is
 * added to per-class totals, for iterations that ran before the stop flag.
 * Switching it (on or off) clears the totals. */
int rve_set_profiling(rve_t h, int on);

/* Copy the per-class totals for the double (fp64 != 0) or float kernels:
 * ms[c] summed milliseconds, launches[c] launch count, for c < RVE_KCLASS_COUNT.
 * cap is the length of both arrays (>= RVE_KCLASS_COUNT).  Returns the number
 * of classes written or RVE_E_INVALID_ARG. */
int rve_kernel_times(rve_t h, int fp64, double* ms, long long* launches, int cap);

/* ------------------------------------------------------------------ no-allocation variant */
/* <W_F(F)> (first Piola-Kirchhoff, row-major 3x3, zero outside the d x d block)
 * for callers that cannot allocate device memory: an application that owns all
 * device memory through its own pool and forbids further allocations, or a
 * latency-critical loop that must not call cudaMalloc/cudaFree because they may
 * synchronise the device.  The paper has no counterpart; this is a systems entry
 * point, with the same result as rve_stress on the same F.
 * Inputs, all DEVICE pointers owned by the caller: F_dev (d*d*N^d DOUBLES in the
 * component-major field layout above; a mixed-precision or float handle keeps F
 * as float, so widen that field to double before passing it), phase_dev (N^d
 * bytes, values < nphase), params_dev (nphase * nparam doubles, {mu, lam} first).
 * Output: S_dev (9 doubles, device).  model is RVE_NEOHOOKE or RVE_LINEAR.  n is
 * not held to the handle's grid rules (even, 2^a 3^b, <= 512): any n >= 2 with
 * N^d within the capacity below is accepted.  Work is queued on cuda_stream
 * (NULL = legacy default stream); the call returns without waiting for it, so
 * it can report an error found on the device only through S_dev: a phase id >=
 * nphase makes every entry NaN (the status is still RVE_OK) -- check S_dev for
 * NaN after synchronising.
 * Nothing is allocated: block partial sums go to a static device array of 2 MiB
 * (+256 B) that every GPU loading this library holds until exit, which limits
 * N^d to 16,777,216 voxels (256^3); larger sizes return RVE_E_INVALID_ARG.  The
 * first call on each device looks up that array's address (call it once before
 * any stream capture); the address is kept for the life of the process, so do
 * not use this entry point after cudaDeviceReset on that device.  All calls
 * share the array and clear its header on entry: calls whose work overlaps on
 * the GPU race, so serialise them (e.g. one stream). */
int rve_stress_noalloc(int dim, int n, int model, const double* F_dev, const uint8_t* phase_dev,
                       const double* params_dev, int nphase, int nparam, double* S_dev, void* cuda_stream);

/* Human-readable name of a status code (static string). */
const char* rve_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* RVE_H */
