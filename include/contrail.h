/*
 * contrail.h -- C ABI of the GB300 contrail finite-volume library.
 *
 * The library advances the explicit finite-volume time step of the paper "Non-Equilibrium
 * Phase Changes in Aircraft Exhaust" (Tegethoff & Wheeler, arXiv 2504.20742): the
 * compressible multi-component axisymmetric (or quasi-1D nozzle) flow of Sec. 3.1,
 * Eqs. (22)-(26), with moment transport of droplets, ice and soot, coupled to the
 * per-cell non-equilibrium phase-change sources of Sec. 2.2, Eqs. (1)-(21), integrated by
 * the second-order explicit Runge-Kutta scheme with a global CFL number and sources in
 * every stage (Sec. 3.2).
 *
 * Conventions
 *   - Every call returns ct_status; none aborts.  On error, ct_last_error() returns a
 *     thread-local message.  CT_ERR_CUDA also reports asynchronous launch errors seen at
 *     the call.
 *   - Device pointers are allocated by the caller (e.g. by PyTorch) and borrowed for
 *     the duration of the call and of the work it enqueues; the library allocates no
 *     device memory.  Host pointers are borrowed for the duration of the call only.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device work is
 *     stream-ordered; calls that return host data synchronise that stream.
 *   - State layout: structure of arrays, U[f*N + j*nx + i], N = nx*nr (nr = 1 for the
 *     nozzle), 14 fields f:
 *        0 rho, 1 rho*u, 2 rho*v, 3 rho*E, 4 rho*Y_v,
 *        5..8  rho*mu_k(liquid)/(1 um)^k, 9..12 rho*mu_k(ice)/(1 um)^k, 13 rho*n_soot
 *     in SI units; mu_k are specific moments (per kg of mixture, Eq. (26)).  A case with
 *     the bimodal liquid (ct_case.bimodal = 1) has 18 fields: 5..8 then hold the droplets
 *     of homogeneous origin and 14..17 rho*mu_k/(1 um)^k of those of heterogeneous origin.
 *     Element type: double for CT_FP64, float for CT_FP32 and CT_FP32_MLP.
 */
#ifndef CONTRAIL_H
#define CONTRAIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CT_NFIELDS 14
#define CT_NFIELDS_BIMODAL 18
#define CT_NDIAG 32
#define CT_NAUX 11
#define CT_MLP_IN 16       /* surrogate inputs */
#define CT_MLP_HIDDEN 128  /* width of its 4 hidden SiLU layers */
#define CT_MLP_OUT 10      /* surrogate outputs */

typedef enum {
  CT_OK = 0,
  CT_ERR_ARG = 1,        /* invalid argument or size */
  CT_ERR_CUDA = 2,       /* a CUDA runtime call or launch failed */
  CT_ERR_NONFINITE = 3,  /* the last step produced a non-finite value */
  CT_ERR_TIMEOUT = 4,    /* a bounded device wait gave up */
  CT_ERR_STATE = 5,      /* call out of order (e.g. step before setup) */
  CT_ERR_SIZE = 6        /* workspace or scratch too small */
} ct_status;

typedef enum { CT_FP64 = 0, CT_FP32 = 1, CT_FP32_MLP = 2 } ct_precision;

/* One plume or nozzle case.  Geometry and boundary conditions follow Sec. 4.1 of the
 * paper, reduced to a single-velocity mixture: geom 0 is the quasi-1D nozzle with area
 * law A/A_t = 1 + area_a (x/x_throat - 1)^2; geom 1 the axisymmetric domain [0,lx]x[0,lr]
 * with a core (r < d_core/2), bypass (r < d_fan/2) and ambient coflow inflow profile at
 * ambient static pressure, an outflow at x = lx, a far field at r = lr and the axis at
 * r = 0.  All quantities SI. */
typedef struct {
  int32_t geom;          /* 0 quasi-1D nozzle, 1 axisymmetric plume */
  int32_t nx, nr;        /* cells (nr ignored for geom 0) */
  int32_t bc_xlo;        /* 0 inflow profile (plume) / total-condition inlet (nozzle), 1 wall */
  int32_t bc_xhi;        /* 0 outflow (zero gradient), 1 wall */
  int32_t bc_rhi;        /* 0 far field (ambient), 1 wall, 2 outflow */
  int32_t phase_change;  /* 0: all phase-change sources off */
  int32_t freezing;      /* 0: no freezing */
  double lx, lr;
  double area_a, x_throat;
  double d_core, d_fan, wall_len;          /* wall_len > 0: duct wall at r = d_fan/2, x < wall_len */
  double T_amb, p_amb, S_ice_amb, mach_coflow;
  double T_core, u_core, Yv_core, T_byp, u_byp;
  double n_soot, soot_rm, soot_sigma;      /* exit soot per m^3; lognormal median, sigma_g */
  double p0, T0, Yv_inlet;                 /* nozzle inlet total conditions */
  double seed_l_n, seed_l_r, seed_s_n, seed_s_r; /* initial monodisperse populations in the core */
  double mix_width;                        /* > 0: core blends into ambient over this width */
  double nu_t;                             /* turbulent kinematic viscosity, m^2/s (viscous = 1) */
  int32_t viscous;                         /* 1: viscous and diffusive fluxes, Eqs. (25)-(26) */
  int32_t tables;                          /* 1: water properties from tables, 2nd-order Taylor */
  int32_t equilibrium;                     /* 1: equilibrium phase change (not with CT_FP32_MLP) */
  int32_t bimodal;                         /* 1: two liquid moment sets, 18-field state (see below) */
} ct_case;

/* Optional parts of the model, each off by default:
 *   viscous = 1      viscous and diffusive fluxes (Sec. 3.1 Eqs. (25)-(26), central
 *                    differences of Sec. 3.2) with effective viscosity mu(T) + rho nu_t,
 *                    conductivity mu c_p/Pr + rho c_p nu_t/0.9, vapour diffusivity
 *                    2.11e-5 (T/273.15)^1.94 (101325/p) + nu_t/0.7 and particle diffusivity
 *                    nu_t/0.7 (m^2/s); walls are adiabatic, impermeable and slip.
 *   tables = 1       ln p_sat (liquid, ice) and the surface tension from tables every 0.5 K
 *                    (150-640 K) with a second-order Taylor expansion about the nearest node
 *                    (Sec. 3.2).  The tables are built once per device on the first call
 *                    that needs them, which synchronises the device: make that call before
 *                    any stream capture.
 *   equilibrium = 1  equilibrium phase change instead of the kinetic model (the comparison
 *                    of Sec. 4.3): every stage leaves each cell's water at saturation over
 *                    its condensate (liquid above 235.15 K, ice below, 1 um monodisperse).
 *   bimodal = 1      the bimodal liquid of Sec. 2.2: one moment set per nucleation
 *                    mechanism, so that spontaneously nucleated and soot-activated droplets
 *                    keep their own size histories (the two-peaked spectrum of Sec. 4.3).
 *                    Homogeneous nucleation feeds fields 5..8, heterogeneous nucleation the
 *                    extra fields 14..17; each set grows at its own r20; only droplets of
 *                    heterogeneous origin freeze by immersion (they hold the soot).  Every
 *                    state buffer then has CT_NFIELDS_BIMODAL planes.  Not with CT_FP32_MLP
 *                    (the surrogate was trained on one set) nor with equilibrium = 1. */

/* Diagnostics record of the last completed step (CT_NDIAG doubles):
 *   0 dt of the step, 1 total mass, 2 total water (vapour + liquid + ice), 3 total energy
 *   (volume integrals per radian for geom 1, per unit throat area for geom 0),
 *   4..6 mass, water and energy that entered through the boundary during the step
 *   (RK2 rule), 7 active cells in stage 2, 8 non-finite values, 9..22 max-norm of
 *   (U^{n+1}-U^n)/dt per field (bimodal: fields 14..17 share the slots of 5..8, the larger
 *   of the two), 23 max log10 J_hom, 24 max log10 J_het (m^-3 s^-1),
 *   25 dt of the next step, 26 surrogate fallback cells (CT_FP32_MLP), 27 steps taken,
 *   28 tensor-core waits that gave up in either stage (CT_FP32_MLP; ct_diagnostics then
 *   returns CT_ERR_TIMEOUT). */

/* Bytes of device workspace needed by a case at a precision (boundary states, reduction
 * partials, time step and diagnostics; for CT_FP64 without the bimodal liquid also the
 * primitive variables of U and U1 with the temperature and c_v, 2 x 16 x N doubles, which
 * each stage writes for the next one so that no cell is converted twice; for CT_FP32_MLP on
 * an inviscid axisymmetric case also the surrogate queue of the column-sweep step, a cell
 * index and 14 floats per cell plus 4096 reduction records, about 60 bytes per cell).
 * Returns 0 for an invalid case. */
size_t ct_workspace_bytes(const ct_case *c, int precision);

/* Validate the case and prepare the workspace: inflow profile per row (row velocity
 * factors ufac_rows_host[nr], host, may be NULL = all 1), ambient state, counters.
 * Must precede every other call on that workspace.  Enqueued on `stream`. */
ct_status ct_setup(const ct_case *c, int precision, const double *ufac_rows_host, void *work,
                   size_t work_bytes, void *stream);

/* Initial state into U (device, CT_NFIELDS*N elements of the precision's type): the plume
 * inflow profile extended over the domain (with the optional seed populations), or the
 * isentropic area-Mach solution of the nozzle.  Also computes the first time step for
 * `cfl`.  Enqueued on `stream`. */
ct_status ct_init_state(const ct_case *c, int precision, void *work, void *U, double cfl,
                        void *stream);

/* Load a caller-provided state (device, same layout and type as U) and compute its time
 * step for `cfl`: use after ct_setup to start from a checkpoint. */
ct_status ct_load_state(const ct_case *c, int precision, void *work, const void *U_src, void *U,
                        double cfl, void *stream);

/* Advance U by nsteps explicit SSP-RK2 steps (Sec. 3.2) with the global CFL number `cfl`.
 * U1 is a stage buffer of the same size.  The time step of each step is the CFL limit
 * of the state at its start, computed on the device; no host synchronisation happens.
 * Enqueued on `stream`.  The workspace carries the time step (and, in CT_FP64, the
 * primitive variables) of the state the last call left in U: after writing U by other
 * means, call ct_load_state before stepping again. */
ct_status ct_step(const ct_case *c, int precision, void *U, void *U1, void *work, int nsteps,
                  double cfl, void *stream);

/* End-to-end variant with host buffers: copies U_host_in (pinned or pageable host memory,
 * state layout, precision's type) to U, computes its time step, advances nsteps and copies
 * the result to U_host_out; synchronises `stream`.  U, U1 and work (after ct_setup) are
 * caller-provided device memory. */
ct_status ct_step_host(const ct_case *c, int precision, const void *U_host_in, void *U_host_out,
                       void *U, void *U1, void *work, int nsteps, double cfl, void *stream);

/* Copy the diagnostics record of the last step (nout <= CT_NDIAG doubles) to host memory;
 * synchronises `stream`.  Returns CT_ERR_NONFINITE when that step produced a non-finite
 * value (the record and the state stay readable). */
ct_status ct_diagnostics(const void *work, double *host_out, int nout, void *stream);

/* Per-cell derived quantity of state U into out (device, N doubles): which =
 * 0 T, 1 p, 2 ln S_l, 3 ln S_i, 4 log10 J_hom, 5 log10 J_het,eff, 6 active flag,
 * 7 r_crit, 8 Kantrowitz phi, 9 G_l(r20), 10 G_s(r20), 11 Koop log10 J_s (cm^-3 s^-1),
 * 12 per-droplet freezing rate omega, 13/14 median radius (um) and geometric standard
 * deviation of the lognormal liquid spectrum with the cell's mu0, mu1, mu2 (the droplet
 * spectra of Sec. 4.3), 15/16 the same for ice, 17/18 the same for the droplets of
 * heterogeneous origin (bimodal cases; 0 otherwise).  With the bimodal liquid, 9 and 12 and
 * 13/14 describe the droplets of homogeneous origin.  Non-applicable values are -inf (logs) or 0.
 * dt enters only the limiters. */
ct_status ct_derived(const ct_case *c, int precision, const void *U, int which, double dt,
                     double *out, void *stream);

/* Copy field `field` (0 .. nf-1, the SoA order of the state) of the state U (device, the
 * precision's type, nf x nr x nx) into host_dst (host, n = nx * nr doubles, x fastest),
 * converting FP32 states to FP64 on the host.  Synchronises `stream` (the copy follows the
 * work already queued on it).  The fields are the conserved variables of Sec. 3.1 (Eqs.
 * 22-26): rho, rho u, rho v, rho E, rho Y_v, then the moments rho mu_k of the liquid, the
 * ice and the soot number (scaled as stated above).  Errors: CT_ERR_ARG for a bad field,
 * size or pointer; CT_ERR_CUDA if the copy fails. */
ct_status ct_read_field(const ct_case *c, int precision, const void *U, int field, double *host_dst, size_t n,
                        void *stream);

/* Phase-change source (Sec. 2.2) of n independent cells: U (device, n x nf doubles,
 * row-major conserved states, nf = CT_NFIELDS_BIMODAL for a bimodal case, else CT_NFIELDS)
 * -> Q (device, n x nf) and aux (device,
 * n x CT_NAUX: ln S_l, ln S_i, ln J_hom, ln J_het,eff, active, r_crit, phi, G_l, G_s,
 * Koop log10 J_s, omega), evaluated at the given precision with limiters of step dt. */
ct_status ct_source_batch(const ct_case *c, int precision, const double *U, int n, double dt,
                          double *Q, double *aux, void *stream);

/* MUSCL reconstruction with the van Leer limiter (Sec. 3.2), the step the FP64 stage kernels
 * take for every field, cell and direction, here for n independent cells.  From the values
 * am (minus-side neighbour), a0 (the cell) and a1 (plus-side neighbour) it forms the states
 * of the cell's two faces, lo = a0 - hs and hi = a0 + hs, where hs = dm dp / (dm + dp) with
 * dm = a0 - am and dp = a1 - a0 where dm dp > 0, and hs = 0 (hi = a0 + 0) otherwise.  The
 * arithmetic and the decisions are the stage kernels' own: the reciprocal by Newton
 * iteration (valid while dm + dp is finite and normal) and the tests on the integer pipe.
 * All arrays are device arrays of n doubles; the call enqueues on `stream`.  n = 0 does
 * nothing; n < 0 or a null array gives CT_ERR_ARG. */
ct_status ct_reconstruct_faces(const double *am, const double *a0, const double *a1, int n, double *lo,
                               double *hi, void *stream);

/* ---- source surrogate (Sec. 2.2 rates; the network is this library's, not the paper's) ----
 * A 16 -> 4x128 (SiLU) -> 10 multilayer perceptron stands in for the stiff pointwise rates
 * of Sec. 2.2 (nucleation Eqs. 3-6/10, growth Eq. 16, the stage relaxation rates) in the
 * FP32 path.  Parameters: one flat FP32 vector, per layer W (out x in, row-major) then b.
 * All pointers below are device pointers; all calls enqueue on `stream`. */

/* Inputs X (n x CT_MLP_IN), targets Y and masks M (n x CT_MLP_OUT, mask 0 where a target is
 * undefined, e.g. nucleation below liquid saturation) of n conserved states U (n x 14
 * doubles, row-major), computed with the FP64 plain source of the case's physics.
 * Inputs: ln p, T, 1/max(ln S_l, 1/4)^2 (the CNT barrier shape), ln Y_v, ln of the 8
 * scaled moments, ln soot per m^3, ln <r_p^2>/um^2, ln S_l, ln S_i.  Targets: ln J/(1+phi)
 * (floored at -30), ln r_crit/um,
 * asinh(G_l/1 um/s), asinh(G_s/1 um/s), ln of the two relaxation rates 1/tau, ln J_hom,
 * ln J_het,eff (floored), ln(1+phi), T_sat,l - T. */
ct_status ct_mlp_dataset(const ct_case *c, const double *U, int n, float *X, float *Y, float *M, void *stream);

/* Number of FP32 parameters of the network. */
int ct_mlp_param_count(void);

/* Bytes of device work memory needed by ct_mlp_forward / ct_mlp_loss_grad for n rows. */
size_t ct_mlp_work_bytes(int n);

/* FP32 forward pass: Y (n x CT_MLP_OUT) = net(X (n x CT_MLP_IN)); inputs and outputs in the
 * standardised units the network was trained in. */
ct_status ct_mlp_forward(const float *params, const float *X, int n, float *Y, void *work, size_t work_bytes,
                         void *stream);

/* Masked mean-squared error L = sum M (net(X) - Y)^2 / max(1, sum M) into loss (1 float) and
 * its gradient with respect to params into grad (overwritten). */
ct_status ct_mlp_loss_grad(const float *params, const float *X, const float *Y, const float *M, int n, float *grad,
                           float *loss, void *work, size_t work_bytes, void *stream);

/* The same loss and gradient with every GEMM (forward, input and weight gradients) on the
 * BF16 tensor cores (tcgen05, FP32 accumulation in TMEM; operands rounded to BF16 as they
 * are staged, FP32 master weights untouched); bias, SiLU, loss and bias gradients in FP32.
 * err_flag (device int) is set to 1 if a bounded tensor-core wait gave up. */
ct_status ct_mlp_loss_grad_tc(const float *params, const float *X, const float *Y, const float *M, int n, float *grad,
                              float *loss, int *err_flag, void *work, size_t work_bytes, void *stream);

/* One Adam step (bias-corrected, step >= 1) on nparam parameters. */
ct_status ct_mlp_adam(float *params, const float *grad, float *m, float *v, int nparam, float lr, float beta1,
                      float beta2, float eps, int step, void *stream);

/* Column statistics of X (n x d, optional mask M of the same shape): out (4 x d floats) =
 * mean, standard deviation, minimum, maximum. */
ct_status ct_mlp_colstats(const float *X, const float *M, int n, int d, float *out, void *stream);

/* In-place standardisation X = (X - mean)/sd, column-wise (sd <= 0 treated as 1). */
ct_status ct_mlp_standardize(float *X, int n, int d, const float *mean, const float *sd, void *stream);

/* Configuration of ct_train_surrogate. */
typedef struct {
  int epochs;          /* passes over the rows */
  int batch;           /* rows per Adam step (the last partial batch of an epoch is left out) */
  float lr, lr_final;  /* learning rate, cosine decay from lr to lr_final over all steps */
  float beta1, beta2, eps;   /* Adam */
  uint64_t seed;       /* per-epoch shuffles: Fisher-Yates from splitmix64 */
  int tensor_cores;    /* 1: BF16 tcgen05 GEMMs with FP32 accumulation and FP32 master weights */
  float out_weight[16];   /* weight of each output's squared error (first CT_MLP_OUT; >= 0, not all 0) */
} ct_train_cfg;

/* Bytes of device workspace ct_train_surrogate needs for n rows (0 for invalid sizes). */
size_t ct_train_workspace_bytes(int n, int batch, int epochs);

/* Train the source surrogate (the paper has no network: it stands in for the rates of
 * Sec. 2.2) in one call: column statistics of X (inputs) and of Y over its mask M
 * (targets, 0 or 1), standardisation, then epochs of shuffled mini-batches, the masked MSE
 * with the per-output weights of cfg and its
 * gradient (ct_mlp_loss_grad, or ct_mlp_loss_grad_tc with tensor_cores) and Adam with the
 * cosine learning-rate schedule.
 * X (n x CT_MLP_IN), Y and M (n x CT_MLP_OUT): device, raw units (ct_mlp_dataset).
 * params: device, ct_mlp_param_count() floats, in: initial weights, out: trained weights
 * (standardised units).  stats: device, 4 x CT_MLP_IN then 4 x CT_MLP_OUT floats out (mean,
 * sd, min, max of the inputs and of the masked targets; sd below 1e-6 stored as 1), the
 * arguments ct_mlp_pack takes.  loss_hist: host, epochs floats out (mean batch loss).
 * work: device, ct_train_workspace_bytes(n, batch, epochs).  Runs on `stream` and returns
 * after it has finished.  Errors: CT_ERR_ARG, CT_ERR_SIZE, CT_ERR_CUDA, CT_ERR_TIMEOUT (a
 * tensor-core wait gave up). */
ct_status ct_train_surrogate(const float *X, const float *Y, const float *M, int n, const ct_train_cfg *cfg,
                             float *params, float *stats, float *loss_hist, void *work, size_t work_bytes,
                             void *stream);

/* Bytes of the device blob of a packed surrogate (BF16 weights in tensor-core operand
 * order, FP32 biases, input/output standardisation and the training hull). */
size_t ct_mlp_blob_bytes(void);

/* Pack trained FP32 parameters and statistics (16-float device arrays: input mean, sd,
 * training-hull min and max; output mean, sd, min and max over the training targets, first
 * CT_MLP_OUT used) into blob (device, ct_mlp_blob_bytes(), 16-byte aligned).  The fused step
 * holds every network output to its training range. */
ct_status ct_mlp_pack(const float *params, const float *x_mean, const float *x_sd, const float *x_min,
                      const float *x_max, const float *y_mean, const float *y_sd, const float *y_min,
                      const float *y_max, void *blob, void *stream);

/* BF16 tensor-core inference (tcgen05, FP32 accumulation) of n raw input rows X
 * (n x CT_MLP_IN floats) into raw outputs Y (n x CT_MLP_OUT).  err_flag (device int) is set
 * to 1 if a bounded wait for the tensor cores timed out. */
ct_status ct_mlp_infer(const void *blob, const float *X, int n, float *Y, int *err_flag, void *stream);

/* Advance an FP32 state (CT_FP32_MLP) by nsteps SSP-RK2 steps like ct_step, with the
 * phase-change rates of active cells inside the surrogate's training hull taken from the
 * BF16 tensor-core network in `blob` (ct_mlp_pack) instead of the plain source (Sec. 2.2);
 * cells outside the hull use the plain source (counted in diagnostics slot 26).  The moment
 * assembly, freezing, limiters and water bookkeeping are the plain path's, so conservation
 * is unaffected.  U, U1, work as for ct_step (workspace set up with CT_FP32_MLP: with the
 * column-sweep tile shape the stage kernel queues the cells its source screen keeps in the
 * workspace, and a second kernel per stage runs the network on them).  Every tile shape
 * gives the same state bit for bit. */
ct_status ct_step_surrogate(const ct_case *c, void *U, void *U1, void *work, const void *blob, int nsteps, double cfl,
                            void *stream);

/* Maximum scratch of ct_step_static, in bytes (6 MiB).  A case needs ct_workspace_bytes(c,
 * CT_FP32) bytes: a 1 KB header, the inflow profile (nr x fields doubles) and 27 doubles of
 * reduction record per tile, counted for the tile shape with the most tiles on the grid (the
 * 16 x 12 shape: 22,016 tiles on a 4096 x 1024 plume, 4.9 MB in all).  So every grid up to
 * 4096 x 1024 cells fits; an 8192 x 2048 plume (88,064 tiles) does not. */
#define CT_STATIC_SCRATCH_BYTES (6u << 20)

/* Allocation-free variant of ct_step.  The paper has no counterpart: this serves callers
 * that cannot allocate device memory (a host framework whose allocator they may not call,
 * a launcher that owns only the buffers it was handed, a process under a fixed memory
 * budget).  Instead of a caller workspace, the step's scratch (inflow profile, time step,
 * reduction partials, diagnostics) lives in one statically allocated device array of
 * CT_STATIC_SCRATCH_BYTES that every GPU loading the library holds until exit.
 * Arguments: ufac_rows_dev (device, nr doubles of inlet velocity factors, or NULL = all 1);
 * U (device, in/out state, precision's type); U1 (device, same size, receives the
 * first-stage state of the last step).  Each call prepares the scratch from the case,
 * computes the time step of U and advances nsteps SSP-RK2 steps on `stream`,
 * asynchronously; it calls no cudaMalloc or cudaFree and no allocating library routine.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current: make it before any stream capture.  All calls share the one
 * array and it keeps the last call's contents, so calls that overlap on the GPU (other
 * streams, other threads) race.  The device address found on the first call stays cached
 * for the process: after cudaDeviceReset() on a device, later calls on that device are
 * invalid (the module, and the array with it, may move).  The step's diagnostics record
 * (totals, time step, non-finite count) stays in the static array and no call returns it,
 * so this path does not report CT_ERR_NONFINITE: a caller that needs that check reads the
 * state it owns.  Errors: CT_ERR_SIZE when the case needs more scratch than
 * CT_STATIC_SCRATCH_BYTES; CT_ERR_ARG for invalid arguments (CT_FP32_MLP is rejected). */
ct_status ct_step_static(const ct_case *c, int precision, const double *ufac_rows_dev, void *U, void *U1,
                         int nsteps, double cfl, void *stream);

/* ---- tile shapes and the autotuner (no counterpart in the paper) -----------------------
 * The fused stage kernel is built for several tile shapes (cells per CTA); the state a step
 * produces does not depend on the shape, only the speed does.  Steps of a case use the
 * shape registered for its (geometry, nx, nr, precision), else shape 0 (32 x 8). */

/* Number of tile shapes the library is built with. */
int ct_tile_shape_count(void);

/* Cells per tile of shape `shape` in x and r. */
ct_status ct_tile_shape(int shape, int *tx, int *ty);

/* CTAs per SM that the registers of shape `shape`'s kernels at `precision` are budgeted for
 * (more CTAs: more resident warps to hide latency, fewer registers per thread); 0 when the
 * shape has no kernels at that precision.  Some shapes carry one precision only: 32 x 8 and
 * 16 x 16 with three FP32 CTAs per SM, 16 x 12 and 16 x 16 with two FP64 CTAs per SM. */
int ct_tile_shape_ctas(int shape, int precision);

/* Register `shape` for cases with this case's geometry, grid and precision (-1: back to the
 * default).  CT_ERR_ARG when the shape's kernel does not fit an SM at that precision. */
ct_status ct_set_tile_shape(const ct_case *c, int precision, int shape);

/* Autotuner: time `reps` first-stage launches of every available shape on state U (device,
 * left unchanged; U1 receives scratch results), with CUDA events on `stream`, register the
 * fastest for the case's grid and return it in shape_out (may be NULL).  ms_out (host,
 * ct_tile_shape_count() floats, may be NULL) receives ms per launch, -1 for shapes not
 * available.  work must be set up for the case; blob is needed for CT_FP32_MLP.
 * Synchronises `stream`. */
ct_status ct_autotune(const ct_case *c, int precision, const void *U, void *U1, void *work, const void *blob, int reps,
                      void *stream, int *shape_out, float *ms_out);

/* ---- batched step: many plume cases in one persistent, graph-captured launch ----------
 * A batch advances ncases independent axisymmetric cases (geom 1) of uneven grids and
 * conditions together.  Each step is two launches of a persistent kernel whose CTAs take
 * the tiles of all cases from one work list; every case keeps its own CFL time step and
 * diagnostics.  Batch state layout: the cases' states (each in the single-case layout)
 * one after another, case k starting at element nf * sum_{k' < k} nx_k' nr_k' (nf = 14, or
 * 18 when the cases are bimodal: all cases of a batch share the flag).  FP32 and FP32_MLP
 * only. */
typedef struct ct_batch ct_batch;   /* host object: case table, tile shape, captured graph */

/* Device workspace bytes of a batch (0 for invalid cases). */
size_t ct_batch_workspace_bytes(const ct_case *cases, int ncases);

/* Elements of one batch state (sum over cases of nf nx nr). */
size_t ct_batch_state_elems(const ct_case *cases, int ncases);

/* Validate 1..96 cases, set up every case's part of `work` (device, 256-byte aligned,
 * ct_batch_workspace_bytes) with its inflow rows (ufac_rows_host: host, sum of nr doubles,
 * case after case, or NULL = all 1), and create the host object.  The batch's calls
 * enqueue on `stream`; the object owns a private stream used only for graph capture.
 * Synchronises `stream`. */
ct_status ct_batch_create(const ct_case *cases, int ncases, int precision, const double *ufac_rows_host, void *work,
                          size_t work_bytes, void *stream, ct_batch **out);

/* Free the host object (not the caller's device memory). */
void ct_batch_destroy(ct_batch *b);

/* Initial state of every case into U (device, batch layout, float) and their first time
 * steps, as ct_init_state. */
ct_status ct_batch_init_state(ct_batch *b, void *U, double cfl);

/* Copy the caller state U_src into U (may be equal) and compute every case's time step. */
ct_status ct_batch_load_state(ct_batch *b, const void *U_src, void *U, double cfl);

/* Use tile shape `shape` for the batch (the kernel's work list is rebuilt). */
ct_status ct_batch_set_tile_shape(ct_batch *b, int shape);

/* The batch's current tile shape. */
int ct_batch_tile_shape(const ct_batch *b);

/* Autotuner of the batched kernel: as ct_autotune, over the whole batch; leaves the
 * fastest shape set.  U is left unchanged, U1 receives scratch results. */
ct_status ct_batch_autotune(ct_batch *b, const void *U, void *U1, const void *blob, int reps, int *shape_out,
                            float *ms_out);

/* Advance every case of the batch by nsteps SSP-RK2 steps (Sec. 3.2), each with its own
 * CFL time step.  The first call with a given (U, U1, blob, nsteps, cfl, shape) captures
 * the 2 nsteps launches into a CUDA graph; later calls with the same arguments replay it
 * with one launch.  blob: packed surrogate for CT_FP32_MLP, else ignored. */
ct_status ct_batch_step(ct_batch *b, void *U, void *U1, const void *blob, int nsteps, double cfl);

/* Diagnostics records of the last step of every case (host, ncases x CT_NDIAG doubles);
 * synchronises the batch's stream.  CT_ERR_NONFINITE when any case produced non-finite
 * values. */
ct_status ct_batch_diagnostics(ct_batch *b, double *host_out);

/* Thread-local description of the last error. */
const char *ct_last_error(void);

/* Library version string. */
const char *ct_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CONTRAIL_H */
