/*
 * gsis.h -- C ABI of libgsis: the general synthetic iterative scheme (GSIS)
 * and plain source iteration (SI) for the steady gray radiative transfer
 * equation on one GPU (sm_103a).
 *
 * Problem (Sec. 2.1, Eq. (RTE_g) without time derivative and without the
 * material equation; Sec. 2.2, Eq. (RTE_SI) with hatted = plain cross sections):
 *
 *     Omega . grad I + sigma_t I = (sigma_s rho + q) / (4 pi),
 *     rho = integral of I over the sphere,   sigma_t = sigma_a + sigma_s,
 *
 * on a 2D Cartesian mesh, discretised by the cell-centred finite-volume
 * discrete-ordinate scheme of Sec. 4.1 (Eqs. (RTE_d), (Iij) with first-order
 * upwind faces), with prescribed intensity entering through the walls and
 * no reflection (Sec. 4.4, Eq. (micro_bc), alpha_w = 0).
 *
 * Conventions shared by every call:
 *   - cells are row-major: cell c = i + nx*j, i along x (0 <= i < nx);
 *   - boundary faces: W faces f = j, E faces f = ny + j, S faces
 *     f = 2*ny + i, N faces f = 2*ny + nx + i (n_bface = 2*(nx+ny));
 *   - q is the angle-integrated volumetric source (angular source q/4pi);
 *   - all floating point arguments are float64 (double);
 *   - "device" pointers are CUDA device (or managed) memory on the current
 *     device; "host" pointers are ordinary host memory;
 *   - every call that takes a stream is stream-ordered on that stream
 *     (cudaStream_t passed as void*, NULL = legacy default stream) and
 *     returns after its device work is enqueued, except where a call states
 *     that it synchronises;
 *   - the library never allocates device memory: scratch comes from the
 *     caller's workspace, sized by gsis_workspace_bytes();
 *   - inputs are never modified; outputs are written only on success or on
 *     GSIS_ERR_MAXITER / GSIS_ERR_STALLED (best iterate so far);
 *   - errors: a negative gsis_status is returned, nothing is thrown and the
 *     process never exits; gsis_last_error() gives a per-thread message.
 */
#ifndef GSIS_H
#define GSIS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GSIS_OK = 0,
    GSIS_ERR_ARG = -1,             /* invalid argument (sizes, NULL, sigma < 0, sum w != 4pi, ...) */
    GSIS_ERR_CUDA = -2,            /* a CUDA runtime call failed (message in gsis_last_error) */
    GSIS_ERR_MAXITER = -3,         /* max_iter reached without Err < tol (outputs = last iterate) */
    GSIS_ERR_DIVERGED = -4,        /* Err became NaN/Inf or exceeded 1e6 */
    GSIS_ERR_STALLED = -5,         /* Err did not decrease for `stall_window` checks */
    GSIS_ERR_DEVICE_TIMEOUT = -6,  /* a bounded device-side wait gave up; results invalid */
    GSIS_ERR_WORKSPACE = -7        /* workspace NULL, too small or misaligned (256 B) */
} gsis_status;

typedef enum { GSIS_SCHEME_SI = 0, GSIS_SCHEME_GSIS = 1 } gsis_scheme;

/* GSIS_FP64: everything in float64.
 * GSIS_FP32_SWEEP: the transport sweep and its angular-moment sums run in
 * float32 (float32 accumulators); the high-order terms, the synthetic solve,
 * Err and all residual norms stay float64. */
typedef enum { GSIS_FP64 = 0, GSIS_FP32_SWEEP = 1 } gsis_precision;

/* Mesh: nx*ny cells; dx[nx], dy[ny] are HOST arrays of positive widths,
 * copied during the call. */
typedef struct {
    int nx, ny;
    const double* dx;
    const double* dy;
} gsis_mesh;

/* Discrete ordinates (Sec. 4.1): K directions with x/y cosines mu[k],
 * eta[k] (mu^2 + eta^2 <= 1) and weights w[k] > 0 with sum w = 4 pi
 * (checked to 1e-10 relative).  HOST arrays, copied during the call. */
typedef struct {
    int K;
    const double* mu;
    const double* eta;
    const double* w;
} gsis_quadrature;

typedef struct {
    int scheme;            /* gsis_scheme */
    int precision;         /* gsis_precision */
    double tol;            /* stop when Err(rho) < tol (Eq. (Err_W)); default 1e-8 */
    int max_iter;          /* iteration cap; default 100000 */
    int fixed_iters;       /* > 0: run exactly this many iterations, ignore tol */
    double synth_rtol;     /* synthetic solve: stop at ||b - D rho|| <= synth_rtol ||b||; default 1e-12 */
    int synth_max_iter;    /* synthetic solve iteration cap; default 20000 */
    double cfl_p;          /* global pseudo-time control CFL_p (Eq. (cfl_pse)); <= 0: off (default) */
    double beta;           /* local pseudo-time control beta (Eq. (tau_pse)); <= 0: off (default) */
    int check_every;       /* iterations between host reads of the device status; default 16 */
    int stall_window;      /* GSIS_ERR_STALLED after this many checks without a new minimum of Err; 0 = off */
    double wait_limit_s;   /* bound of every device-side wait, seconds; default 2.0 */
    int spatial_order;     /* face values of the kinetic step: 1 = first-order upwind (default),
                              2 = second-order upwind (Eqs. (Ii,k), (Iij)) solved in the delta
                              form of Eqs. (RTE_d_increment), (RTE_d_res), (RTE_d_mtx): UW2
                              residual, first-order upwind increment sweep; gsis_solve only */
    int limiter;           /* spatial_order 2: 0 = Barth-Jespersen (the paper's, default),
                              1 = none (unlimited reconstruction) */
} gsis_options;

/* Fills *opt with the defaults listed above (scheme GSIS, precision FP64). */
void gsis_default_options(gsis_options* opt);

/*
 * Level-symmetric S_order discrete-ordinate set for 2D (Sec. 4.1 names S_n
 * sets; the points follow mu_i^2 = mu_1^2 + (i-1) 2(1 - 3 mu_1^2)/(order-2),
 * weights from the even moment conditions; the z > 0 hemisphere is kept with
 * doubled weights).  order in {4,6,...,16}; K = order(order+2)/2.
 * mu, eta, w: HOST arrays of capacity >= K, or all NULL to query *K only.
 * Directions are grouped by quadrant (+,+), (-,+), (+,-), (-,-).
 * Returns GSIS_OK or GSIS_ERR_ARG.
 */
int gsis_quadrature_level_symmetric(int order, double* mu, double* eta, double* w, int* K);

/* Bytes of device workspace needed by gsis_solve / gsis_transport_sweep /
 * gsis_synthetic_step for this mesh, quadrature and options (the maximum
 * over the three).  Returns GSIS_OK or GSIS_ERR_ARG. */
int gsis_workspace_bytes(const gsis_mesh* mesh, const gsis_quadrature* quad,
                         const gsis_options* opt, size_t* bytes);

/*
 * Solve the steady problem by SI (Sec. 2.2, Eq. (SI_update)) or GSIS
 * (Sec. 3.1, Eqs. (GSIS_HoT), (GSIS_M0), (GSIS_update), discretised as in
 * Secs. 4.2-4.4 and 5), starting from rho^0 = 0, until Err(rho) < tol.
 *
 * sigma_a, sigma_s, q: device [N] (N = nx*ny), sigma_a >= 0, sigma_s >= 0,
 *   sigma_a + sigma_s > 0.
 * inflow: device [n_bface * K] (face-major: inflow[f*K + k]) intensity
 *   entering through boundary face f in direction k (read only where
 *   Omega_k . n_f < 0), or NULL for vacuum walls.
 * rho: device [N] out, energy density rho^{m+1}.
 * F: device [2N] out (F_x block then F_y block), first moment of I^{m+1}.
 * P: device [3N] out (P_xx, P_xy, P_yy blocks), second moment of I^{m+1}
 *   (for GSIS the isotropic correction of Eq. (GSIS_update) adds
 *   (rho^{m+1} - rho^{m+1/2})/3 to P_xx and P_yy), or NULL.
 * history: HOST [max_iter] out, Err after each iteration, or NULL.
 * iters_out, err_out: HOST out (may be NULL): iterations done, final Err.
 * workspace: device, >= gsis_workspace_bytes(), 256-byte aligned, owned by
 *   the caller and not used concurrently by another call.
 * This call SYNCHRONISES the stream (it reads the convergence status back
 * every opt->check_every iterations).
 * Returns GSIS_OK, GSIS_ERR_MAXITER, GSIS_ERR_DIVERGED, GSIS_ERR_STALLED,
 * GSIS_ERR_DEVICE_TIMEOUT, GSIS_ERR_ARG, GSIS_ERR_WORKSPACE or GSIS_ERR_CUDA.
 */
int gsis_solve(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
               const double* sigma_a, const double* sigma_s, const double* q,
               const double* inflow, double* rho, double* F, double* P,
               double* history, int* iters_out, double* err_out,
               void* workspace, size_t workspace_bytes, void* stream);

/*
 * One kinetic step (Sec. 4.1; Eq. (RTE_SI) with source S = (sigma_s rho_in + q)/4pi):
 * the exact first-order-upwind sweep of every ordinate and its angular
 * moments (Eqs. (def_rho), (def_F), (RTE_M0)) plus the kinetic net flux
 * F_iw . n of every boundary face (Sec. 4.4, F_iw^init).
 * rho_in: device [N].  rho_half: device [N] out.  F_half: device [2N] out.
 * P_half: device [3N] out or NULL.  bflux: device [n_bface] out or NULL
 * (outward normal component, sum_k w_k (Omega_k . n) I_face,k).
 * opt: only opt->precision and opt->wait_limit_s are read (no pseudo-time).
 * Stream-ordered; does not synchronise.
 */
int gsis_transport_sweep(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                         const double* sigma_a, const double* sigma_s, const double* q,
                         const double* inflow, const double* rho_in,
                         double* rho_half, double* F_half, double* P_half, double* bflux,
                         void* workspace, size_t workspace_bytes, void* stream);

/*
 * One synthetic step of GSIS (Sec. 3.1 and 4.2): adaptive least-squares
 * gradient of rho_half (Sec. 5.2, Eqs. (shifted_j), (new_vector), (LSF_mdf)),
 * high-order terms HoT = F_half + grad(rho_half)/(3 sigma_t) (Eq. (GSIS_HoT)),
 * right-hand side with face-averaged HoT (Eq. (Fij_d)) and the boundary flux
 * of Eqs. (macro_bc_delta_flux), (macro_bc_delta_flux2), and the solve of
 * the finite-volume synthetic equation (Eqs. (MSE_d1), (Gamma_ij_def),
 * (elem_mtx_M), (Gamma_ij_com2)) for rho_out, starting from rho_guess
 * (device [N], may alias nothing else, NULL = start from rho_half).
 * rho_half: device [N], F_half: device [2N], bflux: device [n_bface] in.
 * rho_out: device [N] out.  hot: device [2N] out or NULL.  rhs: device [N]
 * out or NULL (b of D rho = b, multiplied by the cell volume).
 * synth_iters_out: HOST out or NULL.  SYNCHRONISES the stream.
 */
int gsis_synthetic_step(const gsis_mesh* mesh, const gsis_options* opt,
                        const double* sigma_a, const double* sigma_s, const double* q,
                        const double* rho_half, const double* F_half, const double* bflux,
                        const double* rho_guess, double* rho_out, double* hot, double* rhs,
                        int* synth_iters_out,
                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * Bytes of device workspace needed by gsis_adjoint (the gsis_solve layout
 * plus the adjoint intensities and vectors).
 */
int gsis_adjoint_workspace_bytes(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                                 size_t* bytes);

/*
 * Gradient of a functional J(rho*) of the converged GSIS solution rho*
 * (Sec. 3.1, steady, no pseudo-time) with respect to the per-cell opacities,
 * by the adjoint of the GSIS fixed point.  The paper has no counterpart of
 * this call: it differentiates the discrete equations this library solves.
 *   The kinetic step at rho* (I_k = A_k^{-1} s, s = (sigma_s rho* + q)/4pi,
 *   Eqs. (RTE_d), (RTE_SI)) and the synthetic equation D rho* = b (Eqs.
 *   (MSE_d1), (Fij_d), (macro_bc_delta_flux), with the adaptive least-squares
 *   HoT, Eqs. (GSIS_HoT), (shifted_j), (new_vector), (LSF_mdf)) are held as
 *   constraints; the adjoint lam = D nu solves the transposed GSIS iteration
 *   lam = M^T lam + dJ/drho (one synthetic solve, the transposed right-hand
 *   side and one transposed sweep of every ordinate per iteration, iterated
 *   to opt->tol on Err(lam), Eq. (Err_W)); the gradient is the explicit
 *   derivative of the Lagrangian (kinetic source and diagonal, Gamma_f,
 *   boundary beta, HoT weights, V sigma_a).
 * rho_star: device [N], the converged solution of gsis_solve with the same
 *   mesh, quadrature, options and inputs (the kinetic step is retaken at it).
 * dJ_drho: device [N].  grad_sigma_a, grad_sigma_s: device [N] out.
 * iters_out, err_out: host, may be NULL (adjoint iterations, final Err(lam)).
 * Requirements (else GSIS_ERR_ARG): opt->scheme == GSIS_SCHEME_GSIS, no
 *   pseudo-time (opt->cfl_p, opt->beta <= 0), uniform dx and dy (the
 *   transposed upwind sweep is then the sweep of the reflected direction),
 *   a quadrature closed under Omega -> -Omega with equal weights.
 * opt->precision selects FP64 or FP32 transposed sweeps, as in gsis_solve.
 * opt->stall_window ends the iteration as in gsis_solve (the FP32 form has a
 *   floor of Err(lam) near 1e-7).
 * Workspace: gsis_adjoint_workspace_bytes.  Returns GSIS_OK, or
 *   GSIS_ERR_MAXITER / GSIS_ERR_STALLED / GSIS_ERR_DIVERGED for the adjoint
 *   iteration (the gradient is written in every case), or an
 *   argument, CUDA, timeout or workspace error.  Synchronises the stream.
 */
int gsis_adjoint(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                 const double* sigma_a, const double* sigma_s, const double* q, const double* inflow,
                 const double* rho_star, const double* dJ_drho, double* grad_sigma_a, double* grad_sigma_s,
                 int* iters_out, double* err_out, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Time-dependent gray radiation-material problem (Sec. 2.1, Eqs. (RTE_g),
 * (Tm_g), emission phi = a c T^4, isotropic scattering, q a fixed volume
 * source) by backward Euler (Sec. 4.1, Eq. (RTE_d)): nsteps steps of dt from
 * rho^0, T^0 with the isotropic initial intensity I^0 = rho^0 / 4pi.
 * Each step iterates, until Err(rho) < opt->tol (Eq. (Err_W)):
 *   opt->scheme == GSIS_SCHEME_GSIS: the kinetic step (1/(c dt) on the
 *     diagonal, I^n/(c dt) and sigma_a phi(T^m) in the source, Eqs.
 *     (RTE_g_semi), (RTE_d_res)) and the coupled rho-T synthetic system
 *     (Eqs. (GSIS_dse), (MSE_d), (Tm_d)), one Newton step about T^m per
 *     iteration with T eliminated cell by cell (its diagonal gains
 *     V (1/(c dt) + f sigma_a - sigma_a), f = (C_v/dt)/(C_v/dt + 4 a c T^3
 *     sigma_a)); at convergence the step is the implicit discrete solution;
 *   opt->scheme == GSIS_SCHEME_SI: source iteration with the Fleck-Cummings
 *     linearisation about T^n (Eqs. (Tm_semi_linear), (RTE_SI),
 *     (arti_sigmaT); mu = 1 - f with the factor 4 of the derivation).
 * The intensities of consecutive steps stay in the workspace (two K x N
 * arrays, FP32 with GSIS_FP32_SWEEP).
 */
typedef struct {
    double dt;      /* time step, > 0 */
    double c;       /* speed of light, > 0 */
    double a;       /* radiation constant, > 0 */
    double cv;      /* volumetric heat capacity C_v, > 0 */
    int nsteps;     /* backward-Euler steps, >= 1 */
    /* First iterate of each step's iteration: 0 = the previous step's result
     * (rho^n, T^n), as the paper's time loop starts it; 1 = linear, 2 =
     * quadratic extrapolation in time from the last two or three steps'
     * results (fewer steps so far: the highest order they allow), each value
     * kept >= half the previous step's (rho >= 0, T > 0).  Only the starting
     * point changes: every step still iterates to Err < tol, so the result
     * is the same implicit solution within the tolerance, in fewer
     * iterations on smooth transients.  gsis_td_adjoint keeps the history with
 * each checkpoint, so its recomputed steps repeat the forward run's. */
    int predictor;
} gsis_time_params;

/* Bytes of device workspace for gsis_td_solve (the gsis_solve layout plus the
 * previous step's intensities and fourteen per-cell arrays). */
int gsis_td_workspace_bytes(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                            size_t* bytes);

/*
 * sigma_a, sigma_s, q, inflow: as in gsis_solve (opacities do not depend on T).
 * rho0 (>= 0), T0 (> 0): device [N] initial state.  rho, T: device [N] out,
 * the state after the last step.  F: device [2N] out (first moment of the
 * last sweep) or NULL.  step_iters, step_err: HOST [nsteps] out or NULL,
 * inner iterations and final Err of every step.
 * opt: scheme, precision, tol / max_iter / fixed_iters per step, synthetic
 * controls, check_every, stall_window, wait_limit_s; pseudo-time must be off
 * (cfl_p, beta <= 0, else GSIS_ERR_ARG).  Synchronises the stream.
 * stall_window > 0 (without fixed_iters): a step whose Err has reached no new
 *   minimum for stall_window checks (of check_every iterations) ends there,
 *   at its floor, and the run goes on with the next step; step_err holds the
 *   floor reached.  FP32 sweeps stop near Err = 1e-8 on some steps.
 * Returns GSIS_OK when every step converged; GSIS_ERR_STALLED when every
 * step converged or stalled and at least one stalled (all nsteps were run;
 * rho, T hold the final state); GSIS_ERR_MAXITER or GSIS_ERR_DIVERGED when a
 * step did neither (the solve stops there and rho, T hold that step's last
 * iterate); argument, CUDA, timeout, workspace errors.
 */
int gsis_td_solve(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                  const gsis_time_params* tp, const double* sigma_a, const double* sigma_s, const double* q,
                  const double* inflow, const double* rho0, const double* T0, double* rho, double* T,
                  double* F, int* step_iters, double* step_err, void* workspace, size_t workspace_bytes,
                  void* stream);

/*
 * Gradient of J = dJ_drho . rho^N + dJ_dT . T^N, a functional of the state
 * after a time-dependent GSIS run (gsis_td_solve with GSIS_SCHEME_GSIS), with
 * respect to the per-cell opacities and the initial state, by the adjoint of
 * every backward-Euler step (reverse mode).  The paper has no counterpart of
 * this call: it differentiates the discrete equations gsis_td_solve solves.
 *   Step n's converged result is the fixed point of the kinetic step
 *   (Eqs. (RTE_g_semi), (RTE_d)), the synthetic balance (Eqs. (GSIS_dse),
 *   (MSE_d)) and the material equation (Eq. (Tm_d)); its adjoint, with T
 *   eliminated cell by cell, is a transposed GSIS iteration with the step's
 *   Newton-eliminated synthetic operator, the effective scattering
 *   sigma_s + (1 - f) sigma_a and the transposed sweep with 1/(c dt) on the
 *   diagonal, iterated to opt->tol on Err (Eq. (Err_W)) of the adjoint
 *   density; one more transposed sweep per step carries the adjoint of the
 *   intensities to the previous step.
 * Checkpointing: the forward run keeps the input state of every
 *   checkpoint_every-th step; the reverse pass recomputes one segment of
 *   checkpoint_every steps at a time from its checkpoint (one extra forward
 *   run in all) and keeps that segment's fixed points.  Device memory:
 *   ceil(nsteps / checkpoint_every) + checkpoint_every intensity arrays
 *   (K x N, FP32 with GSIS_FP32_SWEEP) on top of the solve's layout; the
 *   gradient does not depend on checkpoint_every (the recomputation repeats
 *   the same arithmetic).
 * Arguments as in gsis_td_solve; dJ_drho, dJ_dT: device [N] or NULL (zero).
 * rho, T: device [N] out or NULL, the state after the last step.
 * grad_sigma_a, grad_sigma_s: device [N] out.  grad_rho0, grad_T0: device
 * [N] out or NULL (the initial intensity is rho^0/4pi).  adj_iters: HOST
 * [nsteps] out or NULL, adjoint iterations of every step.
 * Requirements (else GSIS_ERR_ARG): opt->scheme == GSIS_SCHEME_GSIS, no
 *   pseudo-time, spatial_order 1, uniform dx and dy, a quadrature closed
 *   under Omega -> -Omega with equal weights, checkpoint_every >= 1.
 * Returns GSIS_OK; a forward step's or an adjoint step's status when one did
 * not converge (GSIS_ERR_MAXITER / GSIS_ERR_DIVERGED; the gradient is still
 * written unless a step diverged); argument, CUDA, timeout or workspace
 * errors.  Synchronises the stream.
 */
int gsis_td_adjoint_workspace_bytes(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                                    const gsis_time_params* tp, int checkpoint_every, size_t* bytes);
int gsis_td_adjoint(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                    const gsis_time_params* tp, int checkpoint_every, const double* sigma_a, const double* sigma_s,
                    const double* q, const double* inflow, const double* rho0, const double* T0,
                    const double* dJ_drho, const double* dJ_dT, double* rho, double* T, double* grad_sigma_a,
                    double* grad_sigma_s, double* grad_rho0, double* grad_T0, int* adj_iters, void* workspace,
                    size_t workspace_bytes, void* stream);

/*
 * Measured FP64 FMA rate of the current device in GFLOP/s (host out),
 * the denominator of the FP64-ALU-bound kernels' rooflines.  The paper has
 * no counterpart: a measurement helper.  One kernel of independent
 * dependent-FMA chains over 8 blocks of 256 threads per SM, best of three
 * timed launches (CUDA events on the stream) after one warm-up.  No device
 * memory is allocated.  Synchronises the stream.
 */
int gsis_measure_fp64_fma(double* gflops, void* stream);
/* The same for FP32 FMAs (32 times more iterations per thread). */
int gsis_measure_fp32_fma(double* gflops, void* stream);

/*
 * Batched solve: n independent steady problems, each with its own mesh,
 * quadrature, opacities, sources and inflow, iterated together under one set
 * of options.  The paper solves one problem at a time and has no counterpart
 * of this call: it is a throughput form of gsis_solve.  Each problem goes
 * through exactly the iteration of gsis_solve (Sec. 2.2 / Sec. 3.1, same
 * kernels, same order of operations): rho, F, the iteration count and Err
 * equal gsis_solve's bit for bit whenever the synthetic solver runs on the
 * cluster size gsis_solve picks (tuning->synth_cells_per_cta = 0), and agree
 * to the synthetic tolerance otherwise (its cluster-wide sums are then
 * rounded in another order).
 *
 * Per iteration every step is one launch over all problems: one persistent
 * sweep over the units (ordinate, 32-row band) of every problem, drawn in the
 * order tuning->sweep_order gives, one launch each for the moments and
 * boundary fluxes, the HoT and synthetic right-hand side, and the update, and
 * one strip-solver launch per cluster size (one cluster per problem; the
 * cluster sizes run concurrently).  opt->check_every iterations are captured
 * once as a CUDA graph and replayed; the host reads every problem's status
 * after each replay, and launches skip a problem once it has stopped
 * (converged, diverged, iteration cap, stalled).
 */
typedef struct {
    gsis_mesh mesh;             /* HOST spacing arrays, as in gsis_solve */
    gsis_quadrature quad;       /* HOST arrays, as in gsis_solve */
    const double* sigma_a;      /* device [N] */
    const double* sigma_s;      /* device [N] */
    const double* q;            /* device [N] */
    const double* inflow;       /* device [n_bface*K] or NULL (vacuum) */
    double* rho;                /* device [N] out */
    double* F;                  /* device [2N] out, or NULL */
    int iters;                  /* out: iterations done */
    double err;                 /* out: final Err(rho) */
    int status;                 /* out: the gsis_status gsis_solve would return for this problem */
} gsis_problem;

typedef enum {
    GSIS_ORDER_PROBLEM = 0,      /* problem after problem, in the given order */
    GSIS_ORDER_BAND = 1,         /* band 0 of every problem, then band 1, ... */
    GSIS_ORDER_LONGEST = 2,      /* problem after problem, longest sweep chain (bands x width) first */
    GSIS_ORDER_BAND_LONGEST = 3  /* band-major, longest chains first within a band */
} gsis_sweep_order;

typedef struct {
    int sweep_order;            /* gsis_sweep_order; default GSIS_ORDER_LONGEST */
    int sweep_dynamic;          /* 1: sweep units from a counter in order; 0: static placement
                                   when the whole grid is resident (default 1) */
    int synth_cells_per_cta;    /* strip solver of each problem on the smallest cluster of 2, 4, 8
                                   or 16 CTAs with at most this many cells per CTA (larger where the
                                   levels do not fit a CTA); 0 = the cluster gsis_solve uses
                                   (default 0) */
} gsis_batch_tuning;

/* Fills *t with the defaults above. */
void gsis_default_batch_tuning(gsis_batch_tuning* t);

/* Bytes of device workspace for gsis_solve_batch / gsis_batch_autotune on
 * these problems and options (every problem's gsis_solve workspace plus the
 * batch tables).  Returns GSIS_OK or GSIS_ERR_ARG. */
int gsis_batch_workspace_bytes(const gsis_problem* probs, int n, const gsis_options* opt, size_t* bytes);

/*
 * Solves probs[0..n-1] (1 <= n <= 4096) as described above and writes each
 * problem's rho, F, iters, err and status.  opt is shared (scheme, precision,
 * tolerances, pseudo-time, check_every, stall_window; stall detection is per
 * problem).  tuning: NULL = the tuning gsis_batch_autotune last chose for a
 * batch of the same shapes and options in this process, else the defaults.
 * workspace: device, >= gsis_batch_workspace_bytes(), 256-byte aligned.
 * SYNCHRONISES the stream.  Returns GSIS_OK when every problem returned
 * GSIS_OK, GSIS_ERR_MAXITER / _DIVERGED / _STALLED when some problem did
 * (see probs[p].status), or an argument, CUDA, timeout or workspace error
 * (then no problem's outputs are valid).
 */
int gsis_solve_batch(gsis_problem* probs, int n, const gsis_options* opt, const gsis_batch_tuning* tuning,
                     void* workspace, size_t workspace_bytes, void* stream);

/*
 * Autotuner of gsis_solve_batch: runs trial_iters iterations (after one
 * untimed iteration) of every candidate tuning -- the four sweep orders,
 * static or counter placement, and synth_cells_per_cta in {0, 4096, 16384}
 * -- from rho^0 = 0, timed with CUDA events on the stream, and keeps the
 * fastest per iteration (ties to the earlier candidate).  The choice is
 * remembered for later gsis_solve_batch calls with tuning = NULL on batches
 * of the same shapes and options.
 * best: HOST out.  ms_per_iter: HOST out or NULL, the chosen candidate's time.
 * class_ms: HOST [GSIS_KCLASS_COUNT] out or NULL: device time per iteration of
 *   each kernel class (sweep, moments, HoT / right-hand side, synthetic,
 *   update) of the chosen tuning, from events between the class launches.
 * Problem outputs (rho, F, iters, err, status) are not written.
 * SYNCHRONISES the stream.
 */
int gsis_batch_autotune(gsis_problem* probs, int n, const gsis_options* opt, int trial_iters,
                        gsis_batch_tuning* best, double* ms_per_iter, double* class_ms,
                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * gsis_transport_sweep() for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an interface convenience.
 *
 * Callers without a device allocator of their own (a plain C host program
 * that links only this library, a plug-in whose host application owns all
 * device memory through its own pool) pass only their inputs and outputs;
 * the scratch is one static device array of GSIS_STATIC_SCRATCH_BYTES
 * (32 MiB) inside the library.  Every GPU on which the library's kernels are
 * loaded keeps that array reserved until the process exits.
 * Arguments, layouts and results are those of gsis_transport_sweep().
 * Problems whose kinetic-step workspace exceeds the array are rejected with
 * GSIS_ERR_WORKSPACE before any device work: the workspace that
 * gsis_transport_sweep() needs, which runs first-order upwind without
 * pseudo-time whatever opt asks (gsis_workspace_bytes() of the same options
 * with spatial_order = 1 and cfl_p = beta = 0).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, once per
 * device): make that first call before any stream capture.  All calls share
 * the one array, which keeps the last call's contents (each call clears what
 * must start at zero); calls that overlap on the GPU race on it.  The call
 * allocates no device memory (no cudaMalloc/cudaFree).  Stream-ordered.
 */
#define GSIS_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int gsis_transport_sweep_static(const gsis_mesh* mesh, const gsis_quadrature* quad,
                                const gsis_options* opt, const double* sigma_a,
                                const double* sigma_s, const double* q, const double* inflow,
                                const double* rho_in, double* rho_half, double* F_half,
                                double* P_half, double* bflux, void* stream);

/*
 * Instrumentation (not part of the method): every call counts the kernels it
 * launches per class; after gsis_profile_enable(1) each class launch is also
 * bracketed by CUDA events on the caller's stream and its device time is
 * accumulated when the call synchronises.  Host-global, not thread-safe
 * against concurrent calls.
 */
typedef enum {
    GSIS_KCLASS_SETUP = 0,   /* per-call set-up: coefficients, operator, 1/d table, state init */
    GSIS_KCLASS_SWEEP = 1,   /* the transport sweep */
    GSIS_KCLASS_MOMENTS = 2, /* angular moments + boundary fluxes (2 kernels per launch group) */
    GSIS_KCLASS_HOT_RHS = 3, /* ALSM gradient, HoT, synthetic right-hand side (2 kernels) */
    GSIS_KCLASS_SYNTH = 4,   /* synthetic solve */
    GSIS_KCLASS_UPDATE = 5,  /* Err, convergence decision, next source */
    GSIS_KCLASS_COUNT = 6
} gsis_kernel_class;

typedef struct {
    long long kernels;   /* kernels launched in this class */
    long long groups;    /* launch groups (class calls) */
    long long timed;     /* groups with a device time */
    double total_ms;     /* summed device time of the timed groups */
} gsis_kernel_stats;

/* enable != 0: time later launches; always resets the counters. */
int gsis_profile_enable(int enable);

/* Copies min(n, GSIS_KCLASS_COUNT) entries (indexed by gsis_kernel_class). */
int gsis_profile_read(gsis_kernel_stats* out, int n);

/* Summary of the last gsis_solve() on this host thread (instrumentation). */
typedef struct {
    int iters;                    /* outer iterations done */
    long long synth_inner_iters;  /* FP32 multigrid-CG iterations summed over the synthetic solves */
    double err;                   /* final Err(rho) */
    double synth_relres;          /* last synthetic relative residual (-1: budget spent, not evaluated) */
} gsis_solve_info;

/* Copies the summary of the last gsis_solve() of this thread; GSIS_ERR_ARG if out is NULL. */
int gsis_last_solve_info(gsis_solve_info* out);

/* Static description of a status code (never NULL). */
const char* gsis_status_string(int status);

/* Message of the last failing call on this host thread ("" if none). */
const char* gsis_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GSIS_H */
