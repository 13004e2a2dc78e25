/*
 * tc.h -- C ABI of libtc, a GB300 (sm_103a) implementation of the
 * pseudospectral time step for Taylor-Couette flow (nsCouette, arXiv:1908.00587).
 *
 * Method (paper Sec. 2.1): Fourier-Galerkin in theta and z (z periodic), 9-point
 * finite differences in r on Chebyshev-Gauss-Lobatto points, a semi-implicit
 * predictor-corrector with dynamic time step, optional Boussinesq temperature
 * with a radial temperature drop and gravity along z.  The linear terms are
 * solved independently per Fourier mode (Sec. 2.2); the nonlinear terms are
 * formed on the 3/2-padded physical grid.
 *
 * Units: gap d = r_o - r_i = 1, time d^2/nu, velocity nu/d; r_i = eta/(1-eta).
 * Walls: u_theta(r_i) = Re_i, u_theta(r_o) = Re_o, T(r_i) = +1/2, T(r_o) = -1/2.
 *
 * Spectral state layout (all entry points, host or device): complex128 as
 * interleaved (re, im) doubles, C order [field][r][m][kk], with
 *   field = u_r, u_theta, u_z (, T when Ra != 0),
 *   r  = 0..Nr-1 ascending from the inner wall,
 *   m  = 0..M,  M = floor((Ntheta-1)/3)   (Hermitian half in theta),
 *   kk = 0..2K, K = floor((Nz-1)/3), axial index k = kk for kk <= K and
 *        kk - (2K+1) otherwise (FFT order); axial wavenumber 2 pi k / Lz.
 * The m = 0 column must satisfy u(0,-k) = conj(u(0,k)).
 *
 * Conventions: every call returns a tc_status; nothing is thrown across the
 * ABI.  Errors are not sticky except TC_ERR_CUDA, after which only tc_destroy
 * is valid on that context.  Caller buffers are never retained after a call
 * returns.  All device work runs on the context's stream (default: the legacy
 * default stream; see tc_set_stream); calls that return data to the host
 * synchronise that stream.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_ctx tc_ctx;

typedef enum {
  TC_OK = 0,
  TC_ERR_ARG = 1,          /* invalid argument (size, range, null pointer)      */
  TC_ERR_CUDA = 2,         /* CUDA runtime error; context is poisoned            */
  TC_ERR_OOM = 3,          /* device allocation failed or over memory budget     */
  TC_ERR_NONFINITE = 4,    /* NaN/Inf found in the state                         */
  TC_ERR_CFL = 5,          /* CFL number above the configured limit              */
  TC_ERR_STATE = 6,        /* state violates the m = 0 Hermitian symmetry        */
  TC_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up                 */
  TC_ERR_UNSUPPORTED = 8   /* size or option not supported                       */
} tc_status;

/* Global quantities of the current state (tc_diagnostics).
 *   t          simulated time
 *   dt         last time step used
 *   E          (1/2) int |u|^2 dV
 *   E_pert     same for u minus the basic state of tc_create
 *   torque_i/o 2 pi Lz r^2 (d u_theta/dr - u_theta/r) of the mean flow at r_i / r_o
 *   P_wall     power the walls put into the fluid
 *   eps        viscous dissipation int 2 S:S dV
 *   buoy_work  Gr int u_z T dV  (Gr = Ra/Pr)
 *   Nu_i/o     mean dT/dr at the wall over that of the conductive state (Sec. 4)
 *   div_max    max |div u| over all stored coefficients
 *   div_rms    (int |div u|^2 dV / V)^(1/2)
 *   cfl        CFL number of the last step's start-of-step state times dt
 *   corr_diff  last step: max |X_corr - X_prev| over the stored coefficients
 *              (real and imaginary parts) of its last two iterates (the last
 *              corrector and the one before it, or the predictor)
 */
typedef struct {
  double t, dt, E, E_pert, torque_i, torque_o, P_wall, eps, buoy_work;
  double Nu_i, Nu_o, div_max, div_rms, cfl;
  double corr_diff;
} tc_diag;

/* Sizes derived by tc_create. */
typedef struct {
  int Nr, Ntheta, Nz, M, K, nfields;
  long long coeffs_per_field;   /* Nr * (M+1) * (2K+1) */
  long long state_bytes;        /* nfields * coeffs_per_field * 16 */
  size_t device_bytes;          /* device memory held by the context */
  long long launches;           /* kernels launched since tc_create */
  int tile_mb, tile_lb;         /* nonlinear-stage tiles in use (see "tile_mb") */
  int tile_mbf;                 /* m columns per CTA of the forward axial kernel */
  int tensor_theta;             /* 1: the azimuthal stage runs on the tensor cores */
  int tensor_z;                 /* 1: the inverse axial stage runs on the tensor cores */
} tc_info;

/* Device time of one kernel accumulated while option "timing" is 1. */
typedef struct {
  char name[32];
  long long launches;   /* launches timed since the last tc_reset_timing */
  double ms;            /* summed CUDA-event time of those launches */
} tc_kernel_time;

/* Create a run (Sec. 2.1: one input defines points, modes, rotation rates).
 * Nr >= 9 radial points (walls included); Ntheta, Nz physical (3/2-padded)
 * sizes of the form 2^a 3^b 5^c, Ntheta even and >= 4, Nz >= 4, both <= 1024;
 * 0 < eta < 1; Lz > 0; Pr > 0 when Ra != 0.  Temperature is carried only when
 * Ra != 0.  The state starts as the discrete basic state: circular Couette
 * flow, and with Ra != 0 the conductive temperature and its steady axial flow.
 * Each transform kernel holds a whole batch of sequences in shared memory
 * (two buffers of 16 B per padded point, at most 227 KB per CTA), so the
 * largest azimuthal size is 1000 without temperature and 750 with it (FP64,
 * one z-row per CTA); larger sizes return TC_ERR_UNSUPPORTED.
 * Errors: TC_ERR_ARG, TC_ERR_UNSUPPORTED, TC_ERR_OOM, TC_ERR_CUDA. */
tc_status tc_create(int Nr, int Ntheta, int Nz, double eta, double Lz,
                    double Re_i, double Re_o, double Ra, double Pr, tc_ctx **out);

/* Free everything the context holds.  Accepts NULL. */
tc_status tc_destroy(tc_ctx *ctx);

/* Set a numeric option.  Keys:
 *   "precision" 0: FP64 throughout (default).  1: mixed -- the transforms and
 *               the products u'.grad u' of the perturbation u' = u - U(r)
 *               run in FP32; the products with the (0,0) mean-flow mode U,
 *               the buoyancy, the radial band LU solves, the influence
 *               matrix and the state stay FP64.  Its error against the FP64
 *               path is measured, not bounded (see the tests).
 *   "cfl"       CFL coefficient of the dynamic step (default 0.25)
 *   "dt_max"    largest dynamic step (default 1e-3)
 *   "cfl_limit" abort a step with TC_ERR_CFL above this CFL number (default 0 = off)
 *   "check"     1: report NaN/Inf produced by tc_step (default 1)
 *   "timing"    1: bracket every kernel launch with CUDA events on the
 *               context's stream (tc_get_timing); 0: off (default)
 *   "graph"     1 (default): tc_step captures one step as a CUDA graph and
 *               replays it (re-captured after any option change or a new
 *               fixed dt); 0, or timing on: kernels launched one by one.
 *               Results are identical either way.
 *   "tile_mb"   m columns per CTA of the inverse axial kernel (and, unless
 *               "tile_mbf" is set, of the forward one), "tile_mbf" m columns
 *               per CTA of the forward axial kernel, "tile_lb" z rows per
 *               CTA of the azimuthal kernel (0: size-based default;
 *               TC_ERR_UNSUPPORTED if the shared memory would not fit).  The
 *               tiles change only which CTA computes a transform, not the
 *               arithmetic, so results are identical for every choice.
 *   "n_corr"    corrector passes per step, 1..16 (default 1).  Each pass
 *               solves the stage with c N(X_prev) + (1-c) N^n and the same
 *               explicit part; diagnostics report the last difference.
 *   "flux_constraint"  1: a uniform axial pressure gradient in the (0,0)
 *               u_z equation, solved with every stage, keeps the axial
 *               volume flux int u_z r dr at zero (default 0).  With
 *               temperature it also gives the basic state zero axial flux;
 *               set it before tc_init_perturbation.
 *   "eps_centrifugal"  centrifugal buoyancy coefficient eps (default 0): the
 *               momentum advection u.grad u (with its curvature terms) is
 *               weighted by the density factor 1 - eps T.  Needs the
 *               temperature (Ra != 0) and precision 0; TC_ERR_UNSUPPORTED
 *               otherwise.
 *               The adjoint entry points cover the default scheme only: they
 *               return TC_ERR_UNSUPPORTED when n_corr != 1, flux_constraint is
 *               on (tc_stage_solve_adjoint, tc_adjoint_step) or eps != 0
 *               (tc_nonlinear_adjoint, tc_adjoint_step).
 *   "memory_budget"  largest device memory, in bytes, the context may hold
 *               (0: no limit, the default).  Every allocation made after
 *               tc_create -- the FP32 state copy of precision 1, the buffers
 *               of the first adjoint call, a longer step history in tc_step,
 *               the flux-constraint response, the scratch of
 *               tc_set_state_regrid -- that would take tc_get_info's
 *               device_bytes above it returns TC_ERR_OOM instead, with the
 *               context unchanged and usable.  A failed device allocation
 *               returns TC_ERR_OOM the same way.
 *   "tensor_theta"  1: the inverse azimuthal transforms of the FP64
 *               nonlinear stage run as DFT-matrix products on the tensor
 *               cores (tcgen05), each operand split into 7 BF16 slices of 8
 *               significant bits, the level sums exact in FP32 and combined
 *               exactly in 64-bit integers: FP64-accurate (agrees with the FFT
 *               path to ~4e-16 of the largest term).  Needs Ntheta <= 128 and
 *               precision 0 (otherwise the FFT path runs).  0 (default): the
 *               FP64 FFT.  Which one is faster depends on the size (measured
 *               on GB300: 0.235 against 0.41 ms a launch at 64 x 128 x 128
 *               with temperature, 0.114 against 0.09 ms at 64 x 64 x 64, where
 *               most of the 128 rows of each product are padding); tc_autotune
 *               times both and keeps the faster.  The tile's block of the
 *               input arrives by a tiled TMA copy; if the driver refuses its
 *               tensor map at tc_create, the option has no effect.
 *   "tensor_z"  1: the inverse axial transforms of the FP64 nonlinear stage
 *               (of the state, of its radial derivative and of its axial
 *               derivative) run as products of the folded axial DFT matrix
 *               on the tensor cores, with the same 7-slice split and exact
 *               integer combination as "tensor_theta": FP64-accurate.  The
 *               matrix stacks the cosine rows j = 0 .. Nz/2 over the sine rows
 *               j = 1 .. (Nz-1)/2, and each output v_j, v_(Nz-j) is the exact
 *               sum of one cosine and one sine row before its rounding.
 *               Needs Nz <= 128 and precision 0 (otherwise the FFT path
 *               runs).  0 (default): the FP64 FFT.  Measured on GB300: 0.129
 *               against 0.179 ms a launch at 64 x 128 x 128 with
 *               temperature, 0.049 against 0.040 ms at 64 x 64 x 64 (half of
 *               the 128 matrix rows padding); tc_autotune times both.
 *   "tile_mb_adj"  m columns per CTA of the adjoint's axial kernels, 1 to 8
 *               (0, the default: the forward kernels' tile, at most 4, that
 *               lets three CTAs share an SM).  Results do not depend on it.
 *   "selftest_no_copy"  test hook, default 0.  1: the radial-sweep kernels
 *               and the tensor-core transform kernels ("tensor_theta",
 *               "tensor_z") never
 *               start their shared-memory copies of factors or DFT slices, so
 *               each of their bounded waits runs out (about 1 s) and tc_step
 *               or tc_nonlinear returns TC_ERR_TIMEOUT with its output left
 *               invalid.  Exercises the device-side timeout path without
 *               faulting the GPU.
 * Errors: TC_ERR_ARG for an unknown key or out-of-range value. */
tc_status tc_set_option(tc_ctx *ctx, const char *key, double value);

/* Use a caller-owned cudaStream_t for all device work (NULL: default stream). */
tc_status tc_set_stream(tc_ctx *ctx, void *cuda_stream);

/* Sizes of the run. */
tc_status tc_get_info(const tc_ctx *ctx, tc_info *out);

/* Copy a spectral state in (where = 0: host pointer, 1: device pointer), layout
 * above.  The input is checked on the device before it replaces the state:
 * TC_ERR_NONFINITE on NaN/Inf, TC_ERR_STATE if the m = 0 column's asymmetry
 * exceeds 1e-12 of the largest coefficient; otherwise the m = 0 column is
 * symmetrised (k > 0 kept) and the state replaced.
 * The simulated time is reset to 0 and the dynamic step forgets its history. */
tc_status tc_set_state(tc_ctx *ctx, const void *spec, int where);

/* Restart with a change of resolution (Sec. 2.1: resolution may change at a
 * restart, by interpolation and mode padding).  spec is the state of a run
 * of the same gap and axial period (eta_src, Lz_src must equal this run's,
 * else TC_ERR_ARG) on its own grid: complex128 [nfields_src][Nr_src]
 * [M_src+1][2 K_src+1], k in FFT order (where = 0 host, 1 device; not
 * retained).  Radial: the degree Nr_src - 1 polynomial through the source's
 * Chebyshev-Gauss-Lobatto nodal values, evaluated at this run's nodes (wall
 * values copy exactly).  Fourier: shared modes copied, the rest of this
 * run's modes zero, source modes beyond M, K dropped.  A source without T
 * (nfields_src = 3) given to a run with T gets this run's conductive
 * profile; the reverse drops T.  The result is then checked and committed
 * as tc_set_state does (same errors; time reset to 0).  Its divergence is
 * that of an interpolant; the next stage projects it.  Allocates device
 * scratch for the call (TC_ERR_OOM if that fails). */
tc_status tc_set_state_regrid(tc_ctx *ctx, const void *spec, int Nr_src, int M_src, int K_src,
                              int nfields_src, double eta_src, double Lz_src, int where);

/* Copy the current spectral state out (where = 0 host, 1 device). */
tc_status tc_get_state(const tc_ctx *ctx, void *spec, int where);

/* Copy the pressure of the last corrector stage out: complex128 [r][m][kk].
 * The (0,0) mode is left zero (the mean pressure is not solved for). */
tc_status tc_get_pressure(const tc_ctx *ctx, void *spec, int where);

/* Set the state to the basic state plus a divergence-free perturbation
 * u' = curl(psi) (Sec. 2.1: divergence-free initial conditions exciting
 * selected Fourier modes).
 *   psi    host, complex128 [3][mp+1][2kp+1] raw coefficients of (psi_r,
 *          psi_theta, psi_z), axial index natural (-kp..kp); each component
 *          gets the radial profile (1-x^2)^2, x = 2(r-r_i)-1; the m = 0 column
 *          is made Hermitian (k > 0 kept); u' is zeroed at the wall nodes and
 *          scaled so that max over the physical grid of |u'| equals amp.
 *   tcoef  host, complex128 [mp+1][2kp+1] or NULL: T' = (1-x^2) x tcoef, scaled
 *          so that max |T'| = amp_T (ignored when Ra == 0 or amp_T == 0).
 * A negative amp (amp_T) is taken as the scale factor itself, |amp| times
 * curl psi, without the max-norm rescaling: this keeps the map from the
 * coefficients to the state linear, as the gradient of
 * tc_init_perturbation_adjoint assumes.  Requires mp <= M and kp <= K. */
tc_status tc_init_perturbation(tc_ctx *ctx, const double *psi, int mp, int kp,
                               double amp, const double *tcoef, double amp_T);

/* Advance nsteps predictor-corrector steps (Sec. 2.1).  dt > 0: fixed step;
 * dt <= 0: dynamic step from the CFL bound of each start-of-step state,
 * dt* = min(dt_max, cfl / max(|u_r|/dr, |u_theta|/(r dtheta), |u_z|/dz)),
 * taken at once when smaller than the current step and only above 1.1x the
 * current step when larger.  dt_used (host, nullable) receives nsteps steps.
 * Errors: TC_ERR_ARG, TC_ERR_NONFINITE, TC_ERR_CFL, TC_ERR_CUDA. */
tc_status tc_step(tc_ctx *ctx, int nsteps, double dt, double *dt_used);

/* Clock of the run: the simulated time t of the current state and dt_prev,
 * the step that the next dynamic step is compared with (Sec. 2.1, dynamic
 * time-step control).  dt_prev is 0 after tc_create, tc_set_state,
 * tc_set_state_regrid and tc_init_perturbation (the next dynamic step is
 * then dt* itself), and the last step taken after tc_step.  A restart that
 * puts a saved state back with tc_set_state and then its saved clock with
 * tc_set_clock continues that run: the next dynamic step keeps dt_prev under
 * the rule of tc_step, and the Helmholtz factors are reused when that step is
 * the one they were last built for.  Either output pointer of tc_get_clock
 * (host) may be NULL; for a non-NULL dt_prev it synchronises the context's
 * stream and reads the value from the device (8 bytes).  tc_set_clock enqueues the dt_prev write on the
 * context's stream.  Errors: TC_ERR_ARG for a NULL context, a non-finite t or
 * dt_prev, or dt_prev < 0; TC_ERR_CUDA. */
tc_status tc_get_clock(const tc_ctx *ctx, double *t, double *dt_prev);
tc_status tc_set_clock(tc_ctx *ctx, double t, double dt_prev);

/* Diagnostics of the current state (one small device->host copy). */
tc_status tc_diagnostics(tc_ctx *ctx, tc_diag *out);

/* Stage entry points, used to check each stage on its own.
 * tc_nonlinear: dealiased nonlinear terms [N_r, N_theta, N_z(, N_T)] of a
 *   spectral state given on the device (layout of the state), written to a
 *   device buffer of the same size; *cfl_rate (host, nullable) receives
 *   max(|u_r|/dr, |u_theta|/(r dtheta), |u_z|/dz) over the physical grid.
 *   TC_ERR_TIMEOUT if a bounded device wait ran out (output invalid; the
 *   context stays usable).
 * tc_stage_solve: one implicit stage.  rhs (device) holds the explicit
 *   right-hand side in +- form [R+, R-, R_z(, R_T)] at every radial node
 *   (R+- = R_r +- i R_theta); the solution of (I/dt - L/2) X = R - grad p,
 *   div X = 0 at both walls, with the wall values, is written to x_out
 *   (device, primitive fields) and the pressure to p_out (device, nullable). */
tc_status tc_nonlinear(tc_ctx *ctx, const void *state_dev, void *n_dev, double *cfl_rate);
tc_status tc_stage_solve(tc_ctx *ctx, const void *rhs_dev, double dt, void *x_out_dev,
                         void *p_out_dev);

/* Discrete adjoint of one predictor-corrector step at fixed dt (FP64 path only;
 * TC_ERR_UNSUPPORTED with precision 1).  adj (device, state layout) holds
 * lambda^{n+1} on entry and lambda^n = P_H J(X^n)^T lambda^{n+1} on return,
 * where J is the Jacobian of the step at state_n (device, state layout,
 * caller-owned), transposed in the real Euclidean inner product of the stored
 * (Re, Im) coefficients, and P_H is the orthogonal projection onto
 * u(0,-k) = conj u(0,k).  The step's intermediate states are recomputed from
 * state_n; the context's own state is not changed.  Errors: TC_ERR_ARG,
 * TC_ERR_TIMEOUT, TC_ERR_OOM, TC_ERR_CUDA. */
tc_status tc_adjoint_step(tc_ctx *ctx, const void *state_n_dev, double dt, void *adj_dev);

/* Recorded steps for the reverse sweep (checkpoint segments).
 * tc_record_bytes_per_step: bytes one recorded step takes: X^n and the
 *   predictor state X* (state layout each), then the physical-grid fields of
 *   X^n and of X* (complex128 [Nr][Nz][2 nfields][Ntheta] each: per component
 *   the pairs value + i d/dtheta and d/dr + i d/dz).
 * tc_step_record: advances nsteps steps of fixed dt > 0 like tc_step and
 *   writes step n's record at record_dev + n * that size (device,
 *   caller-owned, record_bytes long; TC_ERR_ARG if too short).
 * tc_adjoint_steps: lambda (adj, device) from step n0 + nsteps back to n0
 *   over nsteps records written by tc_step_record with the same dt, last
 *   first -- the same map as nsteps calls of tc_adjoint_step on the recorded
 *   states, without recomputing any forward stage.  The context's state is
 *   not changed.
 * Both cover the default scheme only (TC_ERR_UNSUPPORTED otherwise, as for
 * tc_adjoint_step).  Errors: TC_ERR_ARG, TC_ERR_NONFINITE (record),
 * TC_ERR_TIMEOUT, TC_ERR_OOM, TC_ERR_CUDA. */
tc_status tc_record_bytes_per_step(const tc_ctx *ctx, long long *bytes);
tc_status tc_step_record(tc_ctx *ctx, int nsteps, double dt, void *record_dev,
                         long long record_bytes);
tc_status tc_adjoint_steps(tc_ctx *ctx, int nsteps, const void *record_dev, double dt,
                           void *adj_dev);

/* Adjoint of the nonlinear stage at state_dev: xbar = (dN/dX)^T nbar (device
 * buffers of the state layout; nbar holds cotangents of N_r, N_theta, N_z(, N_T)). */
tc_status tc_nonlinear_adjoint(tc_ctx *ctx, const void *state_dev, const void *nbar_dev,
                               void *xbar_dev);

/* Adjoint of the linear part of one implicit stage at step dt: rbar (device,
 * +- form like tc_stage_solve's rhs) = A^T xbar (device, primitive fields). */
tc_status tc_stage_solve_adjoint(tc_ctx *ctx, const void *xbar_dev, double dt, void *rbar_dev);

/* Objective of the differentiation form: *J = E_pert of the current state
 * (1/2 int |u - u_base|^2 dV) and, when grad_dev (device, state layout) is
 * non-NULL, dJ/dX = V w_j r_j c_m (u - u_base) (zero for T). */
tc_status tc_objective(tc_ctx *ctx, double *J, void *grad_dev);

/* Gradient with respect to the raw coefficients of the last
 * tc_init_perturbation (the scales that made max|u'| = amp and max|T'| =
 * amp_T are held fixed): lam_dev (device, state layout) is dJ/dX^0; psi_bar
 * (host, complex128 [3][mp+1][2kp+1]) and tcoef_bar (host, nullable,
 * [mp+1][2kp+1]) receive dJ/dRe + i dJ/dIm of each raw coefficient. */
tc_status tc_init_perturbation_adjoint(tc_ctx *ctx, const void *lam_dev, int mp, int kp,
                                       double *psi_bar, double *tcoef_bar);

/* Scale factors the last tc_init_perturbation applied to curl psi and to T'. */
tc_status tc_get_ic_scales(const tc_ctx *ctx, double *s_u, double *s_T);

/* Per-kernel device times recorded while "timing" is on: fills up to cap
 * entries of out (host) and sets *count.  Synchronises the stream. */
tc_status tc_get_timing(tc_ctx *ctx, tc_kernel_time *out, int cap, int *count);
/* Forget the recorded times. */
tc_status tc_reset_timing(tc_ctx *ctx);

/* Sustained FP64 FMA rate of the current device, the peak of the ALU
 * roofline of the FP64 kernels (the paper has no counterpart; it is a
 * measurement aid).  Runs 4 independent FMA chains per thread, 32 warps on
 * every SM, for about target_ms milliseconds (0 < target_ms <= 10000) on
 * `stream` (NULL: default stream), after one untimed launch that also lets
 * the clock settle, and writes the rate in TFLOP/s to *tflops (host).
 * Allocates and frees a small device buffer (SMs x 1024 doubles) and
 * synchronises the stream.  Errors: TC_ERR_ARG for a null tflops or a
 * target_ms out of range (checked before any device call), TC_ERR_OOM if the
 * buffer cannot be allocated, TC_ERR_CUDA for any other CUDA failure (the
 * calling thread's CUDA error state is cleared; no context is involved). */
tc_status tc_measure_fp64_rate(double target_ms, void *stream, double *tflops);

/* Nonlinear terms without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * -- code embedded in a host application that owns all device memory through
 * its own pool (a cudaMalloc there fails once the pool holds the device, or
 * escapes the pool's accounting), and code on a latency-critical path, where
 * cudaMalloc may synchronise the device and stall other work.
 * It computes what tc_nonlinear computes, for the run tc_create would make
 * from (Nr, Ntheta, Nz, eta, Lz, Ra, Pr), with no context: state_dev and n_dev
 * (device, layout of the state, caller-owned) are the only caller buffers.
 * Every other buffer -- radial tables, twiddles, the transformed
 * intermediates, the CFL slot -- lives in one fixed 32 MiB device array that
 * every GPU loading this library holds until the process exits.  Limits:
 * Nr <= 256, Ntheta and Nz <= 512, and the intermediates plus tables must fit
 * in the 32 MiB (3 nfields + nfields planes of Nr * Nz * (M+1) complex128);
 * larger sizes return TC_ERR_UNSUPPORTED, other invalid sizes TC_ERR_ARG.
 * The first call on a device looks up the array's device address for that
 * device (make it before any stream capture); the address is kept for the
 * life of the process, so do not call this entry point on a device after
 * cudaDeviceReset of that device.  Each call copies its small radial and
 * twiddle tables (a few tens of KB) in on `stream` from a buffer on its own
 * host stack; that memory is pageable, so the driver may hold the copy, and
 * the call, until the work already queued on `stream` is done.  All calls share the array and
 * each call overwrites the previous call's contents (the CFL slot is cleared
 * every call), so calls that overlap on the GPU race: serialise them.  Work
 * runs on `stream` (NULL: default stream); *cfl_rate (host, nullable) as in
 * tc_nonlinear, which synchronises the stream when requested. */
tc_status tc_nonlinear_noalloc(int Nr, int Ntheta, int Nz, double eta, double Lz, double Ra,
                               double Pr, const void *state_dev, void *n_dev, void *stream,
                               double *cfl_rate);

/* Ensemble of independent runs of uneven size (batching form).  Each member
 * is an ordinary context on a stream of its own (reach it with
 * tc_ensemble_member to set its state, options or initial condition; do not
 * destroy it or change its stream).  Per-member parameters: */
typedef struct {
  int Nr, Ntheta, Nz;
  double eta, Lz, Re_i, Re_o, Ra, Pr;
  int precision;   /* 0 FP64, 1 mixed (see the "precision" option) */
} tc_params;
typedef struct tc_ens tc_ens;

/* Create n members (arguments validated as in tc_create).  autotune_tiles =
 * 1 times the nonlinear stage for candidate tile shapes once per size class
 * (Nr, Ntheta, Nz, fields, precision) and keeps the fastest; the choice does
 * not change any result.  Errors: those of tc_create, TC_ERR_CUDA. */
tc_status tc_ensemble_create(int n, const tc_params *p, int autotune_tiles, tc_ens **out);

/* The context of member i (owned by the ensemble). */
tc_status tc_ensemble_member(tc_ens *e, int i, tc_ctx **ctx);

/* Advance every member nsteps steps of its own fixed dt (host array of n
 * values > 0), in the ensemble's launch mode (tc_ensemble_set_mode):
 *   1 one persistent kernel launch (per 50 steps) runs the steps
 *     of every member: the work items are the CTA tiles of the step's
 *     kernels; each member moves to its next stage of the predictor-corrector
 *     step when its current stage's tiles are done, and resident CTAs claim
 *     ready tiles of any member, so the members proceed independently.
 *     Nothing in it waits on another CTA; a CTA that finds no ready work for
 *     2 s, or a sweep copy that does not land within 1 s, makes the call
 *     return TC_ERR_TIMEOUT without a fault.  It runs
 *     the default scheme: while any member has n_corr != 1, the flux
 *     constraint or the sweep test hook, the call steps in mode 0 instead.
 *     It shrinks transform tiles that do not fit its shared-memory budget
 *     (results do not depend on tiles).
 *   0 (default) one step of all members captured once into a CUDA graph
 *     (independent branches run concurrently) and replayed nsteps times;
 *     re-captured when a dt or a member option changes.  It is the default
 *     because it is faster: the persistent kernel is compiled for the
 *     register demand of its largest body (16 warps per SM), the members'
 *     own kernels run with more warps.
 * Mode 0 is bit-identical to each member stepped alone.  Mode 1 computes the
 * same tiles with the same device code, but compiled into one kernel, where
 * the compiler may fuse multiplies and adds differently: it agrees with the
 * member stepped alone to round-off (tested: 1e-13 of the largest
 * coefficient after 12 steps).
 * Returns the worst member status (TC_ERR_TIMEOUT, TC_ERR_NONFINITE) after
 * a synchronisation. */
tc_status tc_ensemble_step(tc_ens *e, int nsteps, const double *dt);

/* Launch mode of tc_ensemble_step: 0 graph of per-member kernels (default),
 * 1 persistent kernel, 2 persistent kernel with its test hook -- the end of
 * member 0's first transform stage is never published, so that member never
 * becomes ready again; the others finish, every CTA's bounded idle wait (2 s)
 * runs out and tc_ensemble_step returns TC_ERR_TIMEOUT (member 0's state is
 * then the one before the call, the others have stepped).  Errors:
 * TC_ERR_ARG. */
tc_status tc_ensemble_set_mode(tc_ens *e, int mode);
tc_status tc_ensemble_get_mode(const tc_ens *e, int *mode);

/* Tile autotuner for one context (the one the ensemble runs per size
 * class): times the nonlinear stage on the context's current state for tile
 * shapes {1, 2, 3, 4, 5, 6, 8} of "tile_mb", then {1, 2, 3, 4, 8} of
 * "tile_lb", then (precision 0, Ntheta <= 128) "tensor_theta" 1 against 0,
 * then (precision 0, Nz <= 128) "tensor_z" 1 against 0, then
 * {1, 2, 3, 4, 5, 6, 8} of "tile_mbf", keeps the fastest and returns the
 * first two (host, nullable; tc_get_info reports all five).  Results do not
 * depend on the tiles; the tensor-core stages change them only at round-off
 * (see "tensor_theta", "tensor_z"). */
tc_status tc_autotune(tc_ctx *ctx, int *tile_mb, int *tile_lb);

/* Kernel launches per tc_ensemble_step step: the kernels one graph replay
 * (one step of every member) contains in mode 0; 1 in the persistent modes
 * (one launch covers every step of a call). */
tc_status tc_ensemble_kernels_per_step(const tc_ens *e, long long *count);

/* Free the members, streams and graph.  Accepts NULL. */
tc_status tc_ensemble_destroy(tc_ens *e);

/* Index checks of the debug build (libtc_debug.so, compiled with
 * -DTC_DEBUG; the paper's quality assurance runs short tests with runtime
 * checks and the compilers' tightest debug settings, Sec. 2.5).  In that build the step kernels check the indices
 * of their global and shared-memory accesses (state, nonlinear intermediates,
 * transform buffers, right-hand sides, radial sweeps and their factor copies,
 * influence data); an index out of range sets one bit per check site in a
 * device word and the access is skipped -- nothing traps.  *flags (host)
 * receives the bits set since the last clear (0: every index was in range);
 * clear != 0 resets them.  Synchronises the device.  Errors: TC_ERR_ARG for a
 * NULL flags, TC_ERR_UNSUPPORTED in the normal build (libtc.so, where the
 * checks compile away), TC_ERR_CUDA. */
tc_status tc_debug_flags(unsigned *flags, int clear);

/* Human-readable name of a status. */
const char *tc_status_string(tc_status s);

#ifdef __cplusplus
}
#endif
#endif /* TC_H */
