/*
 * libpmgb -- differentiable particle-mesh (PM) N-body simulation with the adjoint method,
 * hand-written CUDA for sm_103a (GB300).  C ABI.
 *
 * Method: Li et al., "Differentiable Cosmological Simulation with the Adjoint Method"
 * (arXiv:2211.09815).  Forward model: Zel'dovich or 2LPT initial conditions from white
 * noise (Sec. 2.1, Eqs. 2-7; App. A), PM gravity by CIC scatter, FFT Poisson solve with the -ik
 * gradient and CIC gather (Sec. 2.2, Eqs. 10-11), FastPM kick-drift-kick leapfrog
 * (Sec. 2.3, Eqs. 13-16).  Gradient: the discrete adjoint integrated backward in time
 * jointly with the reverse leapfrog (Sec. 3.6, Eqs. 49-51), with optional piecewise
 * resumption from stored states (Sec. 3.5).
 *
 * Conventions (shared with the test oracle):
 *   - lengths in Mpc/h, time in 1/H0, flat LCDM, theta = (A_s, n_s, Omega_m, Omega_b, h);
 *   - mesh n_mesh^3 nodes at g*l, l = box/n_mesh; particle lattice q = j*box/n_ptcl + l/2;
 *   - arrays are C order with the last axis fastest; vector fields are [3][N] (structure
 *     of arrays) with component c along array axis c; particle j is lattice point j;
 *   - particle mass m = n_mesh^3/n_ptcl^3 (mean density 1), delta = rho - 1;
 *   - the forward state is (s, p): displacement s = x - q and canonical momentum p.
 *
 * Memory: every pointer argument is a device pointer unless stated otherwise, allocated
 * and owned by the caller, in the context's precision (float for PM_F32, double for
 * PM_F64).  The context owns its scratch (meshes, fixed-point accumulators, spectra,
 * particle state, checkpoints) and frees it in pm_destroy.  All work is enqueued on the
 * stream given to pm_init; calls return once the work is enqueued, except where a host
 * output pointer forces a synchronisation (noted per call).
 *
 * Errors: every call returns a status (PM_OK = 0).  Arguments are validated on the host
 * before any launch; nothing is written on error.  No exception crosses the ABI.  The
 * device-side waits of the TMA-staged FFT passes are bounded; a wait that gives up sets a
 * device flag and its kernel returns early (the results of that work are then invalid).
 * The flag is read, reported as PM_ERR_TIMEOUT and cleared by pm_check and by every call
 * that synchronises the stream for a host output; an asynchronous call (pm_forward,
 * pm_adjoint with device outputs, pm_gradient_graph, the operators) reports it through the
 * next such call or pm_check.
 */
#ifndef PMGB_PM_H
#define PMGB_PM_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PM_OK = 0,
  PM_ERR_ARG = 1,        /* invalid argument or configuration */
  PM_ERR_OOM = 2,        /* device allocation failed */
  PM_ERR_CUDA = 3,       /* a CUDA call failed (see pm_last_cuda_error) */
  PM_ERR_NONFINITE = 4,  /* non-finite theta */
  PM_ERR_OVERFLOW = 5,   /* fixed-point range exceeded */
  PM_ERR_TIMEOUT = 6,    /* a bounded device wait gave up */
  PM_ERR_STATE = 7       /* call out of order (e.g. pm_adjoint before pm_forward) */
};

enum { PM_F32 = 0, PM_F64 = 1 };

typedef struct pm_ctx pm_ctx; /* opaque, library-owned */

typedef struct {
  double box;       /* periodic box side L in Mpc/h, > 0 */
  int n_mesh;       /* mesh nodes per side: power of two, 8..1024, multiple of n_ptcl */
  int n_ptcl;       /* particles per side: power of two, >= 4 */
  int n_steps;      /* leapfrog steps n >= 1, scale factors linear in a (Sec. 4) */
  double a0, a1;    /* initial and final scale factor, 0 < a0 < a1 */
  int precision;    /* PM_F32 or PM_F64 */
  int ckpt_every;   /* 0: reverse time integration; k > 0: resume the reverse pass from
                       states (s_j, p_j) stored every k steps (Sec. 3.5) */
  int deconv;       /* 1: divide the Green's function by the CIC window prod sinc^4 */
  int batch;        /* independent instances B >= 1 (own theta and omega each) */
  int lpt_order;    /* initial conditions (Sec. 2.1, Eq. 2): 0 or 1 = Zel'dovich (first
                       order), 2 = 2LPT, s = D1 s1 + D2 s2 with the second-order growth of
                       App. A (Eqs. 52-57); the adjoint then also back-propagates through
                       s2 (10 more lattice FFTs forward, 16 in the adjoint, 3 N more values) */
  int fixed_state;  /* 1: displacements and momenta held as 64-bit integers (units of 2^-40
                       cells and 2^-36 cells per unit of drift factor); kicks and drifts add
                       rounded increments that the reverse pass subtracts again, so reverse
                       time integration recovers every forward state exactly (the paper's
                       FP32 reversion error, Sec. 3.5, disappears).  Kernels read working-
                       precision copies.  Not combined with ckpt_every > 0 (PM_ERR_ARG). */
  int half_force;   /* 1 (PM_F32 only, else PM_ERR_ARG): the force meshes that the gathers read
                       are stored in FP16, four halves per cell, each field of a mesh row
                       scaled by a power of two chosen from the row's largest magnitude (an
                       int8 exponent per row and field); the row transforms compute in FP32
                       and the gathers convert back.  Halves the bytes of the [cell][4] mesh
                       written by the C2R x passes and read by the gathers, at FP16 rounding
                       of the force (a reduced-precision form, not the paper's). */
} pm_config;

/*
 * Create a context: validates cfg and theta, computes the FP64 cosmology tables on the
 * host (linear power spectrum Eq. 7 with the Eisenstein-Hu no-wiggle transfer function,
 * growth ODE of App. A Eqs. 52-58, FastPM factors Eq. 15 and their d/dOmega_m), and
 * copies omega into the context.
 *   out    : receives the context (host pointer to a pm_ctx*)
 *   cfg    : host pointer
 *   theta  : host pointer, [batch][5] doubles (A_s, n_s, Omega_m, Omega_b, h)
 *   omega  : device pointer, [batch][n_ptcl^3] white noise (Sec. 2.1, Eq. 6)
 *   stream : a cudaStream_t (0 = legacy default stream)
 * Errors: PM_ERR_ARG (bad sizes, null pointers), PM_ERR_NONFINITE, PM_ERR_OOM.
 */
int pm_init(pm_ctx** out, const pm_config* cfg, const double* theta, const void* omega, void* stream);

/*
 * Forward model (Sec. 2.1-2.3): Zel'dovich or 2LPT ICs at a0 (lpt_order), F_0, then n KDK
 * steps (Eq. 16).
 *   disp_out : optional, [batch][3][n_ptcl^3], final displacement s_n
 *   mom_out  : optional, [batch][3][n_ptcl^3], final momentum p_n
 *   dens_out : optional, [batch][n_mesh^3], final overdensity delta_n (CIC, Eq. 10)
 * The context keeps the final state for pm_adjoint.
 */
int pm_forward(pm_ctx* ctx, void* disp_out, void* mom_out, void* dens_out);

/*
 * Objective J = mean_g (delta_n(g) - target(g))^2 per instance (Sec. 2.4, Eq. 17 as a
 * field-level MSE) and its cotangent dJ/d delta_n = 2 (delta_n - target) / n_mesh^3.
 *   target      : [batch][n_mesh^3]
 *   loss_out    : [batch] doubles, host or device pointer (host: synchronises)
 *   dJ_ddens_out: [batch][n_mesh^3]
 * Requires pm_forward.  FP64 deterministic reduction.
 */
int pm_loss_mse(pm_ctx* ctx, const void* target, double* loss_out, void* dJ_ddens_out);

/*
 * Adjoint (Sec. 3.6, Eqs. 49-51): integrates the leapfrog backward jointly with the
 * adjoint variables (xi, pi), recomputing the forces instead of storing the trajectory
 * (or resuming from stored states if cfg.ckpt_every > 0), then back-propagates through
 * the initial conditions.
 *   dJ_ddens   : optional, [batch][n_mesh^3], dJ/d delta_n on the final density
 *   dJ_ddisp   : optional, [batch][3][n_ptcl^3], dJ/dx_n
 *   dJ_dmom    : optional, [batch][3][n_ptcl^3], dJ/dp_n
 *   dJ_domega  : optional, [batch][n_ptcl^3], receives dJ/d omega
 *   dJ_dtheta  : optional, [batch][5] doubles, host or device (host: synchronises)
 * Requires pm_forward since the last pm_adjoint; consumes the final state.
 */
int pm_adjoint(pm_ctx* ctx, const void* dJ_ddens, const void* dJ_ddisp, const void* dJ_dmom,
               void* dJ_domega, double* dJ_dtheta);

/*
 * Replace the inputs of a context without reallocating: theta (host, [batch][5], optional:
 * the host tables are recomputed) and/or omega (host or device, [batch][n_ptcl^3],
 * optional, copied on the context stream).  Invalidates the forward state.
 */
int pm_set_inputs(pm_ctx* ctx, const double* theta, const void* omega);

/*
 * One gradient evaluation of the density MSE objective with host or device buffers:
 * omega (optional, new white noise) and target ([batch][n_mesh^3]) are copied in,
 * then pm_forward, pm_loss_mse and pm_adjoint run on the context stream, and
 *   loss       : optional [batch] doubles (host or device)
 *   grad_omega : optional [batch][n_ptcl^3] (host or device)
 *   grad_theta : optional [batch][5] doubles (host or device)
 * are copied out.  Synchronises when any output is in host memory.  The first call
 * allocates the context's target, cotangent and gradient buffers.
 */
int pm_gradient(pm_ctx* ctx, const void* omega, const void* target, double* loss, void* grad_omega,
                double* grad_theta);

/*
 * One gradient evaluation (pm_forward, pm_loss_mse, pm_adjoint) on device buffers, replayed
 * from a CUDA graph: the first call (and any call whose pointers differ from the previous
 * one) runs the evaluation once normally, then captures it on the context stream and
 * instantiates the graph; every call launches the graph.  New theta/omega between calls go
 * through pm_set_inputs (they land in the buffers the graph reads).  All of target
 * ([batch][n_mesh^3]), loss ([batch]), grad_omega ([batch][n_ptcl^3]) and grad_theta
 * ([batch][5]) must be device pointers (optional except target), and the context must
 * have been created on a stream other than the legacy default stream (PM_ERR_ARG).
 */
int pm_gradient_graph(pm_ctx* ctx, const void* target, double* loss, void* grad_omega, double* grad_theta);

/*
 * Shell-averaged power spectrum of an overdensity mesh (a summary statistic of the
 * observable, Sec. 2.4): P(k_b) = V / M^2 <|DFT delta(k)|^2> over the modes with
 * b <= |n| < b + 1 (n the integer wavevector), b = 0 .. n_mesh/2 - 1, the mean taken over
 * the full k-space shell.  The sums are deterministic (int64 fixed point with a per-bin
 * scale), accumulated in FP64 precision.
 *   dens   : device [batch][n_mesh^3], or null for the context's last forward density
 *   pk     : [batch][n_mesh/2] doubles, host or device
 *   kmean  : optional [n_mesh/2] doubles, mean |k| per bin in h/Mpc
 *   nmodes : optional [n_mesh/2] doubles, number of modes per bin
 * Synchronises the stream.  Errors: PM_ERR_STATE when dens is null before any forward.
 */
int pm_power_spectrum(pm_ctx* ctx, const void* dens, double* pk, double* kmean, double* nmodes);

/*
 * Objective on the shell-averaged power spectrum (a summary-statistic objective, Sec. 2.4):
 * J = sum_b w_b (P_b - T_b)^2 per instance, P_b as in pm_power_spectrum, and its cotangent
 * for pm_adjoint, dJ/d delta(x) = sum_b 2 w_b (P_b - T_b) 2V / (M^2 C_b)
 * sum_{k in shell b} DFT[delta](k) e^{i k.x}  (C_b modes in shell b, V = box^3,
 * M = n_mesh^3; modes with |n| >= n_mesh/2 do not enter).
 *   dens         : device [batch][n_mesh^3], or null for the context's last forward density
 *   pk_target    : [batch][n_mesh/2] doubles T_b, host or device
 *   weights      : [batch][n_mesh/2] doubles w_b, host or device
 *   loss_out     : optional [batch] doubles, host or device (host: synchronises)
 *   dJ_ddens_out : device [batch][n_mesh^3]
 * Deterministic (the bin sums of pm_power_spectrum).  Errors: PM_ERR_ARG for null
 * target, weights or output; PM_ERR_STATE when dens is null before any forward.
 */
int pm_loss_power(pm_ctx* ctx, const void* dens, const double* pk_target, const double* weights, double* loss_out,
                  void* dJ_ddens_out);

/* Per-category timing of the context's kernel launches with CUDA events on its stream. */
enum {
  PM_PROF_SCATTER = 0,   /* CIC scatter (density, and pi in the adjoint)        */
  PM_PROF_X_R2C = 1,     /* x pass of the R2C FFT (fixed-point -> spectrum)      */
  PM_PROF_COLS = 2,      /* y column passes (forward and inverse)                */
  PM_PROF_Z_FORCE = 3,   /* fused z FFT + Green's function -ik G + inverse z     */
  PM_PROF_Z_ADJ = 4,     /* fused z FFT + adjoint Green's function + inverse z   */
  PM_PROF_X_C2R = 5,     /* x pass of the C2R FFT                                */
  PM_PROF_GATHER_FWD = 6,/* CIC force gather + kick + drift                      */
  PM_PROF_GATHER_ADJ = 7,/* CIC gather of a and alpha + reverse kicks and drift   */
  PM_PROF_OTHER = 8,     /* initial conditions, loss, reductions, IC adjoint       */
  PM_PROF_NCAT = 9
};
/* enable != 0 starts event timing (and clears the accumulators); 0 stops it.  Kernel
 * launch counts are kept either way. */
int pm_profile(pm_ctx* ctx, int enable);
/* Synchronises the stream; writes the milliseconds (events on) and kernel launch counts
 * per category accumulated since the last read into ms[PM_PROF_NCAT] and
 * launches[PM_PROF_NCAT] (either may be null), then clears them. */
int pm_profile_read(pm_ctx* ctx, double* ms, long long* launches);

/* Release the context and all its device memory (synchronises its stream). */
int pm_destroy(pm_ctx* ctx);

/*
 * Synchronise the context's stream and report any bounded device wait that gave up in
 * the work enqueued so far: PM_ERR_TIMEOUT (and the flag is cleared), else PM_OK, or
 * PM_ERR_CUDA if the stream itself failed.
 */
int pm_check(pm_ctx* ctx);

/* Static description of a status code. */
const char* pm_status_string(int status);

/* Message of the last CUDA error seen by this thread ("" if none). */
const char* pm_last_cuda_error(void);

/* Bytes of device scratch the context holds. */
long long pm_scratch_bytes(const pm_ctx* ctx);

/*
 * Launch shapes of the tunable passes (not in the paper; they change speed, never
 * results: the CIC sums are exact integers for any tile shape, and the staged and
 * unstaged column passes run the same radix stages).
 *   tile_log2_density[3] : log2 of the deposit tile extent along axes (z, y, x), the
 *                          density-only deposit of the forward steps; 9..12 in total,
 *                          x at least 2
 *   tile_log2_adjoint[3] : the same for the density + pi deposit of the adjoint steps
 *                          (9..11 in total)
 *   threads_density,
 *   threads_adjoint      : threads per tile, 256 or 512
 *   tma_columns          : 1 = TMA-staged persistent y/z column passes (meshes 128..1024),
 *                          0 = unstaged column passes
 *   fused_x              : bit 0 (forward deposit) and bit 1 (adjoint deposit) set = that
 *                          deposit writes the half spectra of its whole-row tiles (CIC
 *                          deposit and x pass of the R2C in one kernel, meshes 128..1024);
 *                          clear = it writes real meshes and a separate x pass transforms
 *                          them (the tile shapes above apply to that form)
 */
typedef struct pm_tuning {
  int tile_log2_density[3];
  int tile_log2_adjoint[3];
  int threads_density;
  int threads_adjoint;
  int tma_columns;
  int fused_x;      /* deposits fused with the x pass of the R2C (tiles of whole x rows;
                       meshes 128..1024): bit 0 the density deposit of the forward steps,
                       bit 1 the density + pi deposit of the adjoint steps; 0 = separate */
} pm_tuning;

/* Current launch shapes.  Errors: PM_ERR_ARG (null pointers). */
int pm_get_tuning(pm_ctx* ctx, pm_tuning* out);

/* Set launch shapes (validated on the host: PM_ERR_ARG if out of range, or tma_columns = 1
 * for a mesh size without the staged passes). */
int pm_set_tuning(pm_ctx* ctx, const pm_tuning* t);

/*
 * Autotuner: times every candidate deposit tile shape x threads per tile (for the forward
 * and the adjoint deposit separately), then each deposit fused with the x pass against the
 * best separate deposit plus x pass, and both column-pass forms on the context's current
 * particle state (the final state of the last pm_forward, else the Zel'dovich state), each
 * `reps` times with CUDA events on the context's stream (median; reps = 0 means 3), and
 * keeps the fastest.  Uses the context's scratch meshes and its adjoint buffers as scratch
 * (a following pm_adjoint re-initialises them); the forward state is kept.  Synchronises.
 *   chosen  : optional, receives the chosen shapes
 *   ms_best : optional, [3] doubles: best forward deposit, adjoint deposit and y column
 *             pass time (ms)
 * Errors: PM_ERR_ARG (reps outside 0..100), PM_ERR_CUDA.
 */
int pm_autotune(pm_ctx* ctx, int reps, pm_tuning* chosen, double* ms_best);

/* ------------------------------------------------------------------------------------
 * Operator entry points: single rows of the hot path on the context's buffers, for
 * parity tests and benchmarks.  All arrays are device pointers in the context precision.
 * ----------------------------------------------------------------------------------*/

/* Overdensity delta (Sec. 2.2, Eq. 10; deterministic int64 fixed point) of particles at
 * x = q + disp.  disp [batch][3][n_ptcl^3] -> dens_out [batch][n_mesh^3], dens_out aligned
 * to 4 elements (16 bytes FP32, 32 bytes FP64; PM_ERR_ARG otherwise). */
int pm_op_density(pm_ctx* ctx, const void* disp, void* dens_out);

/* PM accelerations a = -grad varphi(q + disp) (Sec. 2.2): scatter, R2C, Green's function
 * with -ik, 3 C2R, gather.  disp, acc_out: [batch][3][n_ptcl^3]. */
int pm_op_force(pm_ctx* ctx, const void* disp, void* acc_out);

/* Force and its vector-Jacobian product alpha = pi . da/dx (Sec. 3.6, Eq. 49 F line).
 * disp, pi, acc_out, alpha_out: [batch][3][n_ptcl^3]. */
int pm_op_force_vjp(pm_ctx* ctx, const void* disp, const void* pi, void* acc_out, void* alpha_out);

/* 3-D real FFT of n^3 meshes, n = n_mesh, in the numpy rfftn layout:
 * real [batch][n][n][n] <-> complex [batch][n][n][n/2+1] (interleaved re, im).
 * dir = -1: forward (unnormalised); dir = +1: inverse (unnormalised, no 1/n^3). */
int pm_op_fft(pm_ctx* ctx, int dir, const void* in, void* out);

/* Zel'dovich displacement for unit growth s1 (Sec. 2.1, Eqs. 3-6) of the context's omega.
 * s1_out: [batch][3][n_ptcl^3]. */
int pm_op_za(pm_ctx* ctx, void* s1_out);

/* Most snapshots pm_set_snapshots accepts. */
#define PM_MAX_SNAPSHOTS 64

/*
 * Observed intermediate states (Sec. 2.4: the observation and the objective may depend on
 * every state z_0..z_n, e.g. snapshots at the end of time steps).
 *   nsnap    : 0..PM_MAX_SNAPSHOTS; 0 clears the snapshots
 *   steps    : host [nsnap] ints, strictly ascending in 0..n_steps; step j is the state
 *              after j leapfrog steps (0: the initial state, n_steps: the final one)
 *   disp_out : optional device [nsnap][batch][3][n_ptcl^3]: every following pm_forward
 *              writes s_j of snapshot q into disp_out[q]
 *   dens_out : optional device [nsnap][batch][n_mesh^3]: delta_j likewise
 *   dJ_ddisp : optional device [nsnap][batch][3][n_ptcl^3], dJ/dx_j
 *   dJ_ddens : optional device [nsnap][batch][n_mesh^3], dJ/d delta_j
 * Every following pm_adjoint adds the cotangents of snapshot q, read when the reverse pass
 * reaches step j (so they may be written between pm_forward and pm_adjoint), to those of
 * the final state.  The buffers stay owned by the caller and must outlive their use.
 * Momenta of the snapshots: pm_set_snapshot_momenta.  Drops a captured pm_gradient_graph
 * and the snapshot momenta.  Errors: PM_ERR_ARG for a bad count or step list.
 */
int pm_set_snapshots(pm_ctx* ctx, int nsnap, const int* steps, void* disp_out, void* dens_out, const void* dJ_ddisp,
                     const void* dJ_ddens);

/*
 * Momenta of the states observed by pm_set_snapshots (Sec. 2.4: an objective on z_j =
 * (x_j, p_j)), the full-step momentum p_j after the kick K2_j (p_0 the initial momentum).
 *   mom_out : optional device [nsnap][batch][3][n_ptcl^3]: every following pm_forward writes
 *             p_j of snapshot q into mom_out[q]
 *   dJ_dmom : optional device [nsnap][batch][3][n_ptcl^3]: dJ/dp_j, added by every following
 *             pm_adjoint where the reverse pass holds p_j: the reverse kick K2_j, which made
 *             p_j, sees pi + dJ/dp_j, the reverse kick K1_{j+1} pi alone (Eq. 49)
 * Null pointers clear the respective part.  Errors: PM_ERR_STATE without snapshots.
 */
int pm_set_snapshot_momenta(pm_ctx* ctx, void* mom_out, const void* dJ_dmom);

/*
 * Positions observed between steps (Sec. 2.4: observations need not fall on the time
 * steps).  For a scale factor a inside step j + 1 (a_j < a <= a_{j+1}) the displacement is
 * that of the step's drift stopped at a,
 *   s(a) = s_j + Dp_j(a) p_{j+1/2},   Dp_j(a) = [D1(a) - D1(a_j)] / G_D(a_{j+1/2})
 * (the FastPM drift factor of Eq. 15 with a in place of a_{j+1}).
 *   na       : 0..PM_MAX_SNAPSHOTS; 0 clears
 *   a        : host [na] doubles, strictly ascending in (a0, a1]
 *   disp_out : optional device [na][batch][3][n_ptcl^3]: every following pm_forward writes
 *              s(a_q)
 *   dens_out : optional device [na][batch][n_mesh^3]: delta at q + s(a_q) (the same
 *              deterministic fixed-point CIC deposit as pm_op_density)
 *   dJ_ddisp, dJ_ddens : optional device cotangents on s(a_q) and delta(a_q): every following
 *              pm_adjoint adds u = dJ/dx(a) (the density part through the CIC weight
 *              gradient at x(a)) to xi_j and Dp_j(a) u to pi_{j+1/2}, with the theta term
 *              (u . p_{j+1/2}) dDp_j/dOmega_m
 * Drops a captured pm_gradient_graph.  Errors: PM_ERR_ARG for a bad count or a list.
 */
int pm_set_interp_snapshots(pm_ctx* ctx, int na, const double* a, void* disp_out, void* dens_out,
                            const void* dJ_ddisp, const void* dJ_ddens);

/*
 * The 64-bit fixed-point state of a context created with fixed_state = 1: displacement
 * U = s / l 2^40 and momentum W = p / l 2^36 (l the cell size), device [batch][3][n_ptcl^3]
 * each (either may be null).  After pm_forward it is the final state; after pm_adjoint the
 * initial state recovered by the reverse pass, equal bit for bit to the one pm_forward
 * started from.  Errors: PM_ERR_STATE for a context without the fixed-point state.
 */
int pm_get_fixed_state(pm_ctx* ctx, long long* disp_fixed, long long* mom_fixed);

/* Initial state at a0 of the context's lpt_order (Sec. 2.1, Eq. 2): s0 = D1 s1 (+ D2 s2),
 * p0 = a^2 H (D1' s1 (+ D2' s2)).  s0_out, p0_out: optional (null: not written),
 * [batch][3][n_ptcl^3].  Clears the forward state like the other operators. */
int pm_op_ic(pm_ctx* ctx, void* s0_out, void* p0_out);

/* ------------------------------------------------------------------------------------
 * Fault injection on the host, for tests of the error paths (no GPU fault is involved).
 * ----------------------------------------------------------------------------------*/

/* Make the device allocation after `after` more successful ones fail with PM_ERR_OOM as
 * if cudaMalloc had failed (no CUDA call is made for it); after < 0 disarms.  Process-wide;
 * the failing allocation disarms it. */
int pm_debug_fail_alloc(long long after);

/* Device bytes held by all live contexts of this process (the allocation-free entry point's
 * fixed array is not counted). */
long long pm_debug_live_bytes(void);

/* Spin limit of the first mbarrier wait of every CTA of the context's TMA-staged FFT passes
 * (spins < 0 restores the normal limit of 2^24 polls; 0 gives up at once, so that the
 * kernels take their timeout path: each CTA sets the flag, waits, bounded, for the copies
 * it has in flight and returns).  PM_ERR_ARG for a null context. */
int pm_debug_first_wait(pm_ctx* ctx, int spins);

/* ------------------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this is a service for
 * callers that cannot call cudaMalloc -- code whose device memory belongs entirely to its
 * own pool allocator (a framework's caching allocator, a server with a fixed memory
 * budget), where a foreign allocation fails or fragments the pool, and loops that must
 * not pay for cudaMalloc/cudaFree, which can synchronise the device.
 * ----------------------------------------------------------------------------------*/

/* Largest mesh (cells) pm_density_noalloc accepts: 128^3.  Its int64 accumulator is a
 * fixed 16 MiB array in the library's device memory, held by every GPU that loads the
 * library until the process exits. */
#define PM_NOALLOC_MAX_CELLS (128LL * 128 * 128)

/*
 * CIC overdensity delta = rho - 1 of particles at x = q + disp (the same deterministic
 * int64 fixed-point deposit as pm_op_density, FP32 only, one instance), using no device
 * allocation and no context.
 *   box      : periodic box side in Mpc/h
 *   n_mesh   : mesh nodes per side, power of two, n_mesh^3 <= PM_NOALLOC_MAX_CELLS
 *   n_ptcl   : particles per side, power of two >= 4, dividing n_mesh
 *   disp     : device, float [3][n_ptcl^3] displacements (caller-owned)
 *   dens_out : device, float [n_mesh^3] (caller-owned)
 *   stream   : a cudaStream_t (0 = legacy default stream)
 * Returns PM_ERR_ARG for bad sizes, including n_mesh^3 > PM_NOALLOC_MAX_CELLS (use
 * pm_op_density with a context for larger meshes).  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device current); make that
 * first call before any stream capture.  Every call clears and reuses the same array, so
 * calls that overlap on one GPU race with each other: serialise them (one stream).
 */
int pm_density_noalloc(double box, int n_mesh, int n_ptcl, const float* disp, float* dens_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PMGB_PM_H */
