/*
 * flame.h -- C ABI of the GB300 (sm_103a) spectral stepper for the
 * Sivashinsky-type model of an expanding spherical flame
 * (V. Karlin, "Global communications in multiprocessor simulations of
 * flames", Sec. 2 eq. (SivCurv1c) and Sec. 3).
 *
 * Model (eq. (SivCurv1c), forcing f = 0, r0(t) = t, Sec. 2):
 *   d Phi_k/dt = omega_k(t) Phi_k + c(t) [|grad Phi|^2]_k,
 *   omega_k(t) = -|kappa|^2/r0^2 + gamma |kappa|/(2 r0),  c(t) = 1/(2 r0^2),
 *   kappa = (s1 k1, s2 k2)   (s1 = s2 = theta_pi as printed in eq. (SivCurv1c)).
 * The quadratic term of eq. (SivCurv1c), -theta_pi^2/(2 r0^2) sum_l
 * l.(k-l) Phi_l Phi_{k-l}, is exactly c(t) times the coefficient of
 * |grad Phi|^2; it is evaluated through zero-padded FFTs (the augmented
 * array of Sec. 3, alias-free because N_i >= 4 K_i + 1).
 *
 * Grid and coefficients: x_i = 2 pi j_i / N_i on an N1 x N2 (theta, phi) grid,
 * Phi(x) = sum_k Phi_k exp(i k.x).
 *
 * STATE LAYOUT ("compact box"): the retained half spectrum k1 = -K1..K1,
 * k2 = 0..K2, stored COLUMN-MAJOR: element (k1, k2) at index
 * k2 * (2 K1 + 1) + (k1 + K1), i.e. k1 fastest (an array of shape
 * (K2 + 1, 2 K1 + 1) in C order); complex interleaved (re, im): double2 for
 * FLAME_FP64, float2 for FLAME_FP32_MIXED; (2 K1 + 1) * (K2 + 1) entries.
 * Column-major keeps every read of the step contiguous: the column passes
 * read whole columns of the state.  The k2 = 0 column is Hermitian
 * (Phi_{-k1,0} = conj(Phi_{k1,0}), the symmetrization of Sec. 3); the k = 0
 * entry is ignored and written as 0: the mean mode Phi_0 lives in a separate
 * double.  The time t is a double on the device.
 *
 * OWNERSHIP: the caller owns every buffer passed in (device memory unless
 * stated).  A handle owns its plan tables, its workspace and its captured
 * graphs.  All calls are asynchronous on the given stream (a cudaStream_t
 * passed as void*; NULL = the legacy default stream) except flame_create,
 * flame_destroy and flame_sync_status, which synchronise.
 *
 * ERRORS: no call aborts.  A call that returns a non-OK status has enqueued
 * no work on the stream.  flame_last_error() gives a thread-local message for
 * the last failing call.  Errors detected on the device (non-finite values;
 * out-of-range indices in the index-checking build) set status words in the
 * handle, read and cleared by flame_sync_status().
 *
 * A handle is not thread-safe: calls on one handle must not overlap in time
 * on the host, and two enqueued calls on one handle must be ordered (same
 * stream or an event), because they share the handle's workspace.
 */
#ifndef FLAME_H
#define FLAME_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FLAME_OK = 0,
    FLAME_EINVAL = 1,        /* bad argument (null pointer, size, params)   */
    FLAME_ENOMEM = 2,        /* device or host allocation failed            */
    FLAME_ECUDA = 3,         /* a CUDA runtime call failed                  */
    FLAME_EUNSUPPORTED = 4,  /* valid request the library does not handle   */
    FLAME_ETIMEOUT = 5,      /* a bounded device-side wait ran out          */
    FLAME_ENONFINITE = 6,    /* a step produced NaN or Inf                  */
    FLAME_EBOUNDS = 7        /* index-checking build: an index was outside
                                its array (the access was skipped)          */
} flame_status;

typedef enum {
    FLAME_FP64 = 0,          /* everything in double precision              */
    FLAME_FP32_MIXED = 1     /* FFTs and pointwise work in FP32; twiddles
                                generated in FP64; mean mode, time and the
                                step coefficients in FP64                    */
} flame_precision;

/* Test modes (flags): drop one of the two terms of eq. (SivCurv1c). */
#define FLAME_LINEAR_ONLY 1u
#define FLAME_NONLINEAR_ONLY 2u

typedef struct {
    int n_theta;       /* N1, power of two, 16..4096                        */
    int n_phi;         /* N2, power of two, 32..8192                        */
    int K1, K2;        /* retained harmonics; 0 = floor((N-1)/4); 4K+1 <= N */
    double gamma;      /* density contrast gamma = 1 - rho_b/rho_u          */
    double theta_pi;   /* integer theta_pi of eq. (SivCurv1c)               */
    double s1, s2;     /* kappa = (s1 k1, s2 k2); 0 = theta_pi              */
    double t0;         /* initial time (r0 = t), t0 > 0                     */
    double dt;         /* explicit Euler step, dt > 0                       */
    flame_precision prec;
    unsigned flags;    /* FLAME_LINEAR_ONLY, FLAME_NONLINEAR_ONLY or 0      */
} flame_params;

typedef struct flame_ctx *flame_t;

/* Creates a handle: validates params (EINVAL / EUNSUPPORTED), resolves K and
 * s, builds the FP64-generated twiddle tables and allocates the workspace on
 * the current CUDA device (ENOMEM, ECUDA).  *out is set only on success.
 * Synchronises the device.
 *
 * It also tunes the handle (see flame_tuning, flame_fused_steps) and, unless
 * FLAME_L2_PERSIST=0, raises this process's persisting-L2 set-aside
 * (cudaLimitPersistingL2CacheSize, a limit of the CUDA context) to the
 * state's size where the device allows it: the column passes then launch
 * with a persisting access window over the caller's state, which is a cache
 * hint only (results are identical either way).  Environment: FLAME_AUTOTUNE=0
 * keeps the default kernel variants, FLAME_FORCE_VARIANTS=a,b fixes them,
 * FLAME_FUSE=0 keeps the column passes of consecutive steps separate,
 * FLAME_BATCH_TMA=1 lets flame_step_batch use the tensor-store variants,
 * FLAME_TUNE_CACHE=path keeps the autotuner's choices in a JSON file. */
flame_status flame_create(const flame_params *params, flame_t *out);

/* Destroys a handle (NULL is accepted).  Synchronises the device. */
flame_status flame_destroy(flame_t h);

/* Copies the resolved parameters (K1, K2, s1, s2 filled in) into *out. */
flame_status flame_get_params(flame_t h, flame_params *out);

/* Kernel variants the autotuner chose for this handle (FP32 grids with
 * N1, N2/2 in 256..4096 are timed once per grid, precision and device at
 * creation, FLAME_AUTOTUNE=0 disables it): pass A 0 = cluster write-out
 * through distributed shared memory, 1 = direct stores, 2 = 8 points per
 * thread with the cluster write-out, 3 = write-out by tensor (TMA) stores,
 * 4 = one line per thread group (N1 <= 2048; pass C then takes the same
 * form); pass B 0 = 16 points per thread, 1 = 8 points per thread, 2 = 16
 * points per thread with the write-out by tensor stores, 3 = one line per
 * thread group (N2/2 <= 2048), 4 = as 2 with, for N2 = 8192, one exchange
 * of each row transform inside a warp (other N2: as 2).  flame_step_batch takes the fastest variants
 * other than the one-line ones (an ensemble fills the GPU without them),
 * unless FLAME_FORCE_VARIANTS fixes the variants.  EINVAL on null pointers. */
flame_status flame_tuning(flame_t h, int *pass_a_variant, int *pass_b_variant);

/* *enabled = 1 when flame_step with nsteps > 1 runs the column pass of each
 * step fused with the first column pass of the next (the same arithmetic as
 * separate steps, one HBM read of the state fewer per step).  Decided by the
 * autotuner at creation for FP32 grids with 256 <= N1 <= 4096;
 * FLAME_FUSE=0 disables it.  EINVAL on null pointers. */
flame_status flame_fused_steps(flame_t h, int *enabled);

/* Number of complex entries of the compact box, (2 K1 + 1) * (K2 + 1). */
size_t flame_state_len(flame_t h);

/* Standalone 2-D real FFTs over the handle's N1 x N2 grid, unnormalised,
 * in the handle's precision (double or float):
 *   r2c: spec_out[k1][k2] = sum_{j1,j2} real_in[j1][j2]
 *                            exp(-2 pi i (k1 j1/N1 + k2 j2/N2)),
 *        real_in N1 x N2 row-major, spec_out N1 x (N2/2+1) complex row-major.
 *   c2r: real_out[j1][j2] = sum over the Hermitian-extended spectrum of
 *        spec_in[k1][k2] exp(+2 pi i (...)), so c2r(r2c(x)) = N1 N2 x.
 *        spec_in is not modified (the handle's workspace is used).
 * The 2-D transform is the tensor product of 1-D ones (Sec. 2): rows, then
 * columns for r2c; columns, then rows for c2r (Sec. 3).  EINVAL on null
 * pointers.  Buffers must be 16-byte aligned. */
flame_status flame_fft_r2c(flame_t h, const void *real_in, void *spec_out,
                           void *stream);
flame_status flame_fft_c2r(flame_t h, const void *spec_in, void *real_out,
                           void *stream);

/* Initial state from a physical-space perturbation.  Sec. 2 starts its runs
 * from Phi(theta, phi, t0) = eps eta(theta, phi), with |eta| <= 1 drawn for
 * every grid point; this call projects such a field on the retained modes:
 *   field     N1 x N2 real, row-major (j1 slowest), device memory, in the
 *             handle's real type (double for FLAME_FP64, float otherwise);
 *   state     the compact box (ABI layout, the handle's complex type):
 *             state(k1, k2) = (1/(N1 N2)) sum_{j1,j2} field[j1][j2]
 *                             exp(-2 pi i (k1 j1/N1 + k2 j2/N2))
 *             for |k1| <= K1, 0 <= k2 <= K2, except that the k = 0 slot is
 *             0 and the k2 = 0 column's k1 < 0 entries are the conjugates of
 *             its k1 > 0 entries (the step's symmetrisation, Sec. 3);
 *   mean_mode one FP64 device value, the field's average (the k = 0
 *             coefficient).
 * The transform is flame_fft_r2c's (rows, then columns) into the handle's
 * spectrum workspace, which flame_fft_c2r also uses: calls on one handle
 * must be ordered (one stream).  EINVAL on null pointers.  Buffers must be
 * 16-byte aligned. */
flame_status flame_state_from_field(flame_t h, const void *field, void *state,
                                    double *mean_mode, void *stream);

/* Advances the state by nsteps explicit Euler steps of eq. (SivCurv1c):
 *   Phi_k <- Phi_k + dt (omega_k(t_n) Phi_k + c(t_n) ghat_k + f_k)   (k != 0),
 *   Phi_0 <- Phi_0 + dt (c(t_n) ghat_0 + f_0),
 * where ghat is the box part of the normalised analysis of |grad Phi|^2 and
 * f the forcing set by flame_set_forcing (f = 0 unless set, as in the
 * paper's runs),
 * followed by the symmetrization of the k2 = 0 column (Sec. 3) and
 * t <- t0 + (n + 1) dt with n = round((t - t0)/dt).
 * state: compact box (see above), in place.  mean_mode, t: one device double
 * each, in place.  nsteps >= 0 (0 is a no-op).  For nsteps > 1 the step
 * sequence is replayed from a captured CUDA graph (captured on first use per
 * (state, mean_mode, t, nsteps, forcing) binding; the handle caches 8 and
 * keeps the ones it evicts until flame_destroy, so that an eviction never
 * waits for the device, except once every 64 evictions).  Non-finite results set
 * FLAME_ENONFINITE in the handle's device status word. */
flame_status flame_step(flame_t h, void *state, double *mean_mode, double *t,
                        int nsteps, void *stream);

/* Records the averaged diagnostics of Sec. 2 on the device at every step of
 * the handle's later step calls (flame_step, flame_step_heun, flame_step_if,
 * flame_step_batch), from the mean-mode work of the column pass at no extra
 * pass over memory.  rec: caller-owned device array of 4 * capacity doubles
 * (NULL stops recording); the step with lattice index n (t_n -> t_{n+1},
 * n = round((t_n - t0)/dt)) writes entry n mod capacity:
 *   rec[4e + 0] = t_n,
 *   rec[4e + 1] = Phi_0(t_n), the mean mode (mean radius = t_n + Phi_0),
 *   rec[4e + 2] = <Phi_t>(t_n) = c(t_n) mean(|grad Phi_n|^2) + f_0, the
 *                 averaged front velocity dPhi_0/dt of eq. (SivCurv1c),
 *   rec[4e + 3] = the surface area A(t_n) of flame_area's definition when
 *                 with_area != 0 (else NaN).
 * The values describe the state entering the step (for two-stage schemes,
 * the first stage's).  With the area, the first stage's row pass runs a
 * variant that also synthesises Phi on its rows and sums R sqrt(R^2 +
 * |grad Phi|^2) there (one more inverse row transform, one CTA per SM),
 * and the column pass adds the row sums; FP64 rows too long for that
 * variant's shared memory (N2 = 8192) use the separate area kernels before
 * the step.  flame_step_batch records no area (NaN).  The library keeps the
 * pointer; graphs are captured per record binding.  EINVAL for a null handle
 * or capacity < 1 with a non-NULL rec. */
flame_status flame_set_record(flame_t h, double *rec, int capacity, int with_area);

/* flame_step on HOST buffers: copies the state in, advances it by nsteps
 * explicit Euler steps (flame_step's arithmetic and kernels) and copies it
 * back, overlapping the copies with the step: the state goes in by column
 * chunks on a copy stream of the handle and the first pass A runs on each
 * chunk as it lands; the last pass C runs by column-pair chunks, each copied
 * out as soon as it is done.
 *   host_state  the compact box (ABI layout, the handle's complex type) in
 *               host memory, in place; pinned memory (cudaHostAlloc or
 *               cudaHostRegister) lets the copies run asynchronously and
 *               overlap (pageable memory works but serialises them);
 *   host_mean, host_t  one host double each, in place.
 * The host buffers may be read or written until the stream reaches the end
 * of the call (synchronise the stream before using them).  The handle
 * allocates a device copy of the state and a copy stream on the first call.
 * The per-step record and forcing apply as in flame_step.  EINVAL on null
 * pointers or nsteps < 0; ENOMEM if the device copy cannot be allocated. */
flame_status flame_step_host(flame_t h, void *host_state, double *host_mean, double *host_t,
                             int nsteps, void *stream);

/* Sets the forcing term f_k(t) of eq. (SivCurv1c) (Sec. 2; the paper's runs
 * have f = 0) for the handle's later step calls (flame_step, flame_step_heun,
 * flame_step_if, flame_step_batch and the adjoint's forward recomputation):
 *   forcing   NULL (f_k = 0) or a caller-owned device box in the state's
 *             layout and precision holding f_k for 0 < |k| in the box (the
 *             k = 0 entry is ignored; the k2 = 0 column should be Hermitian
 *             like the state's).  The library keeps the pointer, not a
 *             copy: the caller keeps the buffer valid while it steps and may
 *             change its contents between calls (a time-dependent forcing
 *             is applied that way, constant within a call).
 *   forcing0  f_0, the mean mode's forcing (FP64).
 * The term enters the right-hand side additively.  Constant forcing leaves
 * the step's Jacobian unchanged, so flame_adjoint stays the adjoint of the
 * forced step.  EINVAL for a null handle or a non-finite forcing0. */
flame_status flame_set_forcing(flame_t h, const void *forcing, double forcing0);

/* Advances the state by nsteps steps of Heun's method, the explicit
 * two-stage Runge-Kutta method of order 2, for eq. (SivCurv1c): a
 * higher-order alternative to flame_step's explicit Euler (the paper leaves
 * its integrator to its references).  With F the right-hand side of
 * flame_step (mean mode included) and t_n = t0 + n dt,
 *   k1 = F(Phi_n, t_n),  Phi* = Phi_n + dt k1,  k2 = F(Phi*, t_{n+1}),
 *   Phi_{n+1} = Phi_n + (dt/2) (k1 + k2),  t <- t_{n+1}.
 * Each stage is one evaluation of the right-hand side (passes A, B) and a
 * pass C whose epilogue applies the stage: the predictor keeps Phi_n, the
 * corrector writes (Phi_n + Phi* + dt k2)/2.  Multi-step calls are
 * graph-captured like flame_step's.  Uses the handle's area workspace and
 * scratch to carry Phi_n between the stages: calls on one handle must be
 * ordered (one stream).  Arguments and errors as flame_step. */
flame_status flame_step_heun(flame_t h, void *state, double *mean_mode, double *t,
                             int nsteps, void *stream);

/* Advances the state by nsteps integrating-factor second-order Runge-Kutta
 * steps (Lawson's method over Heun's scheme) of eq. (SivCurv1c): the
 * stiffness-robust integrator (the paper leaves its time integration to its
 * references).  The linear part omega_k(t) Phi_k is propagated exactly by
 *   E_k = exp(int_{t_n}^{t_{n+1}} omega_k) = exp(-|kappa|^2 (1/t_n - 1/t_{n+1})
 *         + (gamma |kappa|/2) ln(t_{n+1}/t_n))          (r0 = t),
 * and the rest, N = c(t) ghat + f, by Heun's method in the propagated frame:
 *   Phi* = E (Phi_n + dt N(Phi_n, t_n)),
 *   Phi_{n+1} = E (Phi_n + (dt/2) N(Phi_n, t_n)) + (dt/2) N(Phi*, t_{n+1}),
 * the mean mode with E = 1, each stage symmetrised (Sec. 3), t <- t_{n+1}.
 * The linear problem is solved exactly and the step stays stable for
 * dt |omega|_max well above explicit Euler's bound of 2.  E is evaluated per
 * mode in the kernel's precision from FP64 step coefficients.  Same
 * arguments, workspace use and errors as flame_step_heun. */
flame_status flame_step_if(flame_t h, void *state, double *mean_mode, double *t,
                           int nsteps, void *stream);

/* Enqueues one pass of one step: pass 0 = A (derivatives and column
 * inverse FFT), 1 = B (row inverse FFT, |grad Phi|^2, row forward FFT),
 * 2 = C (column forward FFT, linear operator, Euler update, symmetrization,
 * mean mode, time), 3 = C fused with pass A of the next step (only when
 * flame_fused_steps reports 1, else EUNSUPPORTED).  Calling passes 0, 1, 2
 * in order on one stream is exactly flame_step(h, state, mean_mode, t, 1,
 * stream); 0, then (1, 3) n - 1 times, then 1, 2 is exactly flame_step(...,
 * n, ...).  The split exists so that each kernel can be timed with events on
 * the launching stream.  EINVAL for pass outside 0..3 or null pointers. */
flame_status flame_step_pass(flame_t h, int pass, void *state, double *mean_mode, double *t,
                             void *stream);

/* Advances nflames independent flames (each with its own handle, state,
 * mean mode and time; grids may differ; all handles must have the same
 * precision) by nsteps steps.  Flames of equal grid size are grouped so that
 * each pass is one launch per size class; the steps run as a captured CUDA
 * graph of 8 steps (fewer for a shorter call) replayed, one per binding of
 * (handles, states, mean modes, times).  A new binding uploads its
 * descriptors asynchronously on `stream` (from a pinned staging buffer of
 * the first handle); only growing the first handle's descriptor buffers
 * synchronises that stream.  Results equal nflames separate flame_step
 * calls (the same bits where the flame and its size class run the same
 * kernel variants; where the autotuner gave a small grid's single flame the
 * one-line variants, to FP32 rounding).  hs, states, mean_modes and ts are HOST arrays of nflames entries
 * (device pointers).  Calls with the same first handle must be ordered
 * (one stream). */
flame_status flame_step_batch(const flame_t *hs, void *const *states,
                              double *const *mean_modes, double *const *ts,
                              int nflames, int nsteps, void *stream);

/* Flame surface area of the state at time *t (project-defined objective,
 * the equatorial surface element of the model's geometry):
 *   A = sum_grid (2 pi)^2/(N1 N2 s1 s2) R sqrt(R^2 + |grad Phi|^2),
 *   R = r0(t) + Phi(x).
 * Writes A (double, device) to area_out.  If dA_dstate is not NULL it
 * receives dA/dPhi_k on the compact box (precision of the handle) for the
 * full-spectrum inner product <X, Y> = Re sum_{all k} conj(X_k) Y_k, and
 * dA_dmean (device double, may be NULL) receives dA/dPhi_0. */
flame_status flame_area(flame_t h, const void *state, const double *mean_mode,
                        const double *t, double *area_out, void *dA_dstate,
                        double *dA_dmean, void *stream);

/* Reverse-mode gradient through nsteps Euler steps (the discrete adjoint of
 * flame_step) starting from (state0, mean0, t_start = t0 of the handle's
 * lattice, read from the device double t_start):
 *   given lambda_T = dL/dPhi(T) (compact box) and lambda0_T = dL/dPhi_0(T),
 *   returns grad_state0 = dL/dPhi(t_start) (compact box), grad_mean0 =
 *   dL/dPhi_0(t_start) and grad_gamma = dL/dgamma (device doubles).
 * The forward trajectory is recomputed from checkpoints stored every
 * ckpt_every steps (1 <= ckpt_every <= nsteps).  Gradients use the
 * full-spectrum inner product of flame_area.  state0, lambda_T and
 * grad_state0 are device buffers in the handle's precision; mean0,
 * t_start, lambda0_T, grad_mean0, grad_gamma are device doubles. */
flame_status flame_adjoint(flame_t h, const void *state0, const double *mean0,
                           const double *t_start, int nsteps, int ckpt_every,
                           const void *lambda_T, const double *lambda0_T,
                           void *grad_state0, double *grad_mean0,
                           double *grad_gamma, void *stream);

/* flame_step without any allocation (the paper has no counterpart: this is
 * for callers of this library that cannot allocate device memory -- code
 * running inside a host callback or a hook that forbids cudaMalloc, under a
 * memory manager that owns the whole device, or anywhere the allocator must
 * not be re-entered).  No handle is needed: params are validated as in
 * flame_create, and state, mean_mode and t are the caller's buffers exactly
 * as for flame_step, advanced by nsteps explicit Euler steps with the same
 * kernels and the same results.  The twiddle tables, both step workspaces
 * and the status word live in one static device array of 8 MiB that the
 * library image reserves on every GPU that loads it, until the process exits.
 * Grids whose scratch does not fit (roughly N1 x (K2+1) above 170k entries in
 * FP64, 340k in FP32, e.g. 512 x 1024 FP64 fits, 4096 x 8192 does not) are
 * rejected with FLAME_EUNSUPPORTED and a message giving the bytes needed.
 * The function calls no cudaMalloc, cudaFree or other allocating routine.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls on a device share the array and it
 * keeps the last call's contents; each call rewrites the tables and
 * workspaces it reads and clears the status word, but calls whose work
 * overlaps on the GPU (unordered streams) race on the array.  Non-finite
 * values are not reported (there is no handle to read them from). */
flame_status flame_step_noalloc(const flame_params *params, void *state, double *mean_mode,
                                double *t, int nsteps, void *stream);

/* Measured FMA throughput of the current device (the paper has no
 * counterpart: a measurement utility for reporting the FP64 step against the
 * FP64 rate it is bound by).  prec: FLAME_FP64 or FLAME_FP32_MIXED (scalar
 * FP32 FMA).  Runs a calibration kernel of 8 independent FMA chains per
 * thread on every SM, best of 3 timed runs, and writes the rate in FLOP/s
 * (2 per FMA) to *flops_per_s (host).  Allocates a scratch buffer and a
 * stream and synchronises.  EINVAL on a bad argument, ECUDA on a CUDA error. */
flame_status flame_fma_peak(int prec, double *flops_per_s);

/* Index-checking build.  A library compiled with -DFLAME_DEBUG_BOUNDS
 * (paper_0911_2889_gb300/build.py, debug=True: libflame_debug.so) checks
 * every computed global-memory index of the step passes, the standalone FFT
 * passes and flame_state_from_field against the extent of its array before
 * the access; a failing check skips the access and records FLAME_EBOUNDS,
 * with the check's site, index and extent, in the handle's status words
 * (reported by flame_sync_status).  It stands in for a memory checker, and
 * the kernels then run slower.
 *
 * flame_debug_bounds_probe runs one such check of (index, extent) on the
 * stream with no memory access at all: index outside [0, extent) makes the
 * next flame_sync_status return FLAME_EBOUNDS.  It lets a test see the
 * reporting path without any out-of-range access.  The normal build has no
 * checks and returns FLAME_EUNSUPPORTED.  EINVAL on a null handle. */
flame_status flame_debug_bounds_probe(flame_t h, int index, int extent, void *stream);

/* Synchronises the handle's device status words and returns the status they
 * hold (FLAME_OK, FLAME_ENONFINITE, FLAME_ETIMEOUT or, in the index-checking
 * build, FLAME_EBOUNDS); clears them. */
flame_status flame_sync_status(flame_t h);

/* Static description of a status code. */
const char *flame_status_str(flame_status s);

/* Thread-local message of the last failing call on this host thread. */
const char *flame_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FLAME_H */
