/*
 * gl.h -- C-ABI of the B300 oblate-planet transit library (libgl.so).
 *
 * The library evaluates relative-flux light curves of a planet shaped as an
 * oblate spheroid at arbitrary orientation, for many parameter sets and many
 * exposure times at once, on one NVIDIA B300 (sm_103a).
 *
 * Method (arxiv 2410.05408):
 *   - sky-plane projection of the spheroid: Sec. 2, Eqs. dx, dy1, dy2, with the
 *     oblate case b = c of Appendix A and the mean-radius parameter of Sec. 3;
 *   - occulted stellar flux for quadratic limb darkening by Green's theorem:
 *     the integrands f_flat, f_lin, f_quad of Sec. 2 summed over the part of
 *     the projected boundary inside the stellar disk plus the part of the limb
 *     inside the projection (Sec. 2 replaces the latter by "snapping"; here the
 *     boundary is split exactly at the ellipse/limb crossings);
 *   - orbit: Sec. 2 uses a circular orbit; here a Keplerian orbit with
 *     eccentricity e and argument of periastron omega, t0 = time of conjunction
 *     (true anomaly pi/2 - omega), reducing to Sec. 2 for e = 0, omega = pi/2.
 *
 * Conventions.  Lengths in stellar radii, times in days, angles in radians.
 * Sky frame (Sec. 2): z along the line of sight from the observer to the star,
 * y along the transit chord, x completing a right-handed frame.  A planet with
 * z > 0 (behind the star) occults nothing.
 *
 * Memory.  Every array argument may live in host memory (pageable or pinned) or
 * in device memory of the context's GPU; the library finds out with
 * cudaPointerGetAttributes.  The caller owns every buffer; the library never
 * frees or retains them after the call returns.  The context owns its own
 * device workspace (grow-only, freed by gl_context_destroy).
 *
 * Errors.  Every function returns GL_OK (0) or a negative GL_E* code; the
 * message of the last failure is kept per context (gl_last_error).  Invalid
 * physical parameters of one set are not a call error: that set's outputs are
 * NaN and GL_ENUMERIC is reported by the next gl_sync.
 *
 * Streams.  Calls are asynchronous on the given CUDA stream (NULL = the legacy
 * default stream) when every buffer is in device memory.  When any input or the
 * output is in host memory, the call returns only after the outputs are in
 * place.  A context must not be used from two host threads at once.
 */
#ifndef GL_H
#define GL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GL_OK 0
#define GL_EINVAL (-1)    /* bad argument: NULL pointer, negative size, ... */
#define GL_ENOMEM (-2)    /* device workspace could not be allocated */
#define GL_ECUDA (-3)     /* a CUDA runtime call failed */
#define GL_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define GL_ENUMERIC (-5)  /* a parameter set was physically invalid (output NaN) */
#define GL_EIO (-6)       /* a file could not be written or read, or is not a checkpoint */

typedef enum {
  GL_FP64 = 0,  /* plain FP64 path: everything in double */
  GL_FP32C = 1, /* FP32 quadrature with compensated sums; Kepler solve,
                   intersection roots and the exposure sum in FP64 */
} gl_precision;

typedef struct gl_context gl_context;

/* Parameter sets, structure of arrays, n_sets entries each (Sec. 3, Table priors):
 *   t0      time of conjunction (days)          period  orbital period (days)
 *   a_rs    semi-major axis / R*                b       impact parameter at conjunction,
 *                                                       b = a_rs cos(i) (1-e^2)/(1+e sin w)
 *   ecc     eccentricity, 0 <= e < 1            omega   argument of periastron (rad)
 *   k       mean radius ratio r = (a b c)^(1/3)/R* (Sec. 3); the equatorial radius is
 *           R_eq = k (1-f)^(-1/3) and the polar radius R_eq (1-f)
 *   f       flattening (R_eq - R_pol)/R_eq, 0 <= f < 1 (Sec. 1)
 *   eta     rotation about y' (tilt of the spin axis out of the sky plane), rad
 *   xi      rotation about z' (position angle of the spin axis on the sky), rad;
 *           the projected spin axis points along (cos xi, -sin xi) in (x, y)
 *   u1, u2  quadratic limb darkening, I(mu) = 1 - u1 (1-mu) - u2 (1-mu)^2
 * Optional (NULL: the oblate spheroid b = c of the fits, Appendix A):
 *   g       equatorial flattening of a general triaxial ellipsoid (Sec. 2):
 *           semi-axes c (largest, along z'), b = c (1-g) (y'), a = c (1-f) (x'),
 *           k = (a b c)^(1/3), so c = k ((1-f)(1-g))^(-1/3); 0 <= g < 1
 *   zeta    rotation about x', rad (no effect when g = 0)
 */
typedef struct {
  int64_t n_sets;
  const double *t0, *period, *a_rs, *b, *ecc, *omega;
  const double *k, *f, *eta, *xi;
  const double *u1, *u2;
  const double *g, *zeta;   /* optional, may be NULL */
} gl_params;

/* Exposure times.
 *   t         mid-exposure times (days).
 *   offsets   NULL: every set uses the same grid t[0 .. n_times) and the output is
 *             n_sets x n_times, row-major.  Otherwise int64 offsets[n_sets + 1],
 *             non-decreasing, offsets[0] = 0: set s owns t[offsets[s] ..
 *             offsets[s+1]) and the output has the same layout (CSR).
 *   n_times   shared-grid length (ignored when offsets != NULL).
 *   n_total   number of exposures = length of out: n_sets * n_times for a shared
 *             grid, offsets[n_sets] otherwise.  Must be < 2^31.
 *   exptime   per-set exposure length (days, >= 0).
 *   nsuper    per-set number of sub-exposures (int32, >= 1), or NULL to use
 *             nsuper_all for every set.
 * Sub-exposure q of an exposure at t sits at t + ((q + 1/2)/n - 1/2) exptime and
 * the exposure's flux is the mean of its sub-exposure fluxes (the paper does not
 * describe supersampling; this is the midpoint rule).  A time that is NaN or
 * infinite lies outside the transit window, so its flux is 1; for an orbit so
 * tight that its window spans the whole orbit, such a time gives NaN instead.
 */
typedef struct {
  const double *t;
  const int64_t *offsets;
  int64_t n_times;
  int64_t n_total;
  const double *exptime;
  const int32_t *nsuper;
  int32_t nsuper_all;
} gl_times;

/* Create a context bound to CUDA device `device`; uploads the quadrature node
 * tables to that device.  *ctx receives the handle.  GL_EINVAL if ctx is NULL or
 * the device does not exist, GL_ECUDA on a runtime failure. */
int gl_context_create(gl_context **ctx, int device);

/* Wait for the context's outstanding work, free its workspace and the handle.
 * Passing NULL is a no-op returning GL_OK. */
int gl_context_destroy(gl_context *ctx);

/* Message of the last failure on this context ("" if none).  The pointer stays
 * valid until the next call on the context. */
const char *gl_last_error(const gl_context *ctx);

/* Light curves of a batch of parameter sets (Sec. 2 method, see header top).
 *   out[j]  relative flux of exposure j (1 exactly when no sub-exposure occults
 *           the star), FP64, n_total entries, layout as described for gl_times.
 *   prec    GL_FP64 or GL_FP32C.
 *   stream  cudaStream_t to run on, or NULL.
 * Returns GL_OK, GL_EINVAL (NULL pointer, negative size, nsuper < 1, n_total
 * inconsistent with a shared grid or >= 2^31, bad precision), GL_ENOMEM or
 * GL_ECUDA.  Parameter sets that are physically invalid (period <= 0, a_rs <= 0,
 * e outside [0,1), k <= 0, f outside [0,1), |cos i| > 1, non-finite values,
 * exptime < 0, nsuper < 1, limb darkening with no flux) yield NaN outputs and a
 * sticky GL_ENUMERIC reported by gl_sync. */
int gl_lightcurve_batch(gl_context *ctx, const gl_params *p, const gl_times *t, double *out,
                        gl_precision prec, void *stream);

/* Light curves of tidally locked bodies (Appendix B): the body frame turns with
 * the orbit, so the projected ellipse is recomputed for every sub-exposure from
 * the orbital angle alpha from conjunction (alpha = w + nu - pi/2 for the
 * Keplerian orbit; r cos alpha = x0 cos i - z sin i, r sin alpha = y0) and
 * beta = pi/2 - i, by the paper's Eqs. dx-locked, dy1-locked, dy2-locked; shapes
 * as in gl_params (oblate, or triaxial with g and zeta).  One thread per
 * exposure, FP64 Kepler per sub-exposure, the same quadrature as
 * gl_lightcurve_batch.  Same arguments, memory, stream and error rules as
 * gl_lightcurve_batch. */
int gl_lightcurve_locked(gl_context *ctx, const gl_params *p, const gl_times *t, double *out,
                         gl_precision prec, void *stream);

/* Relative flux for given sky positions, bypassing the orbit (geometry level
 * of Sec. 2).  All arrays have n entries:
 *   x0, y0, z       planet centre in the sky frame (stellar radii)
 *   k, f, eta, xi   shape and orientation as in gl_params
 *   u1, u2          limb darkening
 *   out             relative flux, FP64
 * Same memory, stream and error rules as gl_lightcurve_batch. */
int gl_flux_sky(gl_context *ctx, int64_t n, const double *x0, const double *y0,
                const double *z, const double *k, const double *f, const double *eta,
                const double *xi, const double *u1, const double *u2, double *out,
                gl_precision prec, void *stream);

/* Relative flux of a spherical planet of radius p (stellar radii) centred at
 * (x0, y0, z), quadratic limb darkening (u1, u2); n entries each, FP64.  The
 * circle case of the same Green's-theorem formulation (Sec. 2 integrands):
 * crossings, f_flat and f_quad in closed form, f_lin by the mapped Gauss-Legendre
 * rule on the symmetric half-arc (the FP32C order for GL_FP32C, the FP64 order for
 * GL_FP64).  It is the base term of the oblate-minus-spherical surrogate.  Same
 * memory, stream and error rules as gl_flux_sky; invalid inputs (p <= 0,
 * non-finite values, LD with no flux) give NaN and GL_ENUMERIC at gl_sync. */
int gl_flux_sphere(gl_context *ctx, int64_t n, const double *x0, const double *y0,
                   const double *z, const double *p, const double *u1, const double *u2,
                   double *out, gl_precision prec, void *stream);

/* Relative flux at sky positions by the paper's own integration scheme (Sec. 2),
 * for comparison with gl_flux_sky: composite Simpson's rule over `n_intervals`
 * uniform intervals (even, 2..2^24) of the ellipse angle, the boundary "snapped"
 * along its ray onto the limb wherever it lies outside the disk, and no
 * crossings.  The integrand has a kink where the boundary meets the limb, so the
 * error falls as n_intervals^-2 on partial overlaps.  GL_FP32C evaluates the
 * integrands in FP32 with compensated sums (the paper's single precision);
 * GL_FP64 in FP64.  Positions behind the star or with rho >= 1 + R_eq give 1.
 * Same arguments, memory, stream and error rules as gl_flux_sky; GL_EINVAL for an
 * odd or out-of-range n_intervals. */
int gl_flux_sky_simpson(gl_context *ctx, int64_t n, const double *x0, const double *y0,
                        const double *z, const double *k, const double *f, const double *eta,
                        const double *xi, const double *u1, const double *u2, double *out,
                        int n_intervals, gl_precision prec, void *stream);

/* Kipping (2013) map from (q1, q2) in [0,1]^2 to quadratic coefficients,
 * u1 = 2 sqrt(q1) q2, u2 = sqrt(q1) (1 - 2 q2) (cited in Sec. 3, Table priors,
 * note f; the formula is not printed in the paper).  Host arrays of n entries;
 * runs on the host, needs no context.  GL_EINVAL on NULL pointers or n < 0. */
int gl_q_to_u(int64_t n, const double *q1, const double *q2, double *u1, double *u2);

/* Wait for all work the context issued on `stream` and return the sticky status
 * of the device-side checks since the last gl_sync (GL_OK, GL_ENUMERIC or
 * GL_ETIMEOUT), clearing it. */
int gl_sync(gl_context *ctx, void *stream);

/* Number of kernel launches the context has issued since creation (for
 * accounting in benchmarks). */
int64_t gl_launch_count(const gl_context *ctx);

/* Workload counters of the light-curve kernel (gl_counts_read slots). */
#define GL_COUNT_EXPOSURES 0    /* exposures tested */
#define GL_COUNT_KEPT 1         /* exposures passing the FP32 window test */
#define GL_COUNT_IN_WINDOW 2    /* exposures inside the exact FP64 window */
#define GL_COUNT_KEPLER 3       /* exposures whose sub-exposures use the midpoint expansion */
#define GL_COUNT_ITEMS 4        /* sub-exposures of in-window exposures */
#define GL_COUNT_ITEM_KEPLER 5  /* sub-exposures with their own FP64 Kepler solve */
#define GL_COUNT_FULL 6         /* sub-exposures with the whole ellipse on the disk */
#define GL_COUNT_PARTIAL 7      /* sub-exposures needing the crossings */
#define GL_COUNT_SLOTS 8

/* Workload counting for benchmarks and tests.  While enabled, gl_lightcurve_batch
 * runs an instrumented instance of its kernel that adds to the GL_COUNT_* slots
 * (enabling resets them; no graph replay while counting).  GL_EINVAL on a NULL
 * context, GL_ECUDA on a runtime failure. */
int gl_counts_enable(gl_context *ctx, int on);

/* Copy the first n counters (int64) to `counts` after waiting for the device;
 * slots beyond GL_COUNT_SLOTS read 0.  GL_EINVAL on NULL pointers or n < 0. */
int gl_counts_read(gl_context *ctx, int64_t *counts, int n);

/* CUDA-graph replay of gl_lightcurve_batch (on by default).  When every buffer is
 * device memory and neither profiling nor counting is on, the step (per-set
 * constants + light-curve kernel) is captured once per distinct argument set
 * (pointers, sizes, precision; up to 16 kept, least recently used dropped) and
 * replayed with cudaGraphLaunch on the caller's stream.  Arguments are read when
 * the graph runs, so updating the parameter arrays in place between calls is
 * correct.  Turning it off drops the cached graphs.  GL_EINVAL on NULL. */
int gl_graphs_enable(gl_context *ctx, int on);

/* Number of graph replays the context has issued. */
int64_t gl_graph_launches(const gl_context *ctx);

/* Item pipeline of gl_lightcurve_batch (on by default).  With it on, the step
 * after the per-set constants is four flat kernels: window tests over every
 * exposure (flux 1 outside the transit window), one thread per kept exposure
 * (Kepler midpoint state, position and overlap class of each sub-exposure,
 * Sec. 2 geometry), the quadrature of every sub-exposure that meets the disk with
 * warps spread over the whole GPU, and each exposure's FP64 mean in
 * sub-exposure order.  With it off, a tile kernel takes consecutive exposures and does all of
 * this per tile.  The pipeline balances batches whose transits fall in few
 * places; its workspace (56 bytes per sub-exposure and 12 per exposure,
 * context-owned, grown on demand and kept) holds n_total x nsuper_all sub-exposures (16 per exposure
 * with per-set nsuper), at most `max_items` (0 = default 2^23); an exposure that
 * does not fit is finished by the thread holding it.  Every sub-exposure is
 * evaluated by the same compiled functions and every exposure summed in the same
 * order either way, so results are bit-identical with the pipeline on or off
 * and for any workspace size.  While counting (gl_counts_enable) the tile
 * kernel runs.  Drops the cached graphs.  GL_EINVAL on NULL or max_items
 * outside [0, 2^31). */
int gl_item_pipeline(gl_context *ctx, int on, int64_t max_items);

/* Result of gl_autotune. */
typedef struct {
  int threads;         /* threads per CTA of the light-curve kernel */
  int tile;            /* exposures per tile */
  int nodes;           /* Gauss-Legendre nodes per arc */
  double ms;           /* best step time (ms, CUDA events, warm) */
  double default_ms;   /* step time of the default configuration, 0 if inadmissible */
  double max_abs_err;  /* max |flux - FP64 path| of the chosen configuration */
  int candidates;      /* configurations tried */
  int admissible;      /* configurations within 0.9 x tolerance of the FP64 path */
  int quad_ctas_per_sm; /* item pipeline: resident CTAs per SM of the chosen quadrature
                           kernel (4: all registers, 8: 64 registers), else 0 */
  int exposure_block;  /* item pipeline: threads per CTA of the chosen exposure kernel
                          (256 or 64; 64 exposures per CTA either way), else 0 */
} gl_tune_report;

/* Autotuner of the light-curve kernel for the batch (p, t) at precision prec.
 * Candidates: 128 or 256 threads per CTA of the tile kernel (tile = threads,
 * 4 x threads items per round) -- or, with the item pipeline on, the two
 * quadrature kernels (all registers, 4 CTAs per SM; or 64 registers, 8 CTAs per
 * SM) times the two exposure kernels (256 or 64 threads per CTA) -- and, for
 * GL_FP32C, 16, 20, 24 or 28 Gauss-Legendre nodes per arc.  Each
 * candidate runs on the batch; only those whose max |flux - FP64 path| stays
 * within 0.9 x the precision's tolerance (1e-7 FP32C, 1e-10 FP64) are timed (CUDA
 * events, best of 5, each from a cold L2; as CUDA-graph replays when graphs are on,
 * the way later calls run) and the fastest is kept by the context for later calls at
 * that precision.  `out` (device memory, n_total doubles) receives the chosen
 * configuration's last result; the context holds one FP64 reference of n_total
 * doubles, and tuning briefly allocates a buffer of twice the L2 size.
 * Synchronises `stream`; must not be called during stream capture.
 * `rep` may be NULL.  GL_EINVAL for host buffers or an empty batch, GL_ENUMERIC
 * if no candidate meets the tolerance (the previous configuration stays). */
int gl_autotune(gl_context *ctx, const gl_params *p, const gl_times *t, double *out,
                gl_precision prec, void *stream, gl_tune_report *rep);

/* Sets the light-curve configuration for precision prec directly (for example
 * one an earlier gl_autotune chose): threads per CTA of the tile kernel (128 or
 * 256), Gauss-Legendre nodes per arc of the FP32C quadrature (16, 20, 24, 28;
 * the FP64 order is fixed), resident CTAs per SM of the item pipeline's
 * quadrature kernel (4 or 8) and threads per CTA of its exposure kernel (256 or
 * 64).  0 selects the default of each (256 threads, the shape-dependent default
 * order, 4 CTAs, 256 threads).  Drops the cached graphs.  GL_EINVAL for other
 * values. */
int gl_configure(gl_context *ctx, gl_precision prec, int threads, int nodes, int quad_ctas,
                 int exposure_block);

/* Allocation-failure hook (for tests; not in the paper).  With bytes > 0 the
 * context refuses to grow any workspace to more than `bytes`, exactly as if
 * cudaMalloc had failed: the call returns GL_ENOMEM with a message and the
 * context stays usable (the refused buffer is released, so a later call with the
 * limit lifted allocates it again).  bytes = 0 lifts the limit.  GL_EINVAL on
 * NULL or bytes < 0. */
int gl_debug_alloc_limit(gl_context *ctx, int64_t bytes);

/* Kernel kinds for gl_profile_read. */
#define GL_KERNEL_SETUP 0   /* per-set constants */
#define GL_KERNEL_CURVE 1   /* light-curve tile kernel, or the item pipeline's
                               kept-exposure kernel (FP64 or FP32C) */
#define GL_KERNEL_SKY 2     /* geometry-level kernel */
#define GL_KERNEL_SPHERE 3  /* spherical-planet kernel */
#define GL_KERNEL_SIMPSON 5 /* the paper's snapped Simpson scheme (gl_flux_sky_simpson) */
#define GL_KERNEL_QUAD 4    /* item pipeline: quadrature of queued sub-exposures and the
                               exposure means (two kernels) */
#define GL_KERNEL_WINDOW 6  /* item pipeline: the window test of every exposure */
#define GL_KERNEL_ITEMS 7   /* item pipeline: the quadrature kernel alone */
#define GL_KERNEL_STEP 8    /* mode 2 only: the whole captured light-curve step */
#define GL_KERNEL_KINDS 9

/* Per-kernel device timing for benchmarks.
 *   on = 1: every kernel launch of the context is bracketed by CUDA events
 *           recorded on its launch stream; light-curve steps run eagerly (no
 *           graph replay), so host launch gaps fall inside the timed spans.
 *   on = 2: light-curve steps keep their CUDA-graph replay; the step graph is
 *           captured with event-record nodes before the constants kernel and
 *           after each kernel (cudaEventRecordExternal), and every replay points
 *           them at a fresh set of events, so each kernel is timed inside the
 *           replayed graph, on the caller's stream.  Read with kinds SETUP,
 *           WINDOW, CURVE, ITEMS, QUAD (quadrature + exposure sums) and STEP.
 *   on = 0: off.
 * At most 65536 launches (replays) are kept; later ones are not timed.
 * Enabling resets the accumulated times.  GL_EINVAL on a NULL context or another
 * value of on. */
int gl_profile_enable(gl_context *ctx, int on);

/* Total device time in milliseconds and number of timed launches of kernel kind
 * `kind` since profiling was enabled.  Waits for the recorded events.
 * GL_EINVAL on a NULL context or pointer or an unknown kind, GL_ECUDA on a
 * runtime failure. */
int gl_profile_read(gl_context *ctx, int kind, double *ms, int64_t *launches);

/* ------------------------------------------------------------------------
 * Surrogate network (not in the paper): a fully connected network
 * 7 -> 256 -> 256 -> 256 -> 256 -> 1 with SiLU activations and a linear output,
 * predicting the oblate-minus-spherical flux residual from seven features.
 * FP32 master parameters; the three 256 x 256 layers run on the tensor cores
 * (tcgen05, BF16 operands, FP32 accumulation); loss = mean squared error.
 * Parameter vector (FP32, gl_mlp_param_count() = 199681 entries): W1[7][256],
 * b1[256], W2[256][256], b2, W3, b3, W4, b4 (row-major, z = x W + b), w5[256], b5.
 * All functions return GL_OK or a negative GL_E* code. */
typedef struct gl_mlp gl_mlp;

int64_t gl_mlp_param_count(void);
/* Create a network on `device` with all parameters zero. */
int gl_mlp_create(gl_mlp **m, int device);
int gl_mlp_destroy(gl_mlp *m);
/* Copy n = gl_mlp_param_count() FP32 parameters in (host or device memory);
 * resets the Adam state.  GL_EINVAL on NULL or a wrong n. */
int gl_mlp_set_params(gl_mlp *m, const float *p, int64_t n);
int gl_mlp_get_params(gl_mlp *m, float *p, int64_t n);
/* Gradients of the last gl_mlp_loss_grad, same layout. */
int gl_mlp_get_grads(gl_mlp *m, float *g, int64_t n);
/* y[i] = network(x[i][0..7)) for i < n; x (n x 7) and y (n) FP32 device memory. */
int gl_mlp_forward(gl_mlp *m, int64_t n, const float *x, float *y, void *stream);
/* Mean squared error of the network on (x, t) and its gradient (kept by the
 * network); *loss (host, may be NULL) is written after synchronising `stream`. */
int gl_mlp_loss_grad(gl_mlp *m, int64_t n, const float *x, const float *t, double *loss,
                     void *stream);
/* One Adam step (bias-corrected) with the last gradient. */
int gl_mlp_adam(gl_mlp *m, float lr, float beta1, float beta2, float eps, void *stream);
/* GL_ETIMEOUT if a tensor-core wait gave up since the last call, else GL_OK. */
int gl_mlp_status(gl_mlp *m);

/* Kernel kinds for gl_mlp_profile_read. */
#define GL_MLP_KERNEL_GEMM_FWD 0 /* the forward pass's tensor-core work (D = A B^T, bias,
                                    SiLU; 3 x 2 x rows x 256 x 256 flops per forward): one
                                    launch for the three hidden layers when the batch has
                                    at most one 128-row tile per SM, else one per layer */
#define GL_MLP_KERNEL_GEMM_BWD 1 /* a tensor-core layer of the backward pass (dZ W, SiLU') */
#define GL_MLP_KERNEL_WGRAD 2    /* a weight-gradient GEMM (A^T dZ, partial per CTA) */
#define GL_MLP_KERNEL_IN 3       /* the CUDA-core input layer (7 -> 256, SiLU) */
#define GL_MLP_KERNEL_OUT 4      /* the CUDA-core output layer (256 -> 1) */
#define GL_MLP_KERNEL_KINDS 5

/* Kernel timing (instrumentation, not in the paper).  With on = 1 every launch
 * of the kinds above made by gl_mlp_forward, gl_mlp_loss_grad and
 * gl_surrogate_train is bracketed by CUDA events on its stream; on = 0 stops.
 * Enabling resets the accumulated times; at most 65536 launches per kind are
 * timed.  The events are freed by gl_mlp_destroy.  GL_EINVAL on NULL or another
 * value of on. */
int gl_mlp_profile(gl_mlp *m, int on);

/* Total device time in milliseconds and number of timed launches of kernel kind
 * `kind` since timing was enabled (waits for the recorded events).  GL_EINVAL on
 * NULL pointers or an unknown kind, GL_ECUDA on a runtime failure. */
int gl_mlp_profile_read(gl_mlp *m, int kind, double *ms, int64_t *launches);

/* Failure-detection probe (for tests; not in the paper).  With polls > 0, every
 * tensor-core kernel of the following gl_mlp_forward / gl_mlp_loss_grad calls,
 * after allocating its tensor memory and before issuing any MMA, waits `polls`
 * times on an mbarrier phase that nothing completes.  The wait runs out as any
 * bounded device wait that gives up would: the kernel records it (gl_mlp_status
 * then returns GL_ETIMEOUT), frees its tensor memory and returns, leaving that
 * call's outputs undefined.  No tensor-core work is in flight when it gives up.
 * polls = 0 turns the probe off.  GL_EINVAL on NULL or polls < 0. */
int gl_mlp_wait_probe(gl_mlp *m, int polls);

/* Initial parameters: weights U(-sqrt(6 / fan_in), +sqrt(6 / fan_in)), biases
 * U(-0.1, 0.1), each entry i drawn from SplitMix64 (Steele, Lea and Flood 2014)
 * at (seed, i); resets the Adam state.  GL_EINVAL on NULL. */
int gl_mlp_init(gl_mlp *m, uint64_t seed);

/* ------------------------------------------------------------------------
 * Surrogate training, error table and checkpoint (not in the paper).
 *
 * Training minimises the mean squared error of the network on (feat, target)
 * by Adam over mini-batches.  The n samples are visited once per epoch in the
 * order of a permutation drawn afresh each epoch: a four-round Feistel network
 * on the sample index keyed by SplitMix64 at (seed, epoch), walked until it
 * lands below n.  The learning rate of step s of the whole run (epochs x
 * ceil(n / batch) steps) follows a cosine from lr (s = 0) to lr_end (last step).
 * Everything a step draws follows from (seed, s), so a run can be split into
 * calls, or resumed from a checkpoint, and gives the same parameters bit for bit
 * as one uninterrupted call. */
typedef struct {
  int64_t epochs;          /* passes over the training samples (>= 1) */
  int64_t batch;           /* samples per Adam step (1 .. 2^24); the last of an epoch may be short */
  float lr, lr_end;        /* cosine learning-rate schedule (lr > 0, lr_end >= 0) */
  float beta1, beta2, eps; /* Adam (as gl_mlp_adam) */
  uint64_t seed;           /* permutation of each epoch */
} gl_train_config;

/* Steps [first_step, first_step + n_steps) of the run that cfg describes, on n
 * samples: feat (n x 7 FP32) and target (n FP32), device memory.  *mean_loss
 * (host, may be NULL) receives the mean of the steps' mini-batch losses (this
 * synchronises `stream`).  The network keeps a mini-batch workspace of 32 bytes
 * per sample of cfg->batch.  GL_EINVAL for bad arguments or a step range beyond
 * the run. */
int gl_surrogate_train(gl_mlp *m, int64_t n, const float *feat, const float *target,
                       const gl_train_config *cfg, int64_t first_step, int64_t n_steps,
                       double *mean_loss, void *stream);

#define GL_SURROGATE_BINS 16

/* Held-out error table of the network: table[b] = the largest |network(feat_i) -
 * target_i| over the samples with bin_i = b (bins as gl_surrogate_features
 * writes them; -1 ignored), +infinity for a bin without samples (its items are
 * always recomputed exactly).  feat (n x 7), target, bin (n int32) and err (n
 * FP32, optional: the per-sample |error|) in device memory; table
 * (GL_SURROGATE_BINS FP32) host or device.  Synchronises `stream`. */
int gl_surrogate_error_table(gl_mlp *m, int64_t n, const float *feat, const float *target,
                             const int32_t *bin, float *table, float *err, void *stream);

/* Checkpoint of a surrogate: the FP32 parameters, both Adam moments, the Adam
 * step, the next schedule step `train_step`, the training configuration (with
 * its seed, the whole state of the shuffle) and the error table
 * (GL_SURROGATE_BINS FP32, host or device).  A binary file: a fixed header
 * (magic "GLSURR01", version 1, sizes, steps, configuration) followed by the
 * arrays.  Waits for the network's outstanding work.  GL_EIO if the file cannot
 * be written. */
int gl_surrogate_save(gl_mlp *m, const char *path, const float *table,
                      const gl_train_config *cfg, int64_t train_step);

/* Restore a checkpoint written by gl_surrogate_save into m (parameters, Adam
 * moments and step); table (host or device), cfg and train_step (host) receive
 * the rest and may be NULL.  GL_EIO if the file cannot be read or is not a
 * checkpoint of this network. */
int gl_surrogate_load(gl_mlp *m, const char *path, float *table, gl_train_config *cfg,
                      int64_t *train_step);

/* ------------------------------------------------------------------------
 * Surrogate light curves (not in the paper).  For every sub-exposure whose
 * planet overlaps the star, the deficit is the spherical planet's of equal
 * projected area (radius sqrt(dx dy2), gl_flux_sphere arithmetic, FP32) minus
 * the network's predicted oblate-minus-spherical residual times R_eq^2.  Seven
 * features feed the network: the centre distance rho, the angle between the
 * projected spin axis and the radial direction folded into [0, pi/2], k, f,
 * cos(eta) and Kipping's q1 = (u1+u2)^2, q2 = u1/(2 (u1+u2)), each scaled to
 * about [-1, 1].  A sub-exposure whose error bound, bound_table[bin] x R_eq^2,
 * exceeds bound_limit is recomputed by the exact FP32C path.  Bins
 * (GL_SURROGATE_BINS = 16): 8
 * equal bins of k over [0.01, 0.2] (clamped), for sub-exposures with the whole
 * ellipse on the disk (bins 0-7) and with crossings (8-15).  bound_table is 16
 * floats, host or device.  Geometry and orbit as in gl_lightcurve_batch (FP64
 * Kepler, FP64 exposure sum).
 * Device buffers only; nsuper must be uniform (tm->nsuper NULL).  Synchronises
 * `stream` (to size the network pass).  The context keeps a workspace of about
 * 60 bytes per sub-exposure of the batch.  stats may be NULL. */
typedef struct {
  int64_t items;      /* sub-exposures of in-window exposures */
  int64_t exposures;  /* in-window exposures */
  int64_t fallback;   /* sub-exposures recomputed exactly */
} gl_surrogate_stats;

int gl_lightcurve_surrogate(gl_context *ctx, gl_mlp *mlp, const gl_params *p,
                            const gl_times *t, double *out, const float *bound_table,
                            double bound_limit, void *stream, gl_surrogate_stats *stats);

/* Training data of the surrogate (device arrays, n entries): the seven features
 * (feat, n x 7 FP32), scale = R_eq^2 (FP32), the equal-area radius (FP64) and
 * the error-table bin (int32; -1 when the planet does not overlap the star) for
 * sky positions (x0, y0) and shapes (k, f, eta, xi, u1, u2). */
int gl_surrogate_features(gl_context *ctx, int64_t n, const double *x0, const double *y0,
                          const double *k, const double *f, const double *eta, const double *xi,
                          const double *u1, const double *u2, float *feat, float *scale,
                          double *r_area, int32_t *bin, void *stream);
/* t = (f_oblate - f_sphere) / scale (0 where scale is 0). */
int gl_surrogate_targets(gl_context *ctx, int64_t n, const double *f_oblate,
                         const double *f_sphere, const float *scale, float *t, void *stream);

/* Gaussian log-likelihood of n_sets light curves against one data set:
 * loglike[s] = -1/2 sum_j ((flux[s][j] - data[j]) / sigma[j])^2 (constant terms
 * dropped).  flux n_sets x n_times, data and sigma n_times, all device memory. */
int gl_loglike(gl_context *ctx, int64_t n_sets, int64_t n_times, const double *flux,
               const double *data, const double *sigma, double *loglike, void *stream);

/* ------------------------------------------------------------------------
 * The (mu, nu) reparameterisation of Appendix A and a device-resident ensemble
 * sampler.
 *
 * For an oblate spheroid the flux depends on (f, eta) only through
 * mu = (f - 1)^2 + f (f - 2) cos(2 eta); nu in [0, 1] places f between
 * f_min = 1 - sqrt((mu + 1)/2) and 1 (f = f_min + (1 - f_min) nu).  The joint
 * density p(mu, nu) of Appendix A makes the prior on (f, eta) uniform in f and
 * proportional to cos(eta); it is drawn from two uniforms (u, w) by the printed
 * inverse transforms.  Element-wise on n entries, FP64, device memory;
 * GL_EINVAL on NULL or host arrays. */
int gl_munu_to_feta(gl_context *ctx, int64_t n, const double *mu, const double *nu,
                    double *f, double *eta, void *stream);
int gl_feta_to_munu(gl_context *ctx, int64_t n, const double *f, const double *eta,
                    double *mu, double *nu, void *stream);
int gl_munu_prior(gl_context *ctx, int64_t n, const double *u, const double *w,
                  double *mu, double *nu, void *stream);

/* Fit vector of a walker: t0, period, a_rs, b, k, mu, nu, xi, q1, q2 (circular
 * orbit; f and eta from (mu, nu); u1, u2 from (q1, q2) by Kipping's map). */
#define GL_FIT_DIM 10

typedef struct {
  int64_t n_walkers;       /* even, 4 .. 2^26 */
  double *walkers;         /* n_walkers x GL_FIT_DIM, row-major, device; updated in place */
  double *logpost;         /* n_walkers, device; written by init, updated by sweeps */
  const double *lo, *hi;   /* GL_FIT_DIM box bounds of the uniform prior, device */
  const double *t;         /* n_times exposure midpoints (days), device */
  int64_t n_times;
  const double *data, *sigma;   /* n_times observed relative flux and its error, device */
  double exptime;          /* exposure time (days) */
  int nsuper;              /* sub-exposures per exposure */
  double a;                /* stretch scale (> 1; 2 is usual) */
  gl_precision prec;       /* light-curve path */
} gl_ensemble;

/* log posterior of every walker: log prior (uniform in the box, -inf outside,
 * times p(mu, nu)) + Gaussian log likelihood of its light curve (as gl_loglike).
 * The context keeps a workspace of (12 + 2 + n_times) doubles per walker. */
int gl_ensemble_init(gl_context *ctx, const gl_ensemble *e, void *stream);

/* One sweep of the affine-invariant stretch move (Goodman and Weare 2010), all on
 * the device: for each half h = 0, 1 of the ensemble (walkers k = 2 i + h,
 * i < n/2), proposals Y = X_j + z (X_k - X_j) with partner
 * j = 2 floor(r_j n/2) + 1 - h and z = ((a - 1) r_z + 1)^2 / a, their light curves
 * and log posteriors, and acceptance when log(r_u) < (D - 1) log z + lp(Y) - lp(X).
 * rnd: 3 n_walkers uniforms in [0, 1) on the device, laid out per half as
 * (r_z, r_j, r_u), n/2 each.  accepted: optional device counter, incremented per
 * accepted move.  Stream-ordered: no host synchronisation. */
int gl_ensemble_sweep(gl_context *ctx, const gl_ensemble *e, const double *rnd,
                      unsigned long long *accepted, void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free variant of gl_lightcurve_batch.  The paper has no
 * counterpart: this is a deployment aid.
 *
 * Some callers cannot let a library allocate device memory: applications whose
 * device memory belongs to a pool allocator with a fixed budget (an extra
 * cudaMalloc can fail or fragment the pool), latency-critical loops where a
 * cudaMalloc or cudaFree would add a device-wide synchronisation, and plug-ins
 * hosted by a process that forbids allocation outside its own allocator.  This
 * entry point needs no context and calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its per-set workspace is one fixed array compiled into
 * the library: GL_NOALLOC_MAX_SETS x 576 bytes of per-set constants plus 256
 * bytes of status, 2 359 552 bytes (about 2.36 MB), which every GPU that loads
 * the library holds until the process exits.
 *
 *   p, t, out, prec, stream  as for gl_lightcurve_batch, on the current CUDA
 *                            device, except that every array must be device
 *                            memory of that device (host arrays would need a
 *                            staging copy, which would allocate).
 * Returns GL_OK; GL_EINVAL for a NULL or host pointer, n_sets > GL_NOALLOC_MAX_SETS
 * or any size check of gl_lightcurve_batch; GL_ECUDA on a runtime failure.
 * Physically invalid parameter sets give NaN outputs (no status is kept).
 * CSR offsets are not validated by this entry point: offsets that do not rise
 * from 0 to n_total give unspecified light curves (exposures attributed to other
 * sets), still with every read inside offsets[0 .. n_sets], t[0 .. n_total) and
 * the parameter arrays, every write inside out[0 .. n_total), and GL_OK.
 *
 * The first call on a device uploads the quadrature tables and looks up the
 * array's device address on that device; make that first call before any
 * stream capture.  Every call shares the array and overwrites the entries it
 * uses before reading them, so calls that overlap on the GPU (on different
 * streams, or from different threads) race and must be serialised by the
 * caller.  The call is asynchronous on `stream`.
 */
#define GL_NOALLOC_MAX_SETS 4096
int gl_lightcurve_batch_noalloc(const gl_params *p, const gl_times *t, double *out,
                                gl_precision prec, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GL_H */
