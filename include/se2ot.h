/*
 * se2ot.h -- C ABI of libse2ot.so: the left-invariant SE(2) Gibbs-kernel group convolution
 * and the convolutional Sinkhorn barycenter / interpolation of
 * "Optimal Transport on the Lie Group of Roto-translations" (arXiv 2402.15322), on one
 * NVIDIA GB300 (sm_103a).
 *
 * Problem statement (Sec. 2.2, Eq. barywass; Sec. 4.1; Appendix A):
 *   grid     an Nx x Ny x Ntheta discretisation of SE(2): voxel (ix, iy, k) is the group element
 *            (ix/Nx, iy/Ny, 2 pi k / Ntheta), x and y in [0,1), theta periodic (Sec. 2.3,
 *            Sec. 5.1 for the grid of the experiments).
 *   kernel   K(g) = exp(-rho_b(g)^2 / eps) with the half-angle approximation rho_b of the
 *            left-invariant distance for metric weights (w1, w2, w3) (Sec. 4.3, Eq. rho_b and
 *            the half-angle coordinates), truncated to spatial offsets |dx|, |dy| <= radius
 *            voxels with all Ntheta x Ntheta orientation pairs coupled.
 *   conv     (K * f)(g) = sum_h K(h^-1 g) f(h) (Sec. 4.2), uniform voxel weights (Haar measure,
 *            Sec. 2.3; its constant is omitted because it cancels in every barycenter iterate).
 *   bary     the Appendix A iteration: v_i = w_i = 1; repeat { w_i = mu_i / (K * v_i);
 *            d_i = v_i (K * w_i); mu = prod_i d_i^lambda_i; v_i = v_i mu / d_i }.
 *
 * Memory layout of every field: f[((b*Ny + y)*Nx + x)*Ntheta + k], orientation innermost,
 * densely packed, b the batch / measure index.  V = Nx*Ny*Ntheta.
 *
 * Numerics.  The scaling vectors are kept as base-2 logarithms in double-float device memory
 * (pairs of FP32 numbers, ~48 significant bits); every convolution is evaluated as a log-sum-exp
 * with a per-output shift, its terms in FP32.  The
 * paper's linear-domain iteration is the same algorithm; at the regularisations this library
 * targets (eps ~ 1e-4 on 128^2 grids) v_i and w_i span thousands of nats, far outside the
 * FP32 (and FP64) exponent range, so the linear form cannot be evaluated directly.
 *
 * Threading and streams.  Every call enqueues its work on the CUDA stream passed in (a
 * cudaStream_t cast to void*, NULL = the legacy default stream) of the current device and,
 * unless stated otherwise, returns without waiting.  A kernel handle serialises nothing:
 * calls that share one handle must not overlap in time (from several host threads or several
 * streams), because the handle's workspace is reused.
 *
 * Errors.  Every call returns an se2ot_status; nothing aborts.  se2ot_last_error() gives a
 * human-readable message for the calling host thread's most recent failure.
 */
#ifndef SE2OT_H
#define SE2OT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SE2OT_API __attribute__((visibility("default")))
#else
#define SE2OT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SE2OT_OK = 0,
    SE2OT_EINVAL = 1,      /* an argument is out of range; nothing was enqueued           */
    SE2OT_ENOMEM = 2,      /* a device or host allocation failed                          */
    SE2OT_ECUDA = 3,       /* a CUDA runtime call failed (message in se2ot_last_error)     */
    SE2OT_ENONFINITE = 4,  /* an iterate became NaN or infinite (result still written)    */
    SE2OT_ENOTCONV = 5,    /* tol_viol > 0 was not reached within max_iters               */
    SE2OT_ETIMEOUT = 6,
    SE2OT_EBUSY = 7,
    SE2OT_ESHUTDOWN = 8
} se2ot_status;

typedef enum {
    SE2OT_FP32 = 0,        /* log-domain convolution, FP32 terms, FP64 log storage          */
    SE2OT_BF16TC = 1       /* tcgen05 tensor cores, BF16 operands, FP32 accumulation, on the
                              tiles a per-tile rescaling can represent; FP32 path elsewhere   */
} se2ot_precision;

typedef enum {
    SE2OT_BOUNDARY_ZERO = 0,     /* no term outside the grid                               */
    SE2OT_BOUNDARY_PERIODIC = 1  /* spatial indices wrap (theta always wraps)               */
} se2ot_boundary;

/* The distance approximation rho in the Gibbs kernel K(g) = exp(-rho(g)^2 / eps) (Sec. 4.3). */
typedef enum {
    SE2OT_DIST_RHO_B = 0,        /* half-angle approximation rho_b (the paper's kernel)      */
    SE2OT_DIST_RHO_C = 1         /* logarithmic approximation rho_c = ||log g||              */
} se2ot_distance;

/* Grid, metric and kernel.  Valid ranges: nx, ny >= 2*radius + 1; 0 <= radius <= 16;
 * 1 <= ntheta <= 64; w1, w2, w3 > 0; eps > 0. */
typedef struct {
    int nx, ny, ntheta, radius;
    double w1, w2, w3, eps;
    int boundary;                /* se2ot_boundary */
    int distance;                /* se2ot_distance */
} se2ot_kernel_desc;

typedef struct se2ot_kernel_s *se2ot_kernel;   /* opaque; owns tap tables and workspace */

/* Solver options.  max_iters >= 1 Sinkhorn iterations (one iteration = every line of the
 * Appendix A loop body).  check_every > 0 together with tol_viol > 0 evaluates the marginal
 * violation every check_every iterations (a host synchronisation each time) and stops once
 * viol <= tol_viol.  flags: bitwise OR of SE2OT_FLAG_*.
 * precision SE2OT_BF16TC runs the convolutions on the tensor cores (see se2ot_apply) except for
 * the last refine_iters (0 <= refine_iters <= max_iters) of the max_iters iterations, which run on
 * the FP32 path (refinement sweeps); refine_iters is ignored for SE2OT_FP32. */
typedef struct {
    int max_iters;
    int check_every;
    double tol_viol;
    int precision;               /* se2ot_precision */
    int flags;
    int refine_iters;
} se2ot_solve_opts;

#define SE2OT_FLAG_TIME_CONV 1   /* time every convolution launch with CUDA events (stats.conv_ms) */
/* se2ot_interpolate_batched only: the form of the convolution launches (see there); neither flag:
 * the form is chosen by timing both on the first call with a given set of descriptors. */
#define SE2OT_FLAG_BATCH_ONE_LAUNCH 2    /* one launch per convolution line, every radius in it */
#define SE2OT_FLAG_BATCH_PER_RADIUS 4    /* one launch per radius class and convolution line */

/* Results of a solve (written after the call's internal synchronisation).
 *   iters            iterations performed
 *   mass             sum of the returned barycenter (FP64)
 *   viol             sum_i lambda_i ||d_i - mu||_1 / ||mu||_1 after the last iteration (FP64)
 *   ms               wall time of the call from first enqueue to completion
 *   voxel_iters_per_s  V * iters / (ms / 1000)
 *   conv_ms, conv_launches   with SE2OT_FLAG_TIME_CONV: summed CUDA-event time of the
 *                    convolution launches and their number (0 otherwise)
 *   kernel_launches  kernels this call launched
 *   redo_outputs     convolution outputs whose first evaluation fell outside the safe range
 *                    of its shift and were recomputed exactly
 *   evaluated_terms  kernel terms the convolutions evaluated; orientation pairs, kernel rows and
 *                    blocks of window positions whose terms all lie below 2^-64 of the output's
 *                    shift are skipped, so this is at most 2 * iters * n * V * ntheta * (2r+1)^2.
 *                    Counted per block of 4 window positions of a warp: an estimate, within
 *                    10% of the exact count.
 *   logscale_min, logscale_max   smallest and largest natural logarithm of the scaling vectors
 *                    v_i over all measures and voxels after the last iteration (FP64, finite entries
 *                    only): the dynamic range the solve needed, the reason the library keeps the
 *                    scaling vectors as logarithms (FP32 holds e^-87 .. e^88, FP64 e^-708 .. e^709).
 *                    Not measured by se2ot_jko (0).
 *   tc_tiles, tc_fallback_tiles  SE2OT_BF16TC: tiles of 4 rows x 128 positions (all orientations)
 *                    the tensor cores computed, and those they left to the FP32 path because a
 *                    per-tile rescaling could not represent them (0 for SE2OT_FP32). */
typedef struct {
    int iters;
    double mass, viol, ms, voxel_iters_per_s;
    double conv_ms;
    long long conv_launches;
    long long kernel_launches;
    long long redo_outputs;
    long long evaluated_terms;
    double logscale_min, logscale_max;
    long long tc_tiles, tc_fallback_tiles;
} se2ot_stats;

/* Build the kernel for a grid: validates desc, evaluates the taps
 * log2 K = -rho_b(h^-1 g)^2 / (eps ln 2) for every orientation pair and offset on the device
 * in FP64 (Sec. 4.3 Eq. rho_b, Sec. 4.2 kernel definition), kept as the exact FP64 orientation
 * factor plus the spatial part as FP32 value + FP32 rounding residual.
 * Returns EINVAL for an invalid desc, ENOMEM/ECUDA on device failure.  The handle must be
 * released with se2ot_kernel_destroy.  Synchronises `stream` before returning. */
SE2OT_API se2ot_status se2ot_kernel_build(const se2ot_kernel_desc *desc, void *stream, se2ot_kernel *out);

/* Release a kernel handle and its device memory (NULL is a no-op).  Waits for the device. */
SE2OT_API se2ot_status se2ot_kernel_destroy(se2ot_kernel k);

/* Copy the tap table to host memory `taps_host` of ntheta*ntheta*(2r+1)^2 floats, in the
 * order taps[((o*ntheta + i)*(2r+1) + dy + r)*(2r+1) + dx + r] = log2 K for output orientation
 * o, input orientation i and spatial offset (dx, dy) = output voxel - input voxel.
 * Synchronises the device. */
SE2OT_API se2ot_status se2ot_kernel_taps(se2ot_kernel k, float *taps_host);

/* out = K * f for `batch` fields (Sec. 4.2).  f and out: device pointers to batch*V floats,
 * f >= 0 (zeros allowed), may not alias.  Evaluated as exp2 of a log-domain convolution.
 * precision: SE2OT_FP32, or SE2OT_BF16TC for the tcgen05 tensor cores (ntheta <= 16, nx >= 64):
 * per tile of 4 rows x 128 positions and all orientations, the log-domain sum is rescaled by a
 * tilt plane fitted to the outputs, one shift per input and per output orientation, and computed
 * as a GEMM of BF16 operands with FP32 accumulation (relative error of an output ~1e-3, BF16
 * rounding).  Tiles whose rescaled operands cannot represent every output go to the FP32 path,
 * outputs whose accumulator is too small to be trusted to the exact recompute; the result is
 * therefore never worse than BF16 rounding.  EINVAL on batch < 1, NULL pointers, an unknown
 * precision or an unsupported grid. */
SE2OT_API se2ot_status se2ot_apply(se2ot_kernel k, const float *f, float *out, int batch, int precision, void *stream);

/* lout = log(K * exp(lf)) (natural logarithms) for `batch` fields: device pointers to
 * batch*V doubles; -inf entries of lf are zero densities.  May not alias.  precision as in
 * se2ot_apply. */
SE2OT_API se2ot_status se2ot_apply_log(se2ot_kernel k, const double *lf, double *lout, int batch, int precision,
                                       void *stream);

/* Barycenter of n >= 1 measures with weights lambda (Appendix A; Eq. barywass with the
 * entropic kernel of Sec. 4.2).  mu: n*V floats, host or device memory (detected).  The inputs
 * must be measures of equal mass, which the Appendix A iteration assumes: every entry finite and
 * >= 0, every measure with positive mass, and the n masses equal to 1e-6 relative to the largest.
 * This is checked on the device in FP64 before the first iteration (one stream synchronisation);
 * a violation returns EINVAL with a message naming the measure.  The library does not
 * renormalise; a common scale of all inputs is allowed (the barycenter is homogeneous of degree
 * one in it).  lambda: n <= 64 host doubles, >= 0, summing to 1 within 1e-12.  bary: V floats,
 * host or device memory.  opts may be NULL (100 iterations, no checks).  stats may be NULL.
 * Host memory is copied on the stream; the call synchronises the stream before returning (stats
 * need it).  Workspace: 4 n V + V double-floats, 2 n V floats and n V int pairs, owned by the
 * kernel handle and reused.
 * Returns EINVAL for invalid arguments (inputs included), ENONFINITE if an iterate became
 * non-finite, ENOTCONV if tol_viol > 0 was not reached (the result is still written). */
SE2OT_API se2ot_status se2ot_barycenter(se2ot_kernel k, int n, const float *mu, const double *lambda,
                              const se2ot_solve_opts *opts, float *bary, se2ot_stats *stats,
                              void *stream);

/* Interpolation Phi_t(mu0, mu1) (Eq. interpolation operator): the barycenter of (mu0, mu1)
 * with weights (1 - t, t), 0 <= t <= 1, so that t = 0 is the side of mu0.  Arguments as in
 * se2ot_barycenter, each of mu0, mu1, out holding V floats. */
SE2OT_API se2ot_status se2ot_interpolate(se2ot_kernel k, const float *mu0, const float *mu1, double t,
                               const se2ot_solve_opts *opts, float *out, se2ot_stats *stats,
                               void *stream);

/* Entropic optimal transport between two measures (Sec. 4.1): the scaling iterations with both
 * marginals prescribed (prox of the marginal constraint, Eq. (F_i) with n = 2),
 *   a = mu / (K * b),   b = nu / (K * a),          b = 1 initially,
 * one iteration being both steps, then the plan pi(g, h) = a(g) K(h^-1 g) b(h) and its cost
 * for c = rho_b^2 (Eq. (L^{W_p}) with p = 2, the Gibbs kernel being exp(-c / eps)):
 *   cost  = <c, pi> = sum_g a(g) ((cK) * b)(g)     (the entropic estimate of W_2^2)
 *   dual  = eps (<mu, log a> + <nu, log b>)         (natural log; voxels with zero mass skipped)
 *   mass  = sum pi
 *   viol  = ||a (K * b) - mu||_1 / ||mu||_1         (the nu-marginal holds exactly after each b-step)
 * all reduced in FP64 in a fixed order.  mu, nu: V floats each, caller layout [y][x][theta],
 * nonnegative and finite, host or device memory; their masses need not be 1 but must agree to
 * 1e-6 relative (checked on the device before the first iteration: EINVAL otherwise).  opts as in se2ot_barycenter (tol_viol > 0 with check_every > 0 stops once viol
 * <= tol_viol; each check costs two convolutions).  The first call on a kernel handle builds the
 * cost-weighted tap table (same size as the kernel's); workspace is the handle's, as for a
 * 2-measure barycenter.  The call synchronises the stream before returning.
 * Returns EINVAL for invalid arguments, ENONFINITE for a non-finite result, ENOTCONV if tol_viol
 * was not reached (res is still written). */
typedef struct {
    int iters;
    double cost, dual, mass, viol;
    double ms;                   /* wall time of the call */
    long long kernel_launches;
    long long redo_outputs;
} se2ot_w2_result;

SE2OT_API se2ot_status se2ot_w2(se2ot_kernel k, const float *mu, const float *nu, const se2ot_solve_opts *opts,
                                se2ot_w2_result *res, void *stream);

/* Entropic JKO steps of the porous-medium energy F(mu) = sum_g mu(g)^m / (m - 1) (unit Haar weight
 * per voxel; Sec. 2.2 Eq. (GF_JKO), Sec. 6.4): steps x
 *   mu_{k+1} = argmin_nu W_eps(mu_k, nu) + tau F(nu)
 * by the scaling iterations of Sec. 4.1 with the marginal constraint on the first marginal and
 * the KL-proximal map of tau F on the second, opts->max_iters iterations per step from b = 1:
 *   a = mu_k / (K * b),   b = prox_{(tau/eps) F}(K * a) / (K * a),   mu_{k+1} = prox(K * a).
 * The prox solves log s + (tau/eps) m/(m-1) s^(m-1) = log z per voxel (Newton, FP64 result).
 * mu0: V floats, caller layout, strictly positive and finite (a zero density makes the b-update
 * 0/0; checked on the device before the first step: EINVAL otherwise) and on the density scale F
 * is meant for (no normalisation); mu_out: V floats; host or device memory.
 * tau >= 0, m > 1, steps >= 1, opts->tol_viol must be 0.  stats: iters = steps * max_iters, mass =
 * sum mu_out, viol = ||a (K * b) - mu_k||_1 / ||mu_k||_1 of the last step (FP64).  Workspace as for
 * a 2-measure barycenter.  Synchronises the stream.  EINVAL for invalid arguments, ENONFINITE for a
 * non-finite iterate. */
SE2OT_API se2ot_status se2ot_jko(se2ot_kernel k, const float *mu0, double tau, double m, int steps,
                                 const se2ot_solve_opts *opts, float *mu_out, se2ot_stats *stats, void *stream);

/* Lifting / projection helpers of the paper's experiments (Sec. 2.4, 6.2, 6.3).  Device pointers
 * only (EINVAL otherwise); arrays in the caller layout, orientation innermost; enqueued on
 * `stream`, no synchronisation.
 *
 * se2ot_project: P[b][y][x] = sum_k U[b][y][x][k], the projection P(U) = integral of U over theta
 * (Eq. proj) with unit weight per orientation bin (the bin width 2 pi / ntheta is a constant the
 * paper's normalisation of every output removes).  U: batch * ny * nx * ntheta floats, P: batch *
 * ny * nx floats (FP64 accumulation). */
SE2OT_API se2ot_status se2ot_project(const float *U, float *P, int batch, int nx, int ny, int ntheta, void *stream);

/* Lift of an orientation field v = |v| (cos psi, sin psi) onto SE(2) (Sec. 6.3, lifting of vector
 * fields): U[y][x][k] = |v[y][x]| for the bin k whose centre 2 pi k / ntheta is within pi / ntheta
 * of psi = atan2(v_y, v_x) (an angle exactly half-way goes to the upper bin), 0 elsewhere.
 * v: ny * nx * 2 floats (x, y components), U: ny * nx * ntheta floats. */
SE2OT_API se2ot_status se2ot_lift_field(const float *v, float *U, int nx, int ny, int ntheta, void *stream);

/* Reconstruction of the field (Sec. 6.3): v = (sum_k U[y][x][k]) (cos psi*, sin psi*) with psi* the
 * centre of the first largest bin; v = 0 where every bin is 0.  Inverse of se2ot_lift_field on
 * bin-centred angles. */
SE2OT_API se2ot_status se2ot_reconstruct_field(const float *U, float *v, int nx, int ny, int ntheta, void *stream);

/* Interpolation of two signed orientation scores (Sec. 6.2, steps 2-4): the positive and negative
 * parts U+- = max(+-U, 0) get a floor of 1e-6 of their maximum (exact zeros make the scaling
 * update 0/0 wherever the barycenter vanishes too), are normalised to mass 1 and interpolated
 * separately with the same kernel and options (se2ot_interpolate), then
 *   b[y][x] = m+_t P(Phi_t(U0+, U1+)) - m-_t P(Phi_t(U0-, U1-)),   m_t = (1 - t) m_0 + t m_1,
 * with m the parts' masses (FP64), so that b keeps the scale of the scores.  A part that is zero
 * on both sides contributes nothing; zero on one side only is EINVAL (nothing to transport).
 * U0, U1: V floats each (the kernel's grid), b: ny * nx floats, device memory; stats (may be NULL)
 * receives 2 entries, the positive and the negative part's solve.  Synchronises the stream. */
SE2OT_API se2ot_status se2ot_interpolate_signed(se2ot_kernel k, const float *U0, const float *U1, double t,
                                                const se2ot_solve_opts *opts, float *b, se2ot_stats *stats,
                                                void *stream);

/* nprob independent interpolations Phi_t(mu0[p], mu1[p]) (weights (1 - t[p], t[p])) of uneven grid
 * sizes, radii, metrics and regularisations, iterated in lockstep for opts->max_iters Sinkhorn
 * iterations (Appendix A with n = 2 for every problem).  descs[p]: each problem's grid and kernel
 * (zero boundary only).  mu0[p], mu1[p]: device arrays of V_p floats (caller layout), measures of
 * equal mass as for se2ot_barycenter (checked on the device before the first iteration: EINVAL
 * naming the problem otherwise), out[p]: V_p floats, device.  opts: max_iters >= 1, tol_viol must be 0 (no early stop in a batch), NULL =
 * 100 iterations.  stats: NULL or an array of nprob entries (ms and kernel_launches are for the
 * whole batch).
 * One iteration of the batch is, for each of the two convolution lines, the convolution of every
 * tile of every problem and one exact recompute pass, then one update launch, recorded once as a
 * CUDA graph and replayed.  The convolution of a line takes one of two forms:
 *   per radius:  one launch per distinct radius (a work list over that radius's tiles);
 *   one launch:  a single launch over every tile, the largest radius first, each tile running the
 *                code specialised for its problem's radius.
 * opts->flags may force one (SE2OT_FLAG_BATCH_PER_RADIUS, SE2OT_FLAG_BATCH_ONE_LAUNCH; both:
 * EINVAL); otherwise the first call with a set of descriptors times a few iterations of each
 * (se2ot_batch_tuning reports them), keeps the faster for the calls that follow, and starts the
 * iteration again from the inputs.  Each tile runs the same code in either form, so each problem's
 * result is bit-identical to se2ot_interpolate on that problem alone.  The workspace, the graphs
 * and the choice are kept for the next call with the same descriptors; calls are serialised by a
 * library-wide lock.  Synchronises `stream` before returning. */
SE2OT_API se2ot_status se2ot_interpolate_batched(int nprob, const se2ot_kernel_desc *descs, const float *const *mu0,
                                                 const float *const *mu1, const double *t,
                                                 const se2ot_solve_opts *opts, float *const *out,
                                                 se2ot_stats *stats, void *stream);

/* The launch form of the last tuned batch (the paper has no counterpart: a property of this
 * library's batched launches).  form: 1 per radius, 2 one launch, 0 no batch tuned yet (or every
 * call so far forced a form); ms_per_radius, ms_one_launch: the measured milliseconds per batch
 * iteration of each form (0 if not measured).  Host pointers; EINVAL if one is NULL. */
SE2OT_API se2ot_status se2ot_batch_tuning(int *form, double *ms_per_radius, double *ms_one_launch);

/* Serving: a request loop for barycenter solves with continuous batching (no counterpart in the
 * paper; the solve of every request is se2ot_barycenter's).  A server owns one worker thread on
 * `device`.  Requests wait in FIFO order until a slot (at most max_slots run at once) and their
 * device state (tap table, inputs, workspace; about 90 bytes per voxel and measure) fit in
 * device_budget_bytes; an admitted request gets its own stream and stream-ordered memory and is
 * advanced in chunks of check_every iterations (50 without a tolerance), each followed by the
 * FP64 marginal violation; it completes when viol <= tol_viol or after max_iters iterations.
 * Chunks of all admitted requests overlap on the device; memory is returned and the next request
 * admitted as each completes.  A request's result does not depend on the other requests. */
typedef struct se2ot_server_s *se2ot_server;

/* Start a server.  EINVAL for max_slots < 1, a zero budget or an unknown device. */
SE2OT_API se2ot_status se2ot_serve_create(size_t device_budget_bytes, int max_slots, int device, se2ot_server *out);

/* Queue a barycenter of n measures (arguments as in se2ot_barycenter; mu host or device memory,
 * copied before return so the caller may free it; the input check of se2ot_barycenter runs on that
 * host copy, EINVAL on failure).  ticket receives the request's id.  ENOMEM if
 * the request can never fit the budget, EINVAL for invalid arguments, ESHUTDOWN after destroy
 * began. */
SE2OT_API se2ot_status se2ot_serve_submit(se2ot_server sv, const se2ot_kernel_desc *desc, int n, const float *mu,
                                          const double *lambda, const se2ot_solve_opts *opts, uint64_t *ticket);

/* done = 1 once the request has finished (successfully or not). */
SE2OT_API se2ot_status se2ot_serve_poll(se2ot_server sv, uint64_t ticket, int *done);

/* Wait up to timeout_ms (< 0: forever) for the request, then copy its barycenter (V floats, host or
 * device) to out (may be NULL) and its statistics (ms = latency from submit) to stats, and forget
 * the ticket.  Returns the request's status (OK, ENOTCONV if the tolerance was not reached,
 * ENONFINITE, ENOMEM if admission failed, ESHUTDOWN), or ETIMEOUT (the ticket stays valid). */
SE2OT_API se2ot_status se2ot_serve_wait(se2ot_server sv, uint64_t ticket, float *out, se2ot_stats *stats,
                                        int timeout_ms);

/* Stop the server: queued requests finish with ESHUTDOWN, admitted ones run to completion, then
 * the worker exits.  Tickets not yet waited for become invalid. */
SE2OT_API se2ot_status se2ot_serve_destroy(se2ot_server sv);

/* State of the kernel handle's most recent se2ot_barycenter / se2ot_interpolate solve with n
 * measures, for checkpointing and for checking the iteration's invariants: natural logarithms of
 * the scaling vectors v_i and of the marginals d_i = v_i (K w_i) (n*V doubles each) and of the
 * barycenter mu = prod_i d_i^lambda_i (V doubles), in the caller's layout [i][y][x][theta]
 * (Appendix A, after the last v-update).  Any output pointer may be NULL.  Device pointers only
 * (EINVAL otherwise); n must equal the solve's.  Enqueued on `stream`. */
SE2OT_API se2ot_status se2ot_state_export(se2ot_kernel k, int n, double *log_v, double *log_d, double *log_mu,
                                          void *stream);

/* Size of the device array behind se2ot_barycenter_noalloc: 16 MiB on every GPU that loads the
 * library, held until the process exits. */
#define SE2OT_NOALLOC_SCRATCH_BYTES (16u << 20)

/* se2ot_barycenter for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of the same solve.
 *
 * Some callers may not call cudaMalloc: a host application or framework that owns the device's
 * whole memory budget through its own allocator, a latency-critical loop that cannot afford
 * cudaMalloc's implicit synchronisation, a plugin restricted to the buffers it is given.  They
 * cannot create an se2ot_kernel either, because building one allocates its tap table and
 * workspace.  This call takes the kernel descriptor itself and keeps the tap table and every
 * scaling vector in one statically allocated device array of SE2OT_NOALLOC_SCRATCH_BYTES; it
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Arguments as in se2ot_barycenter, except: desc replaces the kernel handle; mu (n*V floats) and
 * bary (V floats) must be device memory (EINVAL otherwise: nothing is staged); stats->conv_ms is
 * not measured (0).  The inputs are checked as in se2ot_barycenter.  A problem whose tap table
 * and workspace need more than the array is rejected with EINVAL and a message giving the size.
 * The array holds, in this order, each part starting on a 256-byte boundary (P = ntheta^2 orientation
 * pairs, D = 2 radius + 1, T = n ntheta ceil(nx/32) ceil(ny/16) tiles):
 *   taps: 8 P, 4 P D^2, 4 P D^2 and 4 P D bytes;  tile maxima: 4 T and 4 T bytes;
 *   logs of mu_i, v_i, w_i, d_i: four arrays of 8 n V bytes;  log of the barycenter: 8 V;
 *   shifts: two arrays of 4 n V;  recompute list: 8 n V;  launch order: 16 T + 8;
 *   counters and sums: 16, 16, 8192 and 32 bytes;  input check: 2080 n bytes.
 * E.g. n = 4 measures on 64 x 64 x 16 with radius 10 fit (14.1 MB); n = 5 there (17.2 MB) and
 * 128 x 128 x 16 do not.
 *
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress) and
 * caches it; make that first call before any stream capture.  Every call shares the one array
 * and finds the previous call's contents in it; it re-initialises all it reads.  Calls whose GPU
 * work overlaps (other threads, other streams) race on the array: serialise them. */
SE2OT_API se2ot_status se2ot_barycenter_noalloc(const se2ot_kernel_desc *desc, int n, const float *mu,
                                                const double *lambda, const se2ot_solve_opts *opts,
                                                float *bary, se2ot_stats *stats, void *stream);

/* Measured throughput of the SFU's ex2.approx instruction on the current device (results per
 * second, all SMs), by a kernel of independent ex2 chains timed with CUDA events on `stream`
 * (about 1 ms; synchronises the stream).  The log-domain convolution evaluates one ex2 per kernel
 * term, so this is the ceiling of its evaluated-term rate.  No counterpart in the paper: a
 * measurement utility for roofline reports.  EINVAL for a NULL pointer, ECUDA on a CUDA failure. */
SE2OT_API se2ot_status se2ot_sfu_ex2_rate(double *ex2_per_s, void *stream);

/* Message for the calling host thread's most recent error ("" if none).  The pointer stays
 * valid until the thread's next failing call. */
SE2OT_API const char *se2ot_last_error(void);

/* Library version string. */
SE2OT_API const char *se2ot_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SE2OT_H */
