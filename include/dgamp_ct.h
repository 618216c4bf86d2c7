/*
 * dgamp_ct.h -- C ABI of the GB300 D-GAMP-CT library (libdgampct.so).
 *
 * D-GAMP-CT (Perelli, Lexa, Can, Davies, "Compressive Computed Tomography
 * Reconstruction through Denoising Approximate Message Passing") reconstructs
 * an attenuation image mu from Poisson transmission counts
 * y_i ~ Poisson(I0 exp(-[A mu]_i)) (Section 2.1, Eq. Poisson_CT) by running
 * GAMP (Algorithm 1) in the preconditioned space x = V mu (Section 2.4,
 * Eq. PPFT preconditioner) with a black-box denoiser (Section 4.3).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Image: float32, row-major [n][n], row 0 at the top.  Pixel (ix, iy) has
 *    centre X = ix - (n-1)/2, Y = (n-1)/2 - iy and unit size.
 *  - Sinogram: float32, row-major [n_views][n_det] (detector axis contiguous).
 *    Bin d sits at u_d = d - (n_det-1)/2; view k at theta_k = k pi / n_views
 *    unless explicit angles are given; ray (theta, u) is the line
 *    X cos(theta) + Y sin(theta) = u.
 *  - A is Joseph's ray-driven linear-interpolation projector (Eq. linCT's
 *    a_ij, which the paper leaves to a toolbox); A^T is its exact transpose.
 *  - H is the detector-axis form of the preconditioner: per view, zero-pad to
 *    P = smallest power of two >= 2 n_det, FFT, multiply by
 *    g_k = sqrt(max(|k/P|, 1/(2P))) (signed frequency), inverse FFT, crop.
 *    A V^-1 = H A (Eq. Aprecon via the Fourier slice theorem) and H = H^T, so
 *    Phi~ = H A and Phi~^T = A^T H (Eq. precondAMP_op).
 *  - Device pointers ("d_") must point to memory of the device that was
 *    current when the plan was made, be 16-byte aligned and not overlap
 *    unless stated.  Host pointers ("h_") may be pageable or pinned.
 *  - Every call is asynchronous on the CUDA stream passed as `stream`
 *    (a cudaStream_t; NULL = legacy default stream) unless stated, and the
 *    caller keeps every buffer alive until the stream reaches the call.
 *  - Ownership: the caller owns all input/output buffers and the stream; the
 *    plan owns its workspace.  A plan must not be used from two streams at
 *    the same time.
 *  - Errors: every int-returning call returns DGAMP_CT_OK (0) or a negative
 *    code below; no exception crosses the ABI.  On DGAMP_CT_ERR_CUDA the CUDA
 *    error is kept and readable through dgamp_ct_last_cuda_error().
 *    Numerical events that do not stop the method (the Newton cap, the tau_x
 *    floor) are counted in dgamp_ct_stats, not returned as errors.
 */
#ifndef DGAMP_CT_H
#define DGAMP_CT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGAMP_CT_OK                        0
#define DGAMP_CT_ERR_INVALID_ARG          -1
#define DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY -2
#define DGAMP_CT_ERR_OOM                  -3
#define DGAMP_CT_ERR_CUDA                 -4
#define DGAMP_CT_ERR_TIMEOUT              -5
#define DGAMP_CT_ERR_NONFINITE            -6

/* Limits of this build (checked by dgamp_ct_plan). */
#define DGAMP_CT_MAX_N        4096   /* image side                         */
#define DGAMP_CT_MAX_VIEWS    4096
#define DGAMP_CT_MAX_P        8192   /* detector FFT length, so n_det <= 4096 */

typedef struct {
    int32_t n;             /* image side, >= 2                                 */
    int32_t n_views;       /* number of measured views (rows of S A, Eq. Phi_mtx) */
    int32_t n_det;         /* detector bins per view, >= 2                      */
    const double* angles;  /* optional host array of n_views angles (radians);
                              NULL = theta_k = k pi / n_views.  Copied.         */
} dgamp_ct_geometry;

typedef struct {
    int32_t  denoiser;     /* 0 = proximal TV (Section 6.3), 1 = the attached CNN,
                              2 = both every iteration, prox-TV as the CNN's fallback and
                              judge: each one's risk R(x, tau_r) of Section 4.3 is estimated
                              by SURE, ||D(r) - r||^2 / N - tau_r + 2 tau_r D'(r) (D' from
                              Eq. MC_SURE for prox-TV, its eps -> 0 limit for the CNN), and
                              the lower estimate gives x and tau_x (a tie keeps prox-TV); the
                              CNN is kept only while 0 < D' < M/N (tau_x = tau_r D' is a
                              variance, and below M/N tau_r shrinks from one iteration to
                              the next when tau_p is large) */
    int32_t  k_tv;         /* Chambolle iterations per denoiser call (fixed)     */
    double   c_tv;         /* TV weight: lambda = c_tv * sqrt(tau_r)             */
    double   eps_rel;      /* MC step: eps = eps_rel * max(max|r|, 1e-6) (Eq. MC_SURE);
                              the learned denoiser takes the eps -> 0 limit instead,
                              b^T J_D(r) b / N by a forward-mode pass (eps is still logged) */
    uint64_t seed;         /* probe key (Philox4x32-10), see dgamp_ct_probe      */
    int32_t  slice_id;     /* probe counter word 2                              */
    int32_t  onsager;      /* 1 = p = z - tau_p s_prev (Algorithm 1); 0 = drop it (Section 7.1) */
    double   damp_x;       /* x <- damp_x x_new + (1-damp_x) x_old (Section 7.2); 1 = off */
    double   damp_s;       /* s <- damp_s s_new + (1-damp_s) s_old; 1 = off      */
    double   tau_x_floor;  /* tau_x = max(tau_r D', tau_x_floor * tau_r)        */
    int32_t  use_graph;    /* 1 = replay one captured CUDA graph per iteration   */
    int32_t  cnn_scale;    /* learned denoiser: 0 = blind, D(r) = r - f(r);
                              1 = D(r) = r - sigma f(r/sigma), sigma = sqrt(tau_r) */
    double   tau_x0;       /* initial tau_x (Algorithm 1 sets 1 in its own, unstated,
                              normalisation of x); default 1 */
    int32_t  truncate_z;   /* 0 (default): the output step's posterior runs over the whole
                              line (Section 4.2); 1: restricted to z >= 0 (mode max(z0, 0);
                              where clamped s = -p/tau_p and tau_s_i = 1/tau_p) */
    int32_t  storage;      /* inside dgamp_ct_solve: 0 (default) FP32; 1 = the sinograms
                              the solve keeps in memory (A x, s, H s, and H A x when the
                              three-kernel form of the tuning runs) and the image copies
                              the projector reads are stored in BF16, every sum in FP32
                              and the GAMP scalars in FP64; the counts and the denoiser's
                              images stay FP32.  The single-step entry points always take
                              FP32 buffers. */
    int32_t  output_moments; /* output step (Algorithm 1, Step 2; Appendix A): 0 (default)
                              Laplace's approximation (mode and curvature); 1 = the exact
                              posterior mean and variance of z by quadrature over the
                              window where the log posterior is within 50 of its maximum
                              (257-point trapezoid rule).  1 with truncate_z = 1 is
                              INVALID_ARG.  Inside a solve, 1 runs the three-kernel form of
                              the sinogram step.  Also used by dgamp_ct_output_step. */
    int32_t  tv_metric;    /* prox-TV norm (Section 6.3), for denoiser 0 and the TV entry
                              points: 0 (default) l2; 1 = the Mahalanobis norm of the
                              covariance Q = (V^T V)^{-1}: x = argmin 1/2 (x-r)^T Q^-1 (x-r)
                              + lambda TV(x), Q the radial gain max(|rho|, 1/(2P)) on the
                              m x m zero-padded grid of dgamp_ct_precond_image, cropped.
                              Solved by k_tv projected-gradient steps on the dual
                              (x(p) = r + lambda Q div p, p <- Proj_{|p|<=1}(p + grad x(p)
                              / (8 q_max lambda)), q_max = the largest gain, from p = 0),
                              returning x(p_k_tv). */
} dgamp_ct_options;

typedef struct {
    /* Optional caller-owned host arrays of length >= iters (NULL = skip).
       Entry t-1 holds the value computed in iteration t of Algorithm 1.  */
    double* tau_x;         /* tau_x^{t+1}                                       */
    double* tau_p;         /* tau_p^t                                           */
    double* tau_s;         /* tau_s^t                                           */
    double* tau_r;         /* tau_r^t                                           */
    double* div;           /* D'(r^t) (Eq. MC_SURE; eps -> 0 limit for the CNN) */
    /* Filled on return (always, when stats is non-NULL). */
    int32_t iters_done;
    int32_t newton_capped; /* output-step elements that hit the iteration cap   */
    int32_t tau_x_floored; /* iterations whose tau_x took the floor             */
    /* Denoiser 2 only (optional host arrays of length >= iters, NULL = skip):
       the SURE risk estimates of prox-TV and of the CNN in iteration t, and
       whether that iteration kept the CNN's output. */
    double* risk_plain;
    double* risk_learned;
    int32_t* kept_learned; /* 1 where iteration t kept the CNN's output, else 0  */
    int32_t learned_kept;  /* denoiser 2: iterations that kept the CNN's output */
} dgamp_ct_stats;

/* Flat-detector fan beam (Section 6), in pixel units with the pixel centres
   of dgamp_ct_geometry: at view angle theta the source sits at
   src_dist (sin theta, -cos theta), the detector centre at
   det_dist (-sin theta, cos theta), and bin d at the detector centre plus
   u_d (cos theta, sin theta), u_d = (d - (n_det-1)/2) det_spacing.  The
   central ray thus runs along the parallel-beam ray (theta, 0).  base.angles
   NULL = theta_k = 2 pi k / n_views (a full rotation). */
typedef struct {
    dgamp_ct_geometry base;
    double src_dist;       /* > n / sqrt(2) + 2 and <= 1e8                       */
    double det_dist;       /* > n / sqrt(2) + 2 and <= 1e8                       */
    double det_spacing;    /* bin pitch at the detector, > 0 and <= 1e4          */
} dgamp_ct_fan_geometry;

typedef struct dgamp_ct_plan_s* dgamp_ct_plan_t;
typedef struct dgamp_ct_cnn_s* dgamp_ct_cnn_t;     /* learned denoiser, see dgamp_ct_cnn_create */
typedef struct dgamp_ct_batch_s* dgamp_ct_batch_t; /* slices run phase by phase, see dgamp_ct_batch_create */

/* Fill *opt with the defaults: TV, k_tv = 20, c_tv = 3, eps_rel = 1e-3,
   seed = 12345, slice_id = 0, onsager = 1, no damping, floor 1e-6, graph on. */
int dgamp_ct_default_options(dgamp_ct_options* opt);

/* Build a plan for one geometry on the current CUDA device (Algorithm 1's
   fixed quantities): view constants, filter gains, FFT twiddles,
   ||Phi~||_F^2 (computed on the device in FP64; Algorithm 1, Steps 1 and 3)
   and the workspace.  Synchronous.  opt may be NULL (defaults).
   Errors: INVALID_ARG (NULL pointers, n < 2, n_det < 2, n_views < 1, limits),
   OOM, CUDA. */
int dgamp_ct_plan(const dgamp_ct_geometry* g, const dgamp_ct_options* opt,
                  dgamp_ct_plan_t* out);

/* Build a fan-beam plan.  A is Joseph's method along each ray's own
   direction (by columns when |v_x| >= |v_y|, else by rows; 32.32 fixed-point
   positions from FP64, so A^T applies exactly A's taps).  Phi~ = A V^-1 with
   the image-domain cone filter of dgamp_ct_precond_image (Eq. precondAMP_op;
   the detector-axis H is the parallel-beam form and does not apply), and
   dgamp_ct_plan_info reports ||Phi~||_F^2 = sum over rays of ||V^-1 a_i||^2
   (FP64, one ray at a time: plan time grows with n_views n_det).
   dgamp_ct_project / dgamp_ct_backproject apply A, A^T (precond = 0) or
   Phi~, Phi~^T (precond = 1); the output step, denoisers, probe and image
   filter work as for any plan, and so do the solve entry points: one
   iteration runs V^-1 x, A, the output step (three-kernel form), A^T and
   V^-1 with the update r = x + tau_r V^-1 A^T s, then the denoiser, all in
   FP32 storage (option storage is ignored).  dgamp_ct_filter returns
   UNSUPPORTED_GEOMETRY.  Synchronous.
   Errors: INVALID_ARG (as dgamp_ct_plan, and the distance limits), OOM, CUDA. */
int dgamp_ct_plan_fan(const dgamp_ct_fan_geometry* g, const dgamp_ct_options* opt,
                      dgamp_ct_plan_t* out);

/* The fan-beam Joseph constants dgamp_ct_plan_fan uploads, on the host (no
   device needed): for ray i = k n_det + d, its position on the interpolated
   axis at step s is (p0[i] + s pstep[i]) / 2^32 in 32.32 fixed point (the
   fractional row in column s when col[i] = 1, the fractional column in row s
   otherwise) and w[i] its path length per step.  Caller-owned host arrays
   of n_views n_det entries.  Errors: INVALID_ARG. */
int dgamp_ct_fan_ray_constants(const dgamp_ct_fan_geometry* g, int64_t* p0, int64_t* pstep, float* w,
                               int32_t* col);

/* Release the plan and its workspace (synchronises the device first).
   NULL is ignored. */
void dgamp_ct_plan_destroy(dgamp_ct_plan_t plan);

/* Replace the plan's options (e.g. another seed or k_tv).  Invalidates the
   captured graph; takes effect for the next call. */
int dgamp_ct_set_options(dgamp_ct_plan_t plan, const dgamp_ct_options* opt);

/* Scalars of the plan: ||Phi~||_F^2 (FP64) and the FFT length P. */
int dgamp_ct_plan_info(dgamp_ct_plan_t plan, double* frob_sq, int32_t* fft_len);

/* Implementation choices of a plan (they change speed, not the operator);
   dgamp_ct_plan makes them by timing on the plan's geometry.  */
typedef struct {
    int32_t filter_mode;  /* 0 = H by FFT, 1 = H as a Toeplitz product with the same
                             kernel h = IFFT_P(g) (no wrap-around since P >= 2 n_det) */
    int32_t tv_kb;        /* Chambolle steps per blocked TV launch, 1..10 */
    int32_t tv_rows;      /* rows of the image region one TV block holds: 32, 64 or 128
                             (the region is 64 columns wide) */
    int32_t sino_fused;   /* inside dgamp_ct_solve, H A x, the output step and H s run as
                             one kernel: 1 = one block per pair of views, H by FFT (needs
                             P <= 8192); 2 = a cluster of 8 blocks per view, each a slice
                             of the bins, H as its Toeplitz product and s shared through
                             distributed shared memory (needs n_det <= 1792); 0 = three
                             kernels, H in filter_mode's form.  The plan times the forms
                             the geometry allows and keeps the faster; filter_mode alone
                             governs the single-step entry points */
    int32_t bp_mode;      /* A^T: 0 = pixel-driven gather (each pixel finds the <= 2 rays
                             of a view that tap it), 1 = ray-driven over 16 x 16 image
                             tiles with per-warp shared-memory accumulators.  Both are the
                             exact transpose of the projector and deterministic */
    int32_t pj_seg;       /* A: warps that split the step range of one group of 32 rays,
                             8, 16 or 32 (the partial sums are added in a fixed order) */
    int32_t tv_vrows;     /* rows of the TV region each thread holds: 4; 8 or 2 (then the
                             region is 64 rows high whatever tv_rows says: half or twice
                             the threads of the 4-row form, twice or half the pixels
                             each).  Inside a solve, both images of the MC pair share a
                             thread for 4-row threads in 32- or 64-row regions and for
                             2-row threads */
    int32_t pj_band;      /* A: 0 = the ray-group form above; 16 or 32 = the banded form:
                             a block copies that many consecutive lines of the staged image
                             into shared memory and takes the steps inside them of a
                             contiguous chunk of rays, writing per-band partial sums that a
                             second kernel adds in band order (inside a solve with
                             sino_fused = 2 the cluster sinogram kernel adds them itself).
                             These are the sums of the ray-group form with the same split.
                             Offered where a 16-line band of FP32 fits in 100 KB, parallel
                             beam only.  Setting pj_seg with pj_band < 0 picks the
                             ray-group form */
    int32_t pj_waves;     /* A, banded form: 1 or 2 full waves of resident blocks; the
                             rays are cut into that many chunks per band */
} dgamp_ct_tuning;

/* get: writes the plan's choices.  set: fields < 0 keep the current choice;
   out-of-range values return INVALID_ARG, a sino_fused form or a pj_band the
   plan does not allow UNSUPPORTED_GEOMETRY (nothing is changed then).
   Setting drops the captured graph. */
int dgamp_ct_get_tuning(dgamp_ct_plan_t plan, dgamp_ct_tuning* out);
int dgamp_ct_set_tuning(dgamp_ct_plan_t plan, const dgamp_ct_tuning* tuning);

/* z = A x (precond = 0) or z = Phi~ x = H A x (precond = 1); Eq. linCT and
   Algorithm 1, Step 1.  d_img [n][n] -> d_sino [n_views][n_det]. */
int dgamp_ct_project(dgamp_ct_plan_t plan, const float* d_img, float* d_sino,
                     int precond, void* stream);

/* x = A^T s (precond = 0) or x = Phi~^T s = A^T H s (precond = 1);
   Eq. precondAMP_op and Algorithm 1, Step 3.  d_sino -> d_img. */
int dgamp_ct_backproject(dgamp_ct_plan_t plan, const float* d_sino, float* d_img,
                         int precond, void* stream);

/* d_out = H d_in on [n_views][n_det] sinograms (Eq. Aprecon, detector-axis
   form).  d_in == d_out is allowed. */
int dgamp_ct_filter(dgamp_ct_plan_t plan, const float* d_in, float* d_out, void* stream);

/* Poisson output step (Algorithm 1, Step 2; Section 4.2 and Appendix A under
   the corrected Laplace reading): p = z - tau_p s_prev, z0 = mode of
   N(z; p, tau_p) Poisson(y; I0 e^{-z}), s = (z0 - p)/tau_p,
   tau_s = mean_i I0 e^{-z0_i} / (1 + tau_p I0 e^{-z0_i}).
   With the plan's option truncate_z = 1 the posterior is restricted to
   z >= 0.  d_s_prev may be NULL (treated as 0) and may equal d_s.  *d_tau_s
   (one device double) receives tau_s. */
int dgamp_ct_output_step(dgamp_ct_plan_t plan, const float* d_z, const float* d_y,
                         const float* d_s_prev, double I0, double tau_p,
                         float* d_s, double* d_tau_s, void* stream);

/* Proximal TV denoiser (Section 6.3): d_x = argmin 1/2||x - r||^2 + lambda TV(x)
   by k_tv Chambolle iterations from a zero dual (tau = 1/8); with the plan's
   option tv_metric = 1 the same prox in the (V^T V)^{-1} norm (see the
   option).  [n][n]. */
int dgamp_ct_denoise_tv(dgamp_ct_plan_t plan, const float* d_r, double lambda,
                        float* d_x, void* stream);

/* Denoiser plus its Monte-Carlo divergence (Eq. D_in and Eq. MC_SURE, K = 1):
   d_x = D(r), *d_div = b^T (D(r + eps b) - D(r)) / (N eps) with b the probe
   of iteration t (dgamp_ct_probe) and eps = eps_rel max(max|r|, 1e-6).
   lambda = c_tv sqrt(tau_r).  d_div: one device double. */
int dgamp_ct_denoise_div(dgamp_ct_plan_t plan, const float* d_r, double tau_r,
                         int32_t t, float* d_x, double* d_div, void* stream);

/* The Gaussian probe b of iteration t: Philox4x32-10 (Salmon et al., SC'11)
   with key (seed mod 2^32, seed >> 32) and counter (i/4, t, slice_id, 0),
   word i%4, u = (word + 1/2) 2^-32, Box-Muller on word pairs (0,1), (2,3).
   If d_words != NULL it receives the raw words (uint32, n of them). */
int dgamp_ct_probe(dgamp_ct_plan_t plan, int32_t t, int64_t n, float* d_b,
                   uint32_t* d_words, void* stream);

/* Image-domain preconditioner map (Algorithm 1, return line; Eq. precondAMP):
   inverse = 1: d_out = V^-1 d_in (radial gain sqrt(max(rho, 1/(2P)))),
   inverse = 0: d_out = V d_in (reciprocal gain); both on a 2n x 2n
   zero-padded 2-D FFT, cropped to [n][n].  d_in == d_out is allowed. */
int dgamp_ct_precond_image(dgamp_ct_plan_t plan, const float* d_in, float* d_out,
                           int inverse, void* stream);

/* D-GAMP-CT, Algorithm 1: x = 0, tau_x = 1, then `iters` iterations of
   Steps 1-4 with the Poisson output step and the plan's denoiser, and
   d_mu_out = V^-1 x.  d_counts: [n_views][n_det] float32 counts (integer
   valued, >= 0).  d_x_out (nullable) receives the final x.  With stats !=
   NULL the call synchronises the stream and fills it; otherwise it only
   enqueues work.  Errors: INVALID_ARG (iters < 1, I0 <= 0 or not finite),
   CUDA, NONFINITE (only with stats: a non-finite scalar appeared), TIMEOUT
   (only with stats, learned denoiser: a tensor-core convolution's bounded
   wait ran out, so the image is not valid; without stats the network keeps
   the flag and its next synchronous call -- a solve with stats or on host
   buffers, a denoise, a gradient pass -- returns TIMEOUT). */
int dgamp_ct_solve(dgamp_ct_plan_t plan, const float* d_counts, double I0,
                   int32_t iters, float* d_mu_out, float* d_x_out,
                   dgamp_ct_stats* stats, void* stream);

/* Attach a learned denoiser to the plan (NULL detaches it).  With
   opt.denoiser = 1 Step 4 then runs D_sigma(r) = r - sigma f(r/sigma),
   sigma = sqrt(tau_r), on r and r + eps b as one batch, and the divergence
   of Eq. MC_SURE from the two outputs.  The network is not owned and must
   outlive its use; it is not re-entrant either (one stream at a time).
   Allocates the pair's workspace; synchronous. */
int dgamp_ct_plan_set_cnn(dgamp_ct_plan_t plan, dgamp_ct_cnn_t net);

/* dgamp_ct_solve without the graph, recording for t = 1..iters the
   denoiser input r^t into d_r_trace[t-1] ([iters][n][n] device floats,
   nullable) and tau_r^t into h_tau_r[t-1] (host, nullable; the call then
   synchronises).  Used to harvest training pairs from the method's own
   iterates. */
int dgamp_ct_solve_trace(dgamp_ct_plan_t plan, const float* d_counts, double I0, int32_t iters,
                         float* d_mu_out, float* d_r_trace, double* h_tau_r, void* stream);

/* dgamp_ct_solve on HOST buffers: copies h_counts to the device, solves and
   copies mu back to h_mu_out; returns after the result is in h_mu_out.
   Errors as dgamp_ct_solve; TIMEOUT is reported with or without stats. */
int dgamp_ct_solve_host(dgamp_ct_plan_t plan, const float* h_counts, double I0,
                        int32_t iters, float* h_mu_out, dgamp_ct_stats* stats,
                        void* stream);

/* A batch of independent slices (the paper reconstructs one 2-D slice per
   solve, Section 6; a volume or a queue of scans is many of them): slice i
   is dgamp_ct_solve(plans[i], d_counts[i], I0[i], iters, d_mu_out[i]).  Plans
   may have different geometries and denoisers but must be distinct and made
   on the current device.  The slices are scheduled largest-first (work =
   n_views * n_det * n, the Joseph steps of one projection) over up to 16
   streams that fork from and join back into `stream`, so small slices run
   concurrently; the call only enqueues work unless stats != NULL, in which
   case it synchronises and fills stats[0..n-1].  The result of each slice is
   bit-identical to its own dgamp_ct_solve.  Learned plans need a network
   each (dgamp_ct_cnn_create per slice, same weights): a network's
   activation workspace serves one solve at a time, and the slices run
   concurrently.  Errors: INVALID_ARG (n < 0, a NULL pointer, a repeated
   plan, two learned plans sharing a network, a plan of another device, a
   learned plan without a network, I0 <= 0 or not finite, iters < 1), CUDA,
   NONFINITE and TIMEOUT (only with stats; the first error met in slice
   order). */
int dgamp_ct_solve_batched(int32_t n, const dgamp_ct_plan_t* plans, const float* const* d_counts,
                           const double* I0, int32_t iters, float* const* d_mu_out,
                           dgamp_ct_stats* stats, void* stream);

/* A batch that runs every phase of an iteration as ONE launch over all its
   slices (the same slices as dgamp_ct_solve_batched: independent, any mix of
   image sizes, view and bin counts and doses; Section 6 reconstructs one
   slice per solve).  Each launch covers a work list of (slice, block)
   items -- A x, the sinogram step (H A x, the output step and H s; a cluster
   of 8 blocks per view), A^T with the update, the probe, and the prox-TV
   launches (20 Chambolle steps: 2 launches) -- so one iteration of any
   number of slices is 6 launches, captured once as a graph and replayed.
   Slice i's result is bit-identical to dgamp_ct_solve on plans[i] with the
   batch's implementation choices (dgamp_ct_tuning pj_seg = 16, pj_band = 0, bp_mode = 1,
   sino_fused = 2, tv_kb = 10, tv_rows = 64, tv_vrows = 4); each plan's own tuning is not
   used here.
   create: n >= 1 distinct parallel-beam plans of the current device with the
   prox-TV denoiser (denoiser = 0, tv_metric = 0, output_moments = 0), one
   storage type and one k_tv (a multiple of 10), c_tv > 0, n_det <= 1792.
   The batch refers to the plans' workspaces: they must outlive it, and a
   plan must not be solved on its own while a batch solve using it runs.
   groups >= 1: the slices are split largest-first into that many groups
   (at most n); each group's six launches form one branch of the iteration
   graph and the branches run concurrently, so one group's denoiser can
   overlap another's projection.  groups = 1 is the single launch per phase.
   Errors: INVALID_ARG, UNSUPPORTED_GEOMETRY, OOM, CUDA.  Synchronous. */
int dgamp_ct_batch_create(int32_t n, const dgamp_ct_plan_t* plans, int32_t groups, dgamp_ct_batch_t* out);
void dgamp_ct_batch_destroy(dgamp_ct_batch_t batch);
/* Solve every slice: slice i takes d_counts[i] ([n_views][n_det] float32 of
   plans[i]) and I0[i], runs `iters` iterations and writes mu to d_mu_out[i]
   ([n][n]).  Stream-ordered; with stats != NULL it synchronises and fills
   stats[0..n-1] (errors as dgamp_ct_solve_batched). */
int dgamp_ct_batch_solve(dgamp_ct_batch_t batch, const float* const* d_counts, const double* I0,
                         int32_t iters, float* const* d_mu_out, dgamp_ct_stats* stats, void* stream);
/* Kernels one dgamp_ct_batch_solve of `iters` iterations launches (for all slices together):
   1 + iters * groups * 6 + 4. */
int64_t dgamp_ct_batch_launches(dgamp_ct_batch_t batch, int32_t iters);

/* Host-only scheduler (no device work): assigns n jobs of the given work
   (>= 0) to `queues` queues, largest job first, each to the least-loaded
   queue (ties: the lowest queue index; equal work keeps input order).
   queue_of[i] receives job i's queue; load (nullable, `queues` entries) the
   total work per queue.  Used for the streams of dgamp_ct_solve_batched and
   to split a batch across processes.  Errors: INVALID_ARG. */
int dgamp_ct_schedule_lpt(int32_t n, const int64_t* work, int32_t queues, int32_t* queue_of, int64_t* load);

/* Number of kernels one dgamp_ct_solve enqueues for `iters` iterations. */
int64_t dgamp_ct_solve_launches(dgamp_ct_plan_t plan, int32_t iters);

/* Kernel-level timing of one Algorithm 1 iteration: enqueues the iteration's
   kernels one at a time on `stream` with a CUDA event before and after each,
   `reps` times, and writes the mean duration (ms) of each kernel to h_ms
   (host array of `cap` doubles) in launch order: A x; H (z), output step,
   H (s) -- one fused kernel when the tuning's sino_fused is 1 or 2; A^T + update,
   probe input, then the denoiser: the blocked TV launches (the last one
   final), or the learned network's pair of passes and its final step.
   *count receives the number of kernels.  The iterations run on the plan's
   current state (normally that of the last dgamp_ct_solve) and advance it.
   Synchronous. */
int dgamp_ct_profile_iteration(dgamp_ct_plan_t plan, int32_t reps, double* h_ms, int32_t cap,
                               int32_t* count, void* stream);

/* Measured FP32 FMA throughput of the current GPU (the denominator of the
   ALU rooflines of the issue-bound kernels; no counterpart in the paper):
   every SM runs as many 256-thread blocks as fit, each thread 8 independent
   FMA chains, `reps` timed launches after one warm-up, CUDA events on
   `stream`.  *h_tflops receives TFLOP/s (an FMA counts as 2 FLOP) and, if
   h_sms is not NULL, *h_sms the SM count.  Changes no clock or other GPU
   setting.  Allocates a small device buffer for the duration of the call;
   synchronous. */
int dgamp_ct_measure_fp32_peak(int32_t reps, double* h_tflops, int32_t* h_sms, void* stream);

/* The same with the chains as packed FP32 pairs (two FMAs per instruction,
   sm_100 and later), counting 4 FLOP per instruction: whether the packed
   form raises the FMA rate or only saves issue slots.  As above otherwise. */
int dgamp_ct_measure_fp32x2_peak(int32_t reps, double* h_tflops, int32_t* h_sms, void* stream);

/* ---------------------------------------------------------------------------
   Learned denoiser (Step 4 of Algorithm 1 with a trained network; the paper's
   Section 4.3 admits any denoiser and Section 1 points to residual CNNs).
     f: `layers` 3x3 same-padded convolutions, 1 -> 64 -> ... -> 64 -> 1,
        a bias per output channel, ReLU after every layer but the last;
     D_sigma(r) = r - sigma f(r / sigma), sigma = sqrt(tau_r) inside a solve.
   Hidden activations are BF16, accumulation FP32 (tensor cores).  Parameters
   are FP32 masters in this flat order, per layer l: W_l[ky][kx][c_in][c_out]
   then b_l[c_out]; the compute copies of the weights are rounded to BF16.
   Images: float32 [batch][H][W] device buffers.  h_sigma: host array of
   `batch` positive floats.  The network object owns its parameters, Adam
   state and workspace (grown on demand).  Every wait inside the tensor-core
   convolution is bounded (2 s); a wait that runs out sets a flag in the
   network instead of hanging.  denoise, denoise_jvp, gradients and
   train_step synchronise the stream before they return and then report a
   flag that was set as DGAMP_CT_ERR_TIMEOUT (clearing it); their outputs
   are then not valid. */

/* New network with He-initialised weights (std sqrt(2/(9 c_in)), last layer
   x0.1) from `seed`, zero biases.  3 <= layers <= 64.  Synchronous. */
int dgamp_ct_cnn_create(int32_t layers, uint64_t seed, dgamp_ct_cnn_t* out);
void dgamp_ct_cnn_destroy(dgamp_ct_cnn_t net);
int64_t dgamp_ct_cnn_num_params(dgamp_ct_cnn_t net);
/* Copy parameters in/out (host float32, exactly num_params values);
   set_params also resets the Adam state.  Synchronous. */
int dgamp_ct_cnn_set_params(dgamp_ct_cnn_t net, const float* h_params, int64_t count);
int dgamp_ct_cnn_get_params(dgamp_ct_cnn_t net, float* h_params, int64_t count);
/* d_out = D_sigma(d_r) for a batch of images. */
int dgamp_ct_cnn_denoise(dgamp_ct_cnn_t net, const float* d_r, const float* h_sigma, int32_t batch,
                         int32_t H, int32_t W, float* d_out, void* stream);
/* d_out = D_sigma(d_r) and d_jb = J_D(d_r) d_b, the directional derivative of
   the denoiser at d_r along d_b (forward mode through the ReLU network:
   J_D b = b - sigma J_f(r / sigma)(b / sigma)), for one H x W image.  This is
   the pass a learned-denoiser solve uses for D' = b^T J_D b / N, the
   eps -> 0 limit of Eq. MC_SURE.  d_r, d_b, d_out, d_jb: device, H*W floats
   each; sigma > 0 and finite, else DGAMP_CT_ERR_INVALID_ARG. */
int dgamp_ct_cnn_denoise_jvp(dgamp_ct_cnn_t net, const float* d_r, const float* d_b, float sigma, int32_t H,
                             int32_t W, float* d_out, float* d_jb, void* stream);
/* Training loss mean(((D_sigma(r) - x) / sigma)^2) over the batch (each image's
   error divided by its own noise level; for sigma = 1 the plain mean squared
   error) and its gradient with respect to every parameter (h_grad: num_params
   floats, may be NULL). */
int dgamp_ct_cnn_gradients(dgamp_ct_cnn_t net, const float* d_r, const float* d_x, const float* h_sigma,
                           int32_t batch, int32_t H, int32_t W, double* h_loss, float* h_grad,
                           void* stream);
/* Timeout test switch (on = 1 or 0).  While it is on, every tensor-core
   convolution of this network first waits with a 1 ms limit on a barrier
   that nothing arrives at, records the timeout and returns without issuing
   any copy or tensor-core instruction, so the calls above return
   DGAMP_CT_ERR_TIMEOUT and the context stays usable.  Synchronises the
   device when the setting changes; solves re-capture their graph. */
int dgamp_ct_cnn_test_timeout(dgamp_ct_cnn_t net, int32_t on);
/* One Adam step (beta 0.9/0.999, eps 1e-8, learning rate lr) on that loss. */
int dgamp_ct_cnn_train_step(dgamp_ct_cnn_t net, const float* d_r, const float* d_x, const float* h_sigma,
                            int32_t batch, int32_t H, int32_t W, float lr, double* h_loss, void* stream);

/* The output step of dgamp_ct_output_step, for callers that cannot allocate
   device memory (the paper has no counterpart: this is a deployment aid).
   A host that reserves all GPU memory for its own pool and forbids library
   allocations, or a latency-critical loop that must not pay for an
   allocation, can call it without a plan: it allocates nothing, neither
   with cudaMalloc nor through any library.  Its scratch (the per-block
   partial sums of tau_s and an arrival counter, about 8 KiB) lives in a
   fixed __device__ array inside the library that every GPU loading the
   library keeps until the process exits.
   Arguments are those of dgamp_ct_output_step plus M, the number of
   measurements (1 <= M <= DGAMP_CT_NOALLOC_MAX_M; larger M returns
   DGAMP_CT_ERR_INVALID_ARG).  The first call on a device looks up the
   scratch's device address with the device current; make that first call
   before any stream capture.  The address belongs to the device's current
   context: after cudaDeviceReset, or when the primary context is released
   and created again, the next call finds a new context id and looks the
   address up again (so make that call outside a capture too).  All calls
   share the one scratch array: calls
   that overlap on the GPU (other streams, other host threads) race and
   must be serialised by the caller. */
#define DGAMP_CT_NOALLOC_MAX_M (1LL << 24)
int dgamp_ct_output_step_noalloc(const float* d_z, const float* d_y, const float* d_s_prev,
                                 int64_t M, double I0, double tau_p, float* d_s, double* d_tau_s,
                                 void* stream);

/* Human-readable text for an error code (static storage). */
const char* dgamp_ct_strerror(int code);

/* The CUDA error (cudaError_t value) behind the last DGAMP_CT_ERR_CUDA. */
int dgamp_ct_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DGAMP_CT_H */
