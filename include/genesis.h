/*
 * genesis.h - C ABI of the GB300 (sm_103a) implementation of the GENESIS
 * Milne-Eddington genetic-algorithm Stokes inversion of Harker & Mighell,
 * "A GPU-Computing Approach to Solar Stokes Profile Inversion" (2012).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an int status: ME_OK (0) or a negative ME_E* code.
 *    me_last_error() returns a thread-local message for the last failure.
 *  - Pointers documented "dev" are device pointers on the current CUDA device;
 *    "host" pointers are read during the call only.  The caller owns every
 *    buffer; no entry point allocates device memory, except serve_create()
 *    and the serve handle it returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it and the call returns without
 *    synchronising; results are valid once the stream reaches that point.
 *  - Invalid arguments are rejected on the host (ME_EINVAL) before anything
 *    is launched; a failed launch returns ME_ECUDA.
 *  - Parameter vectors have M = ME_NPAR = 9 entries in this fixed order
 *    (Section 5, model vector p; v_LOS replaces lambda0 and S0, S1 replace
 *    S0, beta0 with beta0 = S1/S0), or M = 10 with the fill fraction:
 *       0 B [G]          1 theta inclination [deg]   2 chi azimuth [deg]
 *       3 v_LOS [km/s]   4 Doppler width [mA] at lambda_dop_A
 *       5 damping a      6 eta0 (line/continuum opacity ratio)
 *       7 S0             8 S1 (source function S0 + S1 tau)
 *       9 alpha (me_problem.fill_fraction = 1; Section 5.2)
 *  - Stokes arrays are [n][4][n_lambda] (I, Q, U, V), pixel-major, of the
 *    problem's dtype (float for ME_F32, double for ME_F64).
 */
#ifndef GENESIS_H
#define GENESIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define ME_OK 0
#define ME_EINVAL (-1)    /* invalid argument (message in me_last_error)   */
#define ME_ENOMEM (-2)    /* allocation failed (serve handle only)         */
#define ME_ECUDA (-3)     /* CUDA runtime error                            */
#define ME_EAGAIN (-4)    /* serve queue full, retry later                 */
#define ME_EPENDING (-5)  /* serve request still running                   */
#define ME_ETIMEOUT (-6)  /* a bounded wait gave up                        */
#define ME_ENOTFOUND (-7) /* unknown serve ticket                          */

/* ------------------------------------------------------------ limits/enums */
#define ME_NPAR 9      /* model parameters without the fill fraction          */
#define ME_NPAR_MAX 10 /* with it: parameter 9 is alpha (Section 5.2)         */
#define ME_MAX_LINES 4
#define ME_MAX_LAMBDA 512
#define ME_MAX_COMP 9 /* Zeeman components per group in a full pattern (J <= 4) */
#define ME_MIN_POP 32
#define ME_MAX_POP 1024

#define ME_F32 0 /* float cube, FP32 synthesis and chi2            */
#define ME_F64 1 /* double cube, FP64 synthesis and chi2           */

#define ME_W_INVMAX 0 /* Section 5.4 inverse-max weights from the data  */
#define ME_W_USER 1   /* caller-supplied w[npix][4]                     */

/*
 * One spectral line (Table 1).
 *   lambda0_A  rest wavelength [A]
 *   g_eff      effective Lande factor (pattern == 0): an effective Zeeman
 *              triplet, sigma_blue, pi, sigma_red at v + v_B, v, v - v_B with
 *              v_B = 4.6686e-13 g_eff lambda0^2 B / dlambda_D (Section 5)
 *   eta_ratio  eta0 of this line divided by the eta0 parameter (1 for the
 *              reference line); all lines add into one propagation matrix.
 *   pattern    1: use the line's full Zeeman pattern (Section 5: computed at
 *              start-up from the transition), built from the lower level
 *              (j_lower, g_lower) and upper level (j_upper, g_upper) in LS
 *              coupling: components M_u -> M_l, q = M_l - M_u (-1 sigma_blue,
 *              0 pi, +1 sigma_red), shift g_l M_l - g_u M_u Larmor units,
 *              strengths normalised to 1 per group.  |j_lower - j_upper| <= 1,
 *              integer J <= 4, not both 0.
 */
typedef struct me_line {
    double lambda0_A;
    double g_eff;
    double eta_ratio;
    int pattern;
    int j_lower;
    int j_upper;
    double g_lower;
    double g_upper;
} me_line;

/*
 * The synthesis problem (Section 5): line list, wavelength grid and geometry.
 *   n_lines       1..ME_MAX_LINES
 *   n_lambda      1..ME_MAX_LAMBDA
 *   lambda_A      HOST pointer to n_lambda wavelengths [A]; copied into the
 *                 launch parameters, so the caller may free it after the call
 *   lambda_dop_A  wavelength at which parameter 4 (Doppler width) is quoted;
 *                 line l uses dlambda_D * lambda0_l / lambda_dop_A
 *   mu            cosine of the heliocentric angle used when mu_px is NULL
 *   dtype         ME_F32 or ME_F64: element type of obs/stokes arrays and the
 *                 arithmetic of synthesis and chi2
 *   fill_fraction 1: the magnetic fill fraction alpha of Section 5.2 is a 10th
 *                 parameter, Stokes = alpha S_mag + (1 - alpha) I_nm (1,0,0,0)
 *                 with I_nm = S0 + mu S1 / (1 + sum_l eta0_l Re w(v_l, a)), the
 *                 same atmosphere without a field; 0: 9 parameters.
 *
 * Every parameter array of the interface is [n][M] with M = ME_NPAR +
 * fill_fraction, in the order B [G], theta [deg], chi [deg], v_LOS [km/s],
 * Doppler width [mA], damping a, eta0, S0, S1 (, alpha).
 */
typedef struct me_problem {
    int n_lines;
    me_line line[ME_MAX_LINES];
    int n_lambda;
    const double *lambda_A;
    double lambda_dop_A;
    double mu;
    int dtype;
    int fill_fraction;
} me_problem;

/* Parameter bounds u_j <= p_j <= v_j (Section 3, Eq. decode) for j < M; the
 * entries beyond M are ignored.  lo[5] (damping) must be >= 0, lo[4] (Doppler
 * width) > 0 and, with the fill fraction, 0 <= lo[9] < hi[9] <= 1. */
typedef struct me_bounds {
    double lo[ME_NPAR_MAX];
    double hi[ME_NPAR_MAX];
} me_bounds;

/*
 * Genetic-algorithm settings (Section 3, Algorithm 1; Section 5.6).
 *   npop         population, a multiple of 32 in [ME_MIN_POP, ME_MAX_POP]
 *   ngen         generations (>= 0)
 *   nsamp        restart period: every nsamp generations (t < ngen) the worst
 *                half is replaced by new Sobol points; <= 0 disables restarts
 *   pc           crossover probability of a pair
 *   pmut_lsb     per-bit mutation probability of the least significant bit;
 *                bit b (0 = MSB) uses pmut_lsb * pmut_ratio^(15 - b)
 *   seed         Philox key (low, high 32 bits)
 *   weight_mode  ME_W_INVMAX or ME_W_USER
 */
typedef struct ga_config {
    int npop;
    int ngen;
    int nsamp;
    double pc;
    double pmut_lsb;
    double pmut_ratio;
    uint64_t seed;
    int weight_mode;
} ga_config;

/* Zeeman components of a line (host only, no GPU): for each group (0 =
 * sigma_blue, 1 = pi, 2 = sigma_red) the count n[g], the shifts in Larmor
 * units (toward longer wavelength) and the strengths.  An effective triplet
 * (pattern == 0) reports one component per group at -g_eff, 0, +g_eff. */
int me_zeeman_components(const me_line *line, int n[3], double shift[3][ME_MAX_COMP],
                         double strength[3][ME_MAX_COMP]);

/* Thread-local message describing the last failed call ("" if none). */
const char *me_last_error(void);

/* ABI version of this library (major * 100 + minor). */
int me_version(void);

/*
 * me_synth - Unno-Rachkovsky Stokes vectors of n parameter vectors
 * (Section 5: K = 1 + eta0 Phi, Stokes = S0 e + mu S1 K^-1 e, I_c = S0 + mu S1).
 *   params  dev double [n][M]
 *   mu_px   dev double [n] or NULL (then pb->mu)
 *   stokes  dev [n][4][n_lambda] of pb->dtype (output)
 * n = 0 is a no-op.
 */
int me_synth(const me_problem *pb, const double *params, const double *mu_px, int n,
             void *stokes, void *stream);

/*
 * me_synth_jac - analytic Jacobian d stokes / d p of the same synthesis
 * (the derivative of Section 5's closed form, with w'(z) = -2 z w + 2i/sqrt(pi)).
 *   stokes  dev [n][4][n_lambda] of pb->dtype, or NULL
 *   jac     dev [n][4][n_lambda][M] of pb->dtype (output)
 */
int me_synth_jac(const me_problem *pb, const double *params, const double *mu_px, int n,
                 void *stokes, void *jac, void *stream);

/*
 * me_synth_vjp - vector-Jacobian product grad_params = J^T grad_stokes, the
 * adjoint used by the torch.autograd.Function wrapper.
 *   grad_stokes  dev [n][4][n_lambda] of pb->dtype
 *   grad_params  dev double [n][M] (output)
 */
int me_synth_vjp(const me_problem *pb, const double *params, const double *mu_px, int n,
                 const void *grad_stokes, double *grad_params, void *stream);

/*
 * me_chi2 - Eq. chisq, chi2 = (1/nu) sum_s w_s^2 sum_j (O - M)^2 with
 * nu = 4 n_lambda - M, evaluated in FP64 for each pixel's parameters.
 *   obs   dev [npix][4][n_lambda] of pb->dtype
 *   w     dev double [npix][4] (ME_W_USER) or NULL (inverse-max, Section 5.4)
 *   chi2  dev double [npix] (output)
 */
int me_chi2(const me_problem *pb, const void *obs, const double *w, const double *mu_px,
            int npix, const double *params, double *chi2, void *stream);

/*
 * ga_invert_batch - Algorithm 1 per pixel, one thread block per pixel with the
 * population resident in shared memory for all generations:
 * Sobol initial population, then per generation binary tournament selection,
 * one-point crossover, LSB-biased mutation, elitism and fitness evaluation
 * (synthesis + chi2 in pb->dtype arithmetic), with worst-half Sobol restarts
 * every nsamp generations (Section 5.6).  Philox4x32-10 counters are keyed by
 * pixel id = pixel_id0 + i, so a pixel's result does not depend on the batch.
 *   obs         dev [npix][4][n_lambda] of pb->dtype
 *   w           dev double [npix][4] if cfg->weight_mode == ME_W_USER, else NULL
 *   mu_px       dev double [npix] or NULL
 *   best        dev double [npix][M]: decoded best individual (output)
 *   chi2        dev double [npix]: FP64 re-evaluation of best (output)
 *   best_genes  dev uint16 [npix][M] or NULL (output)
 */
int ga_invert_batch(const me_problem *pb, const void *obs, const double *w,
                    const double *mu_px, int npix, uint64_t pixel_id0,
                    const me_bounds *bounds, const ga_config *cfg, double *best,
                    double *chi2, uint16_t *best_genes, void *stream);

/*
 * ga_count_evaluations - the same GA as ga_invert_batch (float cubes,
 * npop <= 256) run by a separate instantiation that also counts work:
 * counts dev uint64[6] receives (added to its contents) the number of
 * syntheses (fitness evaluations), of Faddeeva evaluations by Weideman's
 * series (|z|^2 <= 21), of all Faddeeva evaluations, of those in the far
 * field (|z|^2 > 360), of those in the middle shell (21 < |z|^2 <= 36) and
 * of those in the outer shell (80 < |z|^2 <= 360; the rest, 36 < |z|^2 <= 80,
 * use the 3rd convergent), each real wavelength point classified by its own
 * region (the algorithm's work, whatever branch a point's pair or warp took).
 * The arithmetic and the result `best` are those of ga_invert_batch; the
 * counts turn into algorithmic flops for roofline reporting.
 */
int ga_count_evaluations(const me_problem *pb, const void *obs, const double *w,
                         const double *mu_px, int npix, uint64_t pixel_id0,
                         const me_bounds *bounds, const ga_config *cfg, double *best,
                         unsigned long long *counts, void *stream);

/*
 * ga_fitness - the fitness that ga_invert_batch ranks its population by, for
 * caller-given individuals: Eq. chisq of the Section 5 synthesis, in
 * pb->dtype arithmetic (FP32: the packed two-wavelength pair path with its
 * warp-voted w(z) regions; FP64: the per-wavelength path), with the GA's
 * launch shape and the kernel instantiation ga_invert_batch would choose.
 * One thread block per pixel and one thread per individual; only threads
 * k < nactive evaluate, inside a divergent branch as the GA's restarts do
 * (nactive = npop / 2 = 16 of npop = 32 is the restart of the smallest
 * population), so the w(z) branch votes run over exactly those lanes.  A
 * verification entry point: it exposes the GA's evaluation so that it can be
 * compared with an independent FP64 synthesis.
 *   obs      dev [npix][4][n_lambda] of pb->dtype
 *   w        dev double [npix][4] (the caller's weights) or NULL (Section 5.4
 *            inverse-max weights of the pixel, as ME_W_INVMAX)
 *   mu_px    dev double [npix] or NULL
 *   npop     threads per block, a multiple of 32 in [ME_MIN_POP, ME_MAX_POP]
 *   nactive  1..npop
 *   params   dev double [npix][npop][M], each rounded to pb->dtype (the GA
 *            decodes its genes in that precision)
 *   fitness  dev double [npix][npop] (output): chi2 / nu of individual k for
 *            k < nactive, as computed (NaN is not replaced); rows k >= nactive
 *            are not written
 *   resid    dev [npix][npop][4][n_lambda] of pb->dtype or NULL (output): the
 *            residuals O - S whose weighted squares the fitness sums; rows
 *            k >= nactive are not written
 * Errors: ME_EINVAL for an invalid problem, npop, nactive or a population and
 * grid that exceed shared memory; ME_ECUDA for a failed launch.
 */
int ga_fitness(const me_problem *pb, const void *obs, const double *w, const double *mu_px, int npix,
               int npop, int nactive, const double *params, double *fitness, void *resid, void *stream);

/*
 * me_faddeeva_pairs - the FP32 Voigt and Faraday-Voigt profiles of the GA's
 * pair path, H + iF = w(x + i a) (Section 5: phi = Re w, psi = Im w), for
 * caller-given arguments, through the same branch choice the fitness makes:
 * Weideman's series, the 5th and 3rd convergents of the Laplace continued
 * fraction and the far-field approximant, chosen per pair and voted across
 * the warp.  Thread i (32 to a warp, in index order) holds pair i; a ragged n
 * leaves the last warp partial, and its vote runs over the lanes present.  A
 * verification entry point.
 *   x     dev float [n][2]: the pair's two real arguments (8-byte aligned)
 *   a     dev float [n]: the pair's damping a >= 0
 *   v_b   dev float [n]: Zeeman splitting in Doppler units (mode 2 only;
 *         may be NULL otherwise)
 *   mode  0: one component, regions tested from the outside in (the branch
 *            of full-pattern components);
 *         1: one component, tested from the inside out (components of an
 *            effective triplet near a line core);
 *         2: an effective triplet with pi arguments x and sigma arguments
 *            x +- v_b, its level voted as a whole first, as the fitness does
 *   out   dev float (output): modes 0, 1: [n][2][2] = (Re w, Im w) of each
 *         point; mode 2: [n][2][6] = per point the unit-strength profile
 *         sums (phi_pi, psi_pi, phi_b + phi_r, psi_b + psi_r, phi_r - phi_b,
 *         psi_r - psi_b), phi_b = Re w(x + v_b + i a), phi_r = Re w(x - v_b + i a)
 * Errors: ME_EINVAL for n < 0, a bad mode, NULL or misaligned pointers.
 */
int me_faddeeva_pairs(const float *x, const float *a, const float *v_b, int n, int mode, float *out,
                      void *stream);

/*
 * lm_polish - Levenberg-Marquardt refinement of each pixel's parameters
 * (Levenberg 1944, Marquardt 1963): FP32 analytic Jacobian, normal equations
 * (J^T W^2 J + lambda D) delta = J^T W^2 r summed in the cube's precision
 * and solved by Cholesky in FP64, trial step with the azimuth wrapped into [0, 180) and clamped to the
 * bounds, accepted when chi2 decreases.  iters trial steps are taken.
 *   params_inout  dev double [npix][M]
 *   chi2_out      dev double [npix]: FP64 chi2 of the final parameters
 */
int lm_polish(const me_problem *pb, const void *obs, const double *w, const double *mu_px,
              int npix, const me_bounds *bounds, int iters, double lambda0,
              double *params_inout, double *chi2_out, void *stream);

/*
 * me_fp32_peak - FP32 FMA-pipe throughput probe.  The paper has no
 * counterpart: it measures the FP32 peak of the GPU at the clock it runs, the
 * denominator of the GA kernel's roofline fraction.  nblocks blocks of 256
 * threads, each running 8 independent FMA chains for iters x 16 steps, as
 * scalar FFMA (packed = 0) or packed FFMA2 (packed = 1).
 *   out    dev float [nblocks * 256] (output; values of no interest)
 *   flops  host double* or NULL: receives the launch's FP32 flops (FMA = 2)
 * Errors: ME_EINVAL for nblocks or iters < 1 or a NULL out.
 */
int me_fp32_peak(int packed, int nblocks, int iters, float *out, double *flops, void *stream);

/* ----------------------------------------------------------------- serving
 * A continuous-batching request loop for inversions of slit scans and map
 * tiles of uneven pixel counts (the paper's goal of near real-time pipeline
 * inversions, Section 7).  serve_submit copies a request and queues it; a
 * worker thread admits queued requests in arrival order whenever one of
 * max_inflight slots is free and the request's buffers fit the arena
 * (admission by memory), then runs the GA (and optional L-M polish) of
 * ga_invert_batch / lm_polish on a stream of its own, so admitted requests
 * overlap on the device.  Results are bit-identical to calling
 * ga_invert_batch + lm_polish on the same request alone.
 *
 * The handle owns one device arena and one pinned host arena of arena_bytes
 * each (the only allocations in this library), plus 2 * max_inflight streams.
 */
typedef struct serve_handle serve_handle;

typedef struct serve_config {
    size_t arena_bytes;       /* device and pinned-host arena size (>= 4096)        */
    int max_inflight;         /* requests on the device at once, 1..64              */
    int max_queue;            /* queued requests before serve_submit -> ME_EAGAIN    */
    int small_pixels;         /* npix <= small_pixels run on high-priority streams   */
    int fail_next_admissions; /* fault injection: the next N admissions fail with
                                 ME_ENOMEM (0 in normal use)                         */
} serve_config;

/* A request.  Host arrays are copied by serve_submit (the caller may reuse
 * them on return).  obs: [npix][4][n_lambda] of the problem dtype; w: GA
 * weights [npix][4] (ga.weight_mode == ME_W_USER) or NULL; mu_px: [npix] or
 * NULL; polish_w: L-M weights [npix][4] or NULL (then w, or inverse-max). */
typedef struct serve_request {
    const void *obs;
    const double *w;
    const double *mu_px;
    int npix;
    uint64_t pixel_id0;
    ga_config ga;
    me_bounds bounds;
    int polish_iters;
    double lambda0;
    const double *polish_w;
} serve_request;

/* Completed request: best [npix][M] and chi2 [npix] are caller-owned
 * host buffers (either may be NULL); status is the request's own status;
 * queue_ns = submit -> admission, latency_ns = submit -> results on the host. */
typedef struct serve_result {
    double *best;
    double *chi2;
    int status;
    uint64_t queue_ns;
    uint64_t latency_ns;
} serve_result;

typedef struct serve_stats_t {
    int queued;
    int running;
    size_t arena_used;
    size_t arena_bytes;
} serve_stats_t;

/* Create a serving loop for one problem on the current device.  ME_ENOMEM if
 * an arena cannot be allocated. */
int serve_create(const me_problem *pb, const serve_config *cfg, serve_handle **out);
/* Queue a request; ME_EAGAIN when max_queue requests are waiting, ME_EINVAL
 * for an invalid request or one larger than the arena.  *ticket identifies it. */
int serve_submit(serve_handle *h, const serve_request *rq, uint64_t *ticket);
/* Collect a request: timeout_ms = 0 returns ME_EPENDING at once if it is not
 * done, > 0 waits up to that long (then ME_ETIMEOUT), < 0 waits until done.
 * On completion fills *out and forgets the ticket (ME_ENOTFOUND afterwards);
 * returns the request's status. */
int serve_poll(serve_handle *h, uint64_t ticket, serve_result *out, int timeout_ms);
int serve_stats(serve_handle *h, serve_stats_t *out);
/* Cancel queued requests, wait for running ones, free everything. */
int serve_destroy(serve_handle *h);

/*
 * lm_uncertainty - Section 6 uncertainty estimate at given parameters:
 * sigma_i^2 = [H^-1]_ii chi2 / M (M parameters) with H the Hessian of Eq. chisq
 * in its Gauss-Newton form H = (2/nu) J^T W^2 J (exact where the residuals
 * vanish); J analytic in the problem precision, H and its inverse in FP64.
 *   params  dev double [npix][M] (e.g. the output of lm_polish)
 *   w       dev double [npix][4] or NULL (inverse-max weights)
 *   sigma   dev double [npix][M] (output); +infinity where H is singular
 */
int lm_uncertainty(const me_problem *pb, const void *obs, const double *w, const double *mu_px,
                   int npix, const double *params, double *sigma, void *stream);

/*
 * me_line_centre - Section 5.1 line-centre estimate by centre of symmetry:
 * S_i = sum_{j=1..W} |I(lambda_{i+j}) - I(lambda_{i-j})|, lambda_sym = the
 * lambda_i minimising S over candidates i in [i_lo, i_hi] intersected with
 * [W, n_lambda-1-W] (ties: lowest index), refined by the vertex of the
 * parabola through (lambda, S) at i-1, i, i+1 when both are candidates.  All
 * in FP64.
 *   obs        dev [npix][4][n_lambda] of pb->dtype (the Stokes I rows are used)
 *   half_width W >= 1 grid points
 *   lambda_c   dev double [npix] (output; NaN if no candidate)
 *   index      dev int [npix] (output, argmin index or -1; may be NULL)
 */
int me_line_centre(const me_problem *pb, const void *obs, int npix, int half_width, int i_lo,
                   int i_hi, double *lambda_c, int *index, void *stream);

/* ------------------------------------------ pixel selection and seeding
 * me_classify - Section 2 pixel selection with the weak-field fallback, and
 * the Section 5.5 seeds and polarity, one pixel per warp in FP64.
 *   Threshold: I_c = mean of I over the quiet window [q_lo, q_hi); sigma_s^2
 *   the variance (1/n) of s = Q, U, V there; p = sqrt(Qmax^2 + Umax^2 +
 *   Vmax^2) / I_c with X_max = max |X| over the grid; sigma_P = p_thresh
 *   sqrt(sigma_Q^2 + sigma_U^2 + sigma_V^2) / I_c; flag = (p > sigma_P).
 *   Weak field for line `line` in the window [c_lo, c_hi] (inclusive), kz =
 *   4.6686e-13 g lambda0^2: B_par = (lambda(I+V core) - lambda(I-V core)) /
 *   (2 kz), each core the argmin refined by the three-point parabola vertex;
 *   chi = atan2(-sum U I'', -sum Q I'') / 2 in [0, 180) and B_perp =
 *   sqrt(4 sqrt((sum Q I'')^2 + (sum U I'')^2) / sum I''^2) / kz, the least-
 *   squares fit of (Q, U) = -(kz^2 B_perp^2 / 4)(cos 2chi, sin 2chi) I'' with
 *   I'' the three-point second difference; theta = atan2(B_perp, B_par).
 *   Polarity: +1 when the positive V lobe lies blueward of the negative one,
 *   -1 when redward, 0 when they coincide.
 *   Seeds (B, psi, chi) rows: weak field; integral (B_par = s int|V| /
 *   (kz TV(I)), B_perp = sqrt(4 int L / TV(I')) / kz); centre of gravity of
 *   I_c - (I +- V) for B_par (Rees & Semel 1979); non-magnetic (B = 0).
 *   psi is reflected (180 - psi) into the polarity's half.
 * Sums run in increasing index, so all outputs but the angles are
 * bit-identical to a plain sequential FP64 evaluation.  obs must be finite.
 *   obs       dev [npix][4][n_lambda] of pb->dtype
 *   flag      dev int [npix] (output; may be NULL)
 *   polarity  dev int [npix] (output; may be NULL)
 *   pol       dev double [npix][2] = (p, sigma_P) (output; may be NULL)
 *   weak      dev double [npix][5] = (B, theta, chi, B_par, B_perp) (may be NULL)
 *   seeds     dev double [npix][4][3] (output; may be NULL)
 *   best      dev double [npix][M] or NULL: rows of pixels below the
 *             threshold receive (B, theta, chi, NaN ...); others are untouched
 * Errors: ME_EINVAL for windows outside the grid or line out of range.
 */
int me_classify(const me_problem *pb, const void *obs, int npix, double p_thresh, int q_lo,
                int q_hi, int line, int c_lo, int c_hi, int *flag, int *polarity, double *pol,
                double *weak, double *seeds, double *best, void *stream);

/*
 * me_select - the pixels i (increasing) with flag[i] == want: index dev int
 * [npix] receives them and count dev int [1] their number, both written on
 * the stream (no host synchronisation).  scratch is caller-owned device
 * memory of at least me_select_scratch_bytes(npix) bytes, 4-byte aligned, not
 * shared with a concurrent call.  Selection precedes Algorithm 1 in Section 2:
 * only the pixels above the polarization threshold are inverted.
 */
size_t me_select_scratch_bytes(int npix);
int me_select(const int *flag, int npix, int want, int *index, int *count, void *scratch,
              size_t scratch_bytes, void *stream);

/*
 * me_select_static - me_select without caller scratch and without any
 * allocation: its tile counts live in a file-scope device array of the
 * library, sized for npix <= ME_SELECT_STATIC_MAX_PIX (32 KiB), whose address
 * is looked up once per device at set-up.  The paper has no counterpart; this
 * is a deployment convenience for callers that must not allocate.  npix above
 * the limit -> ME_EINVAL.  Every call on a device shares that array, so calls
 * that overlap in time (other streams or threads) race and must be serialised
 * by the caller; calls in order on one stream are safe.  Results equal
 * me_select's.
 */
#define ME_SELECT_STATIC_MAX_PIX (1 << 24)
int me_select_static(const int *flag, int npix, int want, int *index, int *count, void *stream);

/*
 * ga_invert_subset - ga_invert_batch on a subset of a map, with the Section
 * 5.5 seeds and polarity restriction.  Block b inverts pixel index[b] for
 * b < *count (index and count on the device, e.g. from me_select; index NULL
 * = identity, count NULL = npix); every per-pixel array (obs, w, mu_px,
 * seeds, polarity, best, chi2, best_genes) is indexed by that pixel number,
 * and the random streams by pixel_id0 + pixel number, so a pixel's result is
 * the one a whole-map run gives it.  Out-of-range indices are skipped.
 *   seeds     dev double [npix][nseed][3] of (B, psi, chi); NaN keeps the Sobol
 *             gene.  They replace those genes of the last nseed <= npop/2
 *             individuals of P0, encoded to the nearest gene.
 *   polarity  dev int [npix] or NULL: +1 restricts the inclination domain to
 *             [lo, min(hi, 90)], -1 to [max(lo, 90), hi] (0, or an empty half:
 *             unrestricted); the decode of that gene uses it throughout.
 *   bounds_px dev double [npix][2][M] or NULL: per-pixel search domain
 *             (lo row, hi row; Section 5.3, e.g. from me_prefit_bounds) in
 *             place of *bounds for the decode and the seed encoding; the
 *             polarity restriction applies on top of it.
 */
int ga_invert_subset(const me_problem *pb, const void *obs, const double *w, const double *mu_px,
                     int npix, uint64_t pixel_id0, const me_bounds *bounds, const ga_config *cfg,
                     const double *seeds, int nseed, const int *polarity, const double *bounds_px,
                     const int *index, const int *count, double *best, double *chi2,
                     uint16_t *best_genes, void *stream);

/*
 * lm_fit - lm_polish with a parameter mask, on the subset index[0 .. *count)
 * of a map (as ga_invert_subset; NULL index and count = all npix pixels).
 * Parameters whose bit in free_mask is clear are held: their rows and
 * columns of the normal equations are zeroed, so their step is exactly 0.
 * With B, theta, chi held at B = 0 and weights (w_I, 0, 0, 0) this is the
 * Section 5.3 thermodynamic prefit: a non-magnetic fit of Stokes I.
 */
int lm_fit(const me_problem *pb, const void *obs, const double *w, const double *mu_px, int npix,
           const me_bounds *bounds, int iters, double lambda0, unsigned free_mask, const int *index,
           const int *count, double *params_inout, double *chi2_out, void *stream);

/*
 * me_prefit_bounds - Section 5.3: the prefit's values constrain the GA's
 * search to ranges around them.  For pixel i and parameter k:
 *   lo'_ik = max(lo_k, p_hat_ik - lower[k]), hi'_ik = min(hi_k, p_hat_ik + upper[k]),
 * an infinite margin keeping the global bound; where that leaves no interval
 * (or p_hat_ik is NaN) the global [lo_k, hi_k] stays.
 *   p_hat      dev double [npix][M] (e.g. lm_fit's prefit), M = npar (ME_NPAR or
 *              ME_NPAR_MAX)
 *   lower, upper  host double [M] margins (not NaN)
 *   bounds_px  dev double [npix][2][M] (output: lo' row, then hi' row),
 *              the input of ga_invert_subset
 */
int me_prefit_bounds(const double *p_hat, int npix, int npar, const me_bounds *bounds, const double *lower,
                     const double *upper, double *bounds_px, void *stream);

/* ------------------------------------------------ GA operator entry points
 * The operators of ga_invert_batch run alone on caller-given populations, so
 * that they can be checked bit for bit against a reference with injected
 * fitness values.  nprob independent populations of npop individuals of
 * npar (ME_NPAR or ME_NPAR_MAX) genes; the crossover string has 16 npar bits.
 *
 * ga_breed - one generation of selection, crossover, mutation and elitism
 * (Algorithm 1 Select/Recombine/Mutate) at generation `gen` for pixel ids
 * pixel_id0 + p.
 *   genes    dev uint16 [nprob][npop][npar]
 *   fitness  dev double [nprob][npop] (NaN counts as +infinity)
 *   child    dev uint16 [nprob][npop][npar] (output)
 *   elite    dev int [nprob] (output, may be NULL)
 */
int ga_breed(const uint16_t *genes, const double *fitness, int nprob, int npop, int npar,
             uint64_t pixel_id0, int gen, const ga_config *cfg, uint16_t *child,
             int *elite, void *stream);

/*
 * ga_restart - Section 5.6 restart: the worst npop/2 individuals (stable rank by
 * fitness, then index) take Sobol points sobol_next + r in rank order r.
 *   genes  dev uint16 [nprob][npop][npar], modified in place
 */
int ga_restart(uint16_t *genes, const double *fitness, int nprob, int npop, int npar,
               uint64_t sobol_next, void *stream);

/* Philox4x32-10 of n counters: ctr dev uint32 [n][4], key {lo, hi}, out dev
 * uint32 [n][4]. */
int me_philox(const uint32_t *ctr, int n, uint64_t key, uint32_t *out, void *stream);

/* Sobol points first..first+n-1 of dimensions 0..ndim-1 (ndim <= ME_NPAR_MAX)
 * as 32-bit integers: out dev uint32 [n][ndim]. */
int me_sobol(uint64_t first, int n, int ndim, uint32_t *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GENESIS_H */
