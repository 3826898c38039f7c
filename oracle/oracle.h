/*
 * Plain FP64 CPU oracle for the GENESIS Milne-Eddington genetic-algorithm
 * inversion (Harker & Mighell 2012).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path: every routine here
 * is written from the paper's equations (and, where the paper is silent, from
 * the readings listed in the design notes) in the order the paper states them,
 * with no blocking or fusion.
 *
 * Built with -O2 -ffp-contract=off: every a*b+c is rounded twice, so the
 * results are the same on x86-64 and aarch64 hosts.
 *
 * Parameter vector (M = 9, or 10 with the fill fraction), fixed order:
 *   0 B [G], 1 theta [deg], 2 chi [deg], 3 v_LOS [km/s], 4 Doppler width
 *   [mA] (quoted at lambda_dop), 5 damping a, 6 eta0, 7 S0, 8 S1, and with
 *   fill != 0: 9 alpha, the magnetic fill fraction of Section 5.2.
 *
 * Pins (tests/test_oracle_*.py): the Faddeeva routine against brute-force
 * quadrature, the a->0 closed forms and scipy.special.wofz; the closed-form ME
 * solution against a direct 4x4 solve; physics invariants (B=0, theta=0/90,
 * azimuth flips, weak-field limit); Philox against triton's independent
 * implementation; Sobol dimensions 0-1 against scipy, the (0,m,1)-net
 * property of every dimension, and each dimension's direction numbers against
 * the recurrence of its primitive polynomial (the primitive polynomials over
 * GF(2) in degree-then-encoding order, checked by their order); the GA
 * operators on hand-built bit patterns and a brute-force search; the L-M
 * polish on noiseless truth.
 */
#ifndef GENESIS_ORACLE_H
#define GENESIS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_LINES 4
#define OR_NPAR 9
#define OR_MAXPAR 10   /* with the fill fraction alpha */
#define OR_MAX_COMP 9   /* Zeeman components per group (J <= 4) */

typedef struct {
    int n_lines;
    double lambda0[OR_MAX_LINES];   /* rest wavelength [A] (Table 1) */
    double g[OR_MAX_LINES];         /* effective Lande factor (Table 1) */
    double eta_ratio[OR_MAX_LINES]; /* eta0 of this line / eta0 parameter */
    int pattern[OR_MAX_LINES];      /* 0: effective triplet with g; 1: full pattern */
    int j_lower[OR_MAX_LINES], j_upper[OR_MAX_LINES];
    double g_lower[OR_MAX_LINES], g_upper[OR_MAX_LINES];
    double lambda_dop;              /* [A] wavelength at which param 4 is quoted */
    int n_lambda;
    const double *lambda;           /* [n_lambda] observed wavelengths [A] */
    int fill;                       /* 1: the fill fraction alpha is parameter 9 */
} or_problem;

/* Number of model parameters M of a problem: 9, or 10 with alpha. */
static inline int or_npar(const or_problem *pb) { return OR_NPAR + (pb->fill ? 1 : 0); }

typedef struct {
    int npop, ngen, nsamp;          /* nsamp <= 0: no restarts */
    double pc;                      /* crossover probability */
    double pmut_lsb, pmut_ratio;    /* per-bit mutation: pmut_lsb * ratio^(15-b) */
    uint64_t seed;
} or_ga_config;

/* Wigner 3j symbol for integer arguments (Racah's formula). */
double or_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3);
/* Zeeman components of lower (J_l, g_l) -> upper (J_u, g_u): per group
 * (0 = sigma_blue, q = -1; 1 = pi; 2 = sigma_red, q = +1) the number of
 * components, their shifts in Larmor units (g_l M_l - g_u M_u) and strengths
 * 3 (J_u J_l 1; M_u -M_l q)^2.  Returns non-zero for an invalid transition. */
int or_zeeman_components(int j_lower, double g_lower, int j_upper, double g_upper,
                         int n[3], double shift[3][OR_MAX_COMP], double strength[3][OR_MAX_COMP]);

/* Faddeeva function w(x + i y), y >= 0 (Matta & Reichel 1971 trapezoid). */
void or_faddeeva(double x, double y, double *re, double *im);
void or_faddeeva_batch(int n, const double *x, const double *y, double *re, double *im);

/* Unno-Rachkovsky Stokes vector [4][n_lambda] (I, Q, U, V), closed form. */
void or_synth(const or_problem *pb, const double *p, double mu, double *stokes);
/* Same, but every wavelength solves K x = e by Gaussian elimination. */
void or_synth_lu(const or_problem *pb, const double *p, double mu, double *stokes);
/* Batch of n models, threaded over models. mu_px may be NULL (then mu). */
void or_synth_batch(const or_problem *pb, const double *params, int n,
                    const double *mu_px, double mu, double *stokes, int nthreads);

/* Inverse-max weights w[4] of one observed pixel [4][n_lambda]. */
void or_weights_invmax(const double *obs, int n_lambda, double *w);
/* chi-square of Eq. chisq, nu = 4 n_lambda - m. */
double or_chi2(const double *obs, const double *model, const double *w,
               int n_lambda, int m);

/* Philox4x32-10 (Salmon et al. 2011). */
void or_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Sobol point n (Gray-code order, point 0 = origin), dimension dim, 32 bits. */
uint32_t or_sobol_u32(uint64_t n, int dim);
/* Direction numbers V[0..31] of dimension dim (for inspection). */
void or_sobol_directions(int dim, uint32_t v[32]);

/* Eq. decode of m uint16 genes into parameters within [lo, hi]. */
void or_ga_decode(const uint16_t *g, const double *lo, const double *hi, int m, double *p);

/* One generation of the GA operators (select, crossover, mutate, elitism) on a
 * given population genes[npop][m] with fitness f[npop]; writes child genes.
 * Returns the elite index. */
int or_ga_breed(const uint16_t *genes, const double *f, int npop, int m,
                uint64_t pixel_id, int gen, const or_ga_config *cfg,
                uint16_t *child);

/* Restart step: ranks f (stable) and overwrites the worst npop/2 individuals
 * with Sobol points sobol_next, sobol_next+1, ... in rank order. Writes the
 * replaced slot indices to replaced[npop/2] (may be NULL). */
void or_ga_restart(uint16_t *genes, const double *f, int npop, int m,
                   uint64_t sobol_next, int *replaced);

/* Full GA inversion of npix pixels (Algorithm 1 with the readings above).
 * obs [npix][4][n_lambda]; w [npix][4] or NULL (inverse-max); mu_px [npix]
 * or NULL (mu); lo/hi [m] bounds. Outputs best [npix][m], chi2 [npix] (FP64
 * re-evaluation with the fitness weights), best_genes [npix][m] (may be NULL)
 * and margin [npix] (may be NULL): the smallest relative gap between two
 * unequal fitness values whose order decided a selection, elitism or restart
 * step.  Section 5.5: seeds [npix][nseed][3] (B, psi, chi; NaN keeps the
 * Sobol gene) replace those genes of the last nseed <= npop/2 individuals of
 * P0; polarity [npix] (may be NULL) restricts the inclination domain per
 * pixel (or_polarity_bounds).  bounds_px [npix][2][m] (may be NULL) replaces
 * lo/hi per pixel (Section 5.3), the polarity applying on top. */
uint16_t or_ga_encode(double x, double lo, double hi);
void or_polarity_bounds(int pol, double lo, double hi, double *plo, double *phi);
int or_ga_invert(const or_problem *pb, const double *obs, const double *w,
                 const double *mu_px, double mu, int npix, uint64_t pixel_id0,
                 const double *lo, const double *hi, const or_ga_config *cfg,
                 const double *seeds, int nseed, const int *polarity,
                 const double *bounds_px, double *best, double *chi2, uint16_t *best_genes,
                 double *margin, int nthreads);

/* Jacobian d stokes / d p, [4*n_lambda][M], by central differences
 * with Richardson extrapolation. */
void or_jacobian(const or_problem *pb, const double *p, double mu, double *jac);

/* Levenberg-Marquardt polish of npix pixels (Marquardt damping). params_inout
 * [npix][M]; chi2_out [npix]; parameters outside free_mask are held. */
int or_lm_polish(const or_problem *pb, const double *obs, const double *w,
                 const double *mu_px, double mu, int npix, const double *lo,
                 const double *hi, int iters, double lambda0, unsigned free_mask,
                 double *params_inout, double *chi2_out, int nthreads);

/* Section 5.3 bounds from a thermodynamic prefit p_hat [npix][m]:
 * lo'_k = max(lo_k, p_hat_k - lower_k), hi'_k = min(hi_k, p_hat_k + upper_k)
 * (an infinite margin keeps the global bound); where that leaves no interval
 * (or p_hat_k is NaN) the global bounds stay.  out [npix][2][m]. */
void or_prefit_bounds(const double *p_hat, int npix, int m, const double *lo, const double *hi,
                      const double *lower, const double *upper, double *out);

/* Section 5.1 line centre by centre of symmetry (see me.c). */
void or_line_centre(const double *rows, int npix, int stride, int nl, const double *lam, int half_width,
                    int i_lo, int i_hi, double *lam_c, int *idx);

/* Section 2 pixel selection and weak-field fallback (see me.c). */
void or_classify(const or_problem *pb, const double *obs, int npix, double p_thresh, int q_lo, int q_hi,
                 int line, int c_lo, int c_hi, int *flag, int *polarity, double *out_pol, double *out_weak,
                 double *seeds);

/* Section 6 uncertainties sigma [npix][M] at params. */
void or_lm_uncertainty(const or_problem *pb, const double *obs, const double *w, const double *mu_px,
                       double mu, int npix, const double *params, double *sigma);

#ifdef __cplusplus
}
#endif
#endif
