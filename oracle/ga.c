/*
 * Oracle: the genetic algorithm of Section 3 (Algorithm 1) applied per pixel,
 * with the operators fixed as follows (the paper names them but does not give
 * their exact form):
 *   encode/decode  uint16 word per parameter (Section 3.2), p = u + (v-u) g/65535
 *   selection S    binary tournament, two distinct entrants, ties to the
 *                  lower index (a "sampling without replacement" biased
 *                  toward better fitness)
 *   recombination  one-point crossover of the MSB-first 16M-bit string of a
 *                  pair (2q, 2q+1) with probability pc
 *   mutation M     bit b (0 = MSB) of every word flips on its own with
 *                  probability q_b = pmut_lsb * ratio^(15-b): less-significant
 *                  bits mutate more
 *   elitism        child slot 0 takes the best parent unchanged
 *   restart        every nsamp generations (t < ngen) the worst half is
 *                  replaced by the next Sobol points (Section 5.6)
 * Random numbers: Philox4x32-10, key = (seed lo, seed hi), counter =
 * (pixel id lo, pixel id hi, generation, index << 8 | purpose).  Purpose 0:
 * words 0, 1 drive the tournament of child slot index, and for an even index
 * words 2, 3 drive the crossover of the pair (index, index + 1).  Purposes
 * 2, 3, ...: the child slot's mutation draws, four per block, used in order.
 * The mutation places the flips of each word by jumps: with bits 0..b of the
 * word still open (b = 15, the LSB, first), a draw u at or above
 * A(b, 0) = floor(2^32 P(a flip among bits 0..b)) leaves them unflipped;
 * otherwise the next flip is bit c, the largest c <= b with u < A(b, c) =
 * floor(2^32 (1 - prod_{d=c..b} (1 - q_d))), and bits 0..c-1 remain open.
 * Each bit thus flips independently with probability q_b (up to the 2^-32
 * rounding of the thresholds), at about 1 + sum_b q_b draws per word.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static inline double clean(double f) { return (f == f) ? f : INFINITY; }

static inline void philox_at(uint64_t seed, uint64_t pid, int gen, uint32_t idx,
                             uint32_t purpose, uint32_t out[4])
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)gen,
                             (idx << 8) | purpose};
    or_philox4x32(ctr, key, out);
}

/* floor(p * 2^32) as a threshold compared against a uniform u32; p >= 1
 * gives 2^32 (always true), p <= 0 gives 0 (never). */
static uint64_t prob_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 1ull << 32;
    return (uint64_t)floor(p * 4294967296.0);
}

/* A[b][c] for c <= b: floor(2^32 (1 - prod_{d=c..b} (1 - q_d))), the chance
 * that a flip falls among bits c..b, with q_d = pmut_lsb ratio^(15-d) clamped
 * to [0, 1] (ratio^k by repeated multiplication, the product taken from d = b
 * down to c). */
static void mutation_table(const or_ga_config *cfg, uint64_t A[16][16])
{
    double q[16];
    for (int d = 0; d < 16; ++d) {
        double r = 1.0;
        for (int k = 0; k < 15 - d; ++k) r *= cfg->pmut_ratio;
        const double p = cfg->pmut_lsb * r;
        q[d] = p > 0.0 ? (p < 1.0 ? p : 1.0) : 0.0;
    }
    for (int b = 0; b < 16; ++b) {
        double none = 1.0;
        for (int c = b; c >= 0; --c) {
            none *= 1.0 - q[c];
            A[b][c] = prob_threshold(1.0 - none);
        }
    }
}

static int argmin_f(const double *f, int n)
{
    int e = 0;
    for (int i = 1; i < n; ++i)
        if (clean(f[i]) < clean(f[e])) e = i;
    return e;
}

int or_ga_breed(const uint16_t *genes, const double *f, int npop, int m,
                uint64_t pid, int gen, const or_ga_config *cfg, uint16_t *child)
{
    const int e = argmin_f(f, npop);
    /* S: one binary tournament per child slot */
    for (int k = 0; k < npop; ++k) {
        uint32_t u[4];
        philox_at(cfg->seed, pid, gen, (uint32_t)k, 0u, u);
        const int i = (int)(((uint64_t)u[0] * (uint64_t)npop) >> 32);
        const int j = (int)((i + 1 + (int)(((uint64_t)u[1] * (uint64_t)(npop - 1)) >> 32)) % npop);
        const double fi = clean(f[i]), fj = clean(f[j]);
        const int win = (fj < fi || (fj == fi && j < i)) ? j : i;
        memcpy(child + (size_t)k * m, genes + (size_t)win * m, sizeof(uint16_t) * m);
    }
    /* R: one-point crossover of each pair, from words 2, 3 of the even slot's block */
    const uint64_t tc = prob_threshold(cfg->pc);
    const int nbits = 16 * m;
    for (int q = 0; q < npop / 2; ++q) {
        uint32_t u[4];
        philox_at(cfg->seed, pid, gen, (uint32_t)(2 * q), 0u, u);
        if ((uint64_t)u[2] >= tc) continue;
        const int c = 1 + (int)(((uint64_t)u[3] * (uint64_t)(nbits - 1)) >> 32);
        uint16_t *a = child + (size_t)(2 * q) * m;
        uint16_t *b = child + (size_t)(2 * q + 1) * m;
        /* bits [c, nbits) of the MSB-first string change owners */
        for (int bit = c; bit < nbits; ++bit) {
            const int w = bit / 16;
            const uint16_t mask = (uint16_t)(1u << (15 - bit % 16));
            const uint16_t ta = a[w] & mask, tb = b[w] & mask;
            a[w] = (uint16_t)((a[w] & ~mask) | tb);
            b[w] = (uint16_t)((b[w] & ~mask) | ta);
        }
    }
    /* M: per-bit mutation placed by jumps between flips (see above) */
    uint64_t A[16][16];
    mutation_table(cfg, A);
    for (int k = 0; k < npop; ++k) {
        uint16_t *g = child + (size_t)k * m;
        uint32_t u[4];
        int used = 4;
        uint32_t block = 0;
        for (int w = 0; w < m; ++w) {
            int b = 15;
            while (b >= 0) {
                if (used == 4) {
                    philox_at(cfg->seed, pid, gen, (uint32_t)k, 2u + block, u);
                    ++block;
                    used = 0;
                }
                const uint64_t draw = u[used++];
                if (draw >= A[b][0]) break;
                int c = b;
                while (!(draw < A[b][c])) --c;
                g[w] ^= (uint16_t)(1u << (15 - c));
                b = c - 1;
            }
        }
    }
    /* elitism: slot 0 keeps the best parent */
    memcpy(child, genes + (size_t)e * m, sizeof(uint16_t) * m);
    return e;
}

/* stable rank of individual i: how many precede it in (fitness, index) order */
static int stable_rank(const double *f, int n, int i)
{
    int r = 0;
    const double fi = clean(f[i]);
    for (int j = 0; j < n; ++j) {
        const double fj = clean(f[j]);
        if (fj < fi || (fj == fi && j < i)) ++r;
    }
    return r;
}

void or_ga_restart(uint16_t *genes, const double *f, int npop, int m,
                   uint64_t sobol_next, int *replaced)
{
    const int half = npop / 2;
    int *rank = (int *)malloc(sizeof(int) * npop);
    for (int i = 0; i < npop; ++i) rank[i] = stable_rank(f, npop, i);
    for (int i = 0; i < npop; ++i) {
        if (rank[i] < half) continue;
        const uint64_t n = sobol_next + (uint64_t)(rank[i] - half);
        for (int d = 0; d < m; ++d) genes[(size_t)i * m + d] = (uint16_t)(or_sobol_u32(n, d) >> 16);
        if (replaced) replaced[rank[i] - half] = i;
    }
    free(rank);
}

/* Eq. decode: p_j = u_j + (v_j - u_j) / (2^N - 1) * (integer value of the
 * N = 16 bit word, bit 0 = MSB). */
static void decode(const uint16_t *g, const double *lo, const double *hi, int m,
                   double *p)
{
    for (int j = 0; j < m; ++j) p[j] = lo[j] + (hi[j] - lo[j]) * ((double)g[j] / 65535.0);
}

void or_ga_decode(const uint16_t *g, const double *lo, const double *hi, int m, double *p)
{
    decode(g, lo, hi, m, p);
}

/* The inverse of the decode for a seed value, rounded to the nearest gene:
 * t = (x - u) / (v - u) clamped to [0, 1], g = floor(t (2^N - 1) + 1/2). */
uint16_t or_ga_encode(double x, double lo, double hi)
{
    double t = (x - lo) / (hi - lo);
    if (!(t > 0.0)) t = 0.0;
    if (t > 1.0) t = 1.0;
    return (uint16_t)floor(t * 65535.0 + 0.5);
}

/* Section 5.5 polarity restriction of the inclination domain: +1 keeps
 * [u, min(v, 90)], -1 keeps [max(u, 90), v], 0 (or an empty half) keeps [u, v]. */
void or_polarity_bounds(int pol, double lo, double hi, double *plo, double *phi)
{
    double a = lo, b = hi;
    if (pol > 0 && hi > 90.0) b = 90.0;
    if (pol < 0 && lo < 90.0) a = 90.0;
    if (!(a < b)) { a = lo; b = hi; }
    *plo = a;
    *phi = b;
}

/* ---------------------------------------------------------------- margins */

static inline double rel_gap(double a, double b)
{
    const double s = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    return s > 0.0 ? fabs(a - b) / s : 0.0;
}

static inline void note_pair(double *margin, const double *f, const uint16_t *genes,
                             int m, int i, int j)
{
    const double fi = clean(f[i]), fj = clean(f[j]);
    if (isinf(fi) && isinf(fj)) return;
    if (fi == fj) {
        if (memcmp(genes + (size_t)i * m, genes + (size_t)j * m, sizeof(uint16_t) * m) == 0)
            return; /* identical genotypes tie on any evaluator */
        *margin = 0.0;
        return;
    }
    const double g = rel_gap(fi, fj);
    if (g < *margin) *margin = g;
}

/* every comparison the breeding step's decisions depend on */
static void breed_margin(double *margin, const uint16_t *genes, const double *f,
                         int npop, int m, uint64_t pid, int gen, uint64_t seed)
{
    const int e = argmin_f(f, npop);
    for (int i = 0; i < npop; ++i)
        if (i != e) note_pair(margin, f, genes, m, i, e);
    for (int k = 0; k < npop; ++k) {
        uint32_t u[4];
        philox_at(seed, pid, gen, (uint32_t)k, 0u, u);
        const int i = (int)(((uint64_t)u[0] * (uint64_t)npop) >> 32);
        const int j = (int)((i + 1 + (int)(((uint64_t)u[1] * (uint64_t)(npop - 1)) >> 32)) % npop);
        note_pair(margin, f, genes, m, i, j);
    }
}

static void restart_margin(double *margin, const uint16_t *genes, const double *f,
                           int npop, int m)
{
    for (int i = 0; i < npop; ++i)
        for (int j = i + 1; j < npop; ++j) note_pair(margin, f, genes, m, i, j);
}

/* ---------------------------------------------------------------- driver */

typedef struct {
    const or_problem *pb;
    const double *obs, *w, *mu_px;
    double mu;
    int npix;
    uint64_t pid0;
    const double *glo, *ghi;
    const or_ga_config *cfg;
    const double *seeds;
    int nseed;
    const int *polarity;
    const double *bounds_px;
    double *best, *chi2, *margin;
    uint16_t *best_genes;
    int t0, t1;
} ga_job;

static double fitness(const or_problem *pb, const double *obs, const double *w,
                      double mu, const uint16_t *g, const double *lo,
                      const double *hi, double *model)
{
    double p[OR_MAXPAR];
    decode(g, lo, hi, or_npar(pb), p);
    or_synth(pb, p, mu, model);
    return clean(or_chi2(obs, model, w, pb->n_lambda, or_npar(pb)));
}

static void ga_pixel(const ga_job *J, int ip)
{
    const or_problem *pb = J->pb;
    const int nl = pb->n_lambda, npop = J->cfg->npop, m = or_npar(pb);
    const double *obs = J->obs + (size_t)ip * 4 * nl;
    const double mu = J->mu_px ? J->mu_px[ip] : J->mu;
    const uint64_t pid = J->pid0 + (uint64_t)ip;
    double lo[OR_MAXPAR], hi[OR_MAXPAR];
    if (J->bounds_px) {
        memcpy(lo, J->bounds_px + (size_t)ip * 2 * m, sizeof(double) * m);
        memcpy(hi, J->bounds_px + (size_t)ip * 2 * m + m, sizeof(double) * m);
    } else {
        memcpy(lo, J->glo, sizeof(double) * m);
        memcpy(hi, J->ghi, sizeof(double) * m);
    }
    if (J->polarity) or_polarity_bounds(J->polarity[ip], lo[1], hi[1], &lo[1], &hi[1]);
    double w[4];
    if (J->w) memcpy(w, J->w + (size_t)ip * 4, sizeof w);
    else or_weights_invmax(obs, nl, w);

    uint16_t *genes = (uint16_t *)malloc(sizeof(uint16_t) * npop * m);
    uint16_t *child = (uint16_t *)malloc(sizeof(uint16_t) * npop * m);
    double *f = (double *)malloc(sizeof(double) * npop);
    double *model = (double *)malloc(sizeof(double) * 4 * nl);
    int *replaced = (int *)malloc(sizeof(int) * npop);
    double margin = INFINITY;

    /* create P0 from Sobol points 1..npop, the last nseed individuals taking
     * the seeds' (B, psi, chi) genes (Section 5.5), and evaluate F0 */
    for (int k = 0; k < npop; ++k) {
        for (int d = 0; d < m; ++d)
            genes[(size_t)k * m + d] = (uint16_t)(or_sobol_u32((uint64_t)(k + 1), d) >> 16);
        const int si = k - (npop - J->nseed);
        if (si >= 0) {
            const double *sd = J->seeds + ((size_t)ip * J->nseed + si) * 3;
            for (int d = 0; d < 3; ++d)
                if (sd[d] == sd[d]) genes[(size_t)k * m + d] = or_ga_encode(sd[d], lo[d], hi[d]);
        }
        f[k] = fitness(pb, obs, w, mu, genes + (size_t)k * m, lo, hi, model);
    }
    uint64_t sobol_next = (uint64_t)npop + 1;
    const int ngen = J->cfg->ngen, nsamp = J->cfg->nsamp;
    for (int t = 1; t <= ngen; ++t) {
        if (J->margin) breed_margin(&margin, genes, f, npop, m, pid, t, J->cfg->seed);
        const int e = or_ga_breed(genes, f, npop, m, pid, t, J->cfg, child);
        const double fe = f[e];
        uint16_t *tmp = genes; genes = child; child = tmp;
        f[0] = fe;
        for (int k = 1; k < npop; ++k)
            f[k] = fitness(pb, obs, w, mu, genes + (size_t)k * m, lo, hi, model);
        if (nsamp > 0 && t % nsamp == 0 && t < ngen) {
            if (J->margin) restart_margin(&margin, genes, f, npop, m);
            or_ga_restart(genes, f, npop, m, sobol_next, replaced);
            for (int r = 0; r < npop / 2; ++r) {
                const int k = replaced[r];
                f[k] = fitness(pb, obs, w, mu, genes + (size_t)k * m, lo, hi, model);
            }
            sobol_next += (uint64_t)(npop / 2);
        }
    }
    if (J->margin) {
        /* the final argmin is a decision too */
        const int b = argmin_f(f, npop);
        for (int i = 0; i < npop; ++i)
            if (i != b) note_pair(&margin, f, genes, m, i, b);
        J->margin[ip] = margin;
    }
    const int b = argmin_f(f, npop);
    double *best = J->best + (size_t)ip * m;
    decode(genes + (size_t)b * m, lo, hi, m, best);
    or_synth(pb, best, mu, model);
    J->chi2[ip] = or_chi2(obs, model, w, nl, m);
    if (J->best_genes) memcpy(J->best_genes + (size_t)ip * m, genes + (size_t)b * m, sizeof(uint16_t) * m);
    free(genes); free(child); free(f); free(model); free(replaced);
}

static void *ga_worker(void *arg)
{
    const ga_job *J = (const ga_job *)arg;
    for (int ip = J->t0; ip < J->t1; ++ip) ga_pixel(J, ip);
    return NULL;
}

int or_ga_invert(const or_problem *pb, const double *obs, const double *w,
                 const double *mu_px, double mu, int npix, uint64_t pid0,
                 const double *lo, const double *hi, const or_ga_config *cfg,
                 const double *seeds, int nseed, const int *polarity,
                 const double *bounds_px, double *best, double *chi2, uint16_t *best_genes,
                 double *margin, int nthreads)
{
    if (cfg->npop < 2 || (cfg->npop & 1) || cfg->ngen < 0 || npix < 0) return 1;
    if (nseed < 0 || nseed > cfg->npop / 2 || (nseed > 0 && !seeds)) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > npix) nthreads = npix > 0 ? npix : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    ga_job *jobs = (ga_job *)malloc(sizeof(ga_job) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        ga_job J = {pb, obs, w, mu_px, mu, npix, pid0, lo, hi, cfg, seeds, nseed, polarity,
                    bounds_px, best, chi2, margin, best_genes, (int)((long)npix * t / nthreads),
                    (int)((long)npix * (t + 1) / nthreads)};
        jobs[t] = J;
        pthread_create(&th[t], NULL, ga_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs);
    return 0;
}

void or_prefit_bounds(const double *p_hat, int npix, int m, const double *lo, const double *hi,
                      const double *lower, const double *upper, double *out)
{
    for (int ip = 0; ip < npix; ++ip) {
        const double *p = p_hat + (size_t)ip * m;
        double *ol = out + (size_t)ip * 2 * m, *oh = ol + m;
        for (int k = 0; k < m; ++k) {
            double a = p[k] - lower[k], b = p[k] + upper[k];
            if (!(a > lo[k])) a = lo[k];
            if (!(b < hi[k])) b = hi[k];
            if (!(a < b)) { a = lo[k]; b = hi[k]; }
            ol[k] = a;
            oh[k] = b;
        }
    }
}
