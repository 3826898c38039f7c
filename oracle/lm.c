/*
 * Oracle: finite-difference Jacobian, Levenberg-Marquardt polish and the
 * threaded batch synthesis.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * L-M (Levenberg 1944, Marquardt 1963, cited in Section 1): minimise the
 * chi2 of Eq. chisq from a starting vector.  Each iteration solves
 *     (A + lambda D) delta = g,  A = J^T W^2 J,  g = J^T W^2 (O - M),
 * D = diag(max(A_jj, 1e-12 max_k A_kk)) (Marquardt's diagonal scaling with a
 * floor so that a parameter without influence keeps a non-singular system),
 * by Cholesky factorisation; a failed factorisation multiplies lambda by 10
 * and retries.  The trial vector p + delta has its azimuth wrapped into
 * [0, 180) and is then clamped to the bounds; it is accepted if its chi2 is
 * lower (lambda /= 10), otherwise rejected (lambda *= 10).  A fixed number of
 * trial steps is taken.  Parameters outside free_mask (bit k = parameter k)
 * are held: their Jacobian columns are zero, so A and g have zero rows and
 * columns there and delta_k = 0 (Section 5.3's prefit fits Stokes I with the
 * field held at B = 0).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* typical magnitude of each parameter, used to size finite-difference steps */
static const double fd_scale[OR_MAXPAR] = {100.0, 1.0, 1.0, 0.1, 1.0, 0.01, 0.1, 0.01, 0.01, 0.01};

/*
 * d stokes / d p_k by central differences D(h) = (f(p + h) - f(p - h)) / 2h,
 * Richardson-extrapolated: (4 D(h/2) - D(h)) / 3, error O(h^4).
 * h_k = 1e-3 max(|p_k|, scale_k).
 */
void or_jacobian(const or_problem *pb, const double *p, double mu, double *jac)
{
    const int nl = pb->n_lambda, ns = 4 * nl, M = or_npar(pb);
    double *fp = (double *)malloc(sizeof(double) * ns);
    double *fm = (double *)malloc(sizeof(double) * ns);
    double *d1 = (double *)malloc(sizeof(double) * ns);
    for (int k = 0; k < M; ++k) {
        const double h = 1e-3 * (fabs(p[k]) > fd_scale[k] ? fabs(p[k]) : fd_scale[k]);
        double q[OR_MAXPAR];
        for (int pass = 0; pass < 2; ++pass) {
            const double hh = pass == 0 ? h : 0.5 * h;
            memcpy(q, p, sizeof(double) * M);
            q[k] = p[k] + hh;
            or_synth(pb, q, mu, fp);
            q[k] = p[k] - hh;
            or_synth(pb, q, mu, fm);
            for (int i = 0; i < ns; ++i) {
                const double d = (fp[i] - fm[i]) / (2.0 * hh);
                if (pass == 0) d1[i] = d;
                else jac[(size_t)i * M + k] = (4.0 * d - d1[i]) / 3.0;
            }
        }
    }
    free(fp); free(fm); free(d1);
}

/* Solve (N) x = b in place for symmetric positive definite N (n x n, row
 * major).  Returns 0 if a pivot is not positive. */
static int cholesky_solve(int n, double *N, double *b)
{
    for (int j = 0; j < n; ++j) {
        double d = N[j * n + j];
        for (int k = 0; k < j; ++k) d -= N[j * n + k] * N[j * n + k];
        if (!(d > 0.0)) return 0;
        const double ljj = sqrt(d);
        N[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = N[i * n + j];
            for (int k = 0; k < j; ++k) s -= N[i * n + k] * N[j * n + k];
            N[i * n + j] = s / ljj;
        }
    }
    for (int i = 0; i < n; ++i) { /* L y = b */
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= N[i * n + k] * b[k];
        b[i] = s / N[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) { /* L^T x = y */
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= N[k * n + i] * b[k];
        b[i] = s / N[i * n + i];
    }
    return 1;
}

static double wrap_azimuth(double chi)
{
    double c = fmod(chi, 180.0);
    if (c < 0.0) c += 180.0;
    if (c >= 180.0) c -= 180.0;
    return c;
}

static void lm_pixel(const or_problem *pb, const double *obs, const double *w,
                     double mu, const double *lo, const double *hi, int iters,
                     double lambda0, unsigned free_mask, double *p, double *chi2_out)
{
    const int nl = pb->n_lambda, ns = 4 * nl, M = or_npar(pb);
    double *model = (double *)malloc(sizeof(double) * ns);
    double *jac = (double *)malloc(sizeof(double) * ns * M);
    double A[OR_MAXPAR * OR_MAXPAR], g[OR_MAXPAR];
    or_synth(pb, p, mu, model);
    double chi2 = or_chi2(obs, model, w, nl, M);
    double lam = lambda0;
    int need_jac = 1;
    for (int it = 0; it < iters; ++it) {
        if (need_jac) {
            or_jacobian(pb, p, mu, jac);
            for (int i = 0; i < ns; ++i)
                for (int a = 0; a < M; ++a)
                    if (!((free_mask >> a) & 1u)) jac[(size_t)i * M + a] = 0.0;
            memset(A, 0, sizeof A);
            memset(g, 0, sizeof g);
            for (int i = 0; i < ns; ++i) {
                const double ws = w[i / nl] * w[i / nl];
                const double r = obs[i] - model[i];
                for (int a = 0; a < M; ++a) {
                    g[a] += ws * jac[(size_t)i * M + a] * r;
                    for (int b = 0; b < M; ++b)
                        A[a * M + b] += ws * jac[(size_t)i * M + a] * jac[(size_t)i * M + b];
                }
            }
            need_jac = 0;
        }
        double dmax = 0.0;
        for (int a = 0; a < M; ++a) if (A[a * M + a] > dmax) dmax = A[a * M + a];
        if (!(dmax > 0.0)) break;
        double delta[OR_MAXPAR];
        int ok = 0;
        for (int tries = 0; tries < 30 && !ok; ++tries) {
            double N[OR_MAXPAR * OR_MAXPAR];
            memcpy(N, A, sizeof(double) * M * M);
            for (int a = 0; a < M; ++a) {
                const double d = A[a * M + a] > 1e-12 * dmax ? A[a * M + a] : 1e-12 * dmax;
                N[a * M + a] += lam * d;
            }
            memcpy(delta, g, sizeof(double) * M);
            ok = cholesky_solve(M, N, delta);
            if (!ok) lam *= 10.0;
        }
        if (!ok) break;
        double q[OR_MAXPAR];
        for (int a = 0; a < M; ++a) q[a] = p[a] + delta[a];
        q[2] = wrap_azimuth(q[2]);
        for (int a = 0; a < M; ++a) {
            if (q[a] < lo[a]) q[a] = lo[a];
            if (q[a] > hi[a]) q[a] = hi[a];
        }
        double *mtrial = (double *)malloc(sizeof(double) * ns);
        or_synth(pb, q, mu, mtrial);
        const double c2 = or_chi2(obs, mtrial, w, nl, M);
        if (c2 < chi2) {
            memcpy(p, q, sizeof(double) * M);
            memcpy(model, mtrial, sizeof(double) * ns);
            chi2 = c2;
            lam /= 10.0;
            need_jac = 1;
        } else {
            lam *= 10.0;
        }
        free(mtrial);
    }
    *chi2_out = chi2;
    free(model); free(jac);
}

/*
 * Section 6: sigma_i^2 = [H^-1]_ii chi2 / M at p, with H = (2/nu) J^T W^2 J the
 * Gauss-Newton Hessian of Eq. chisq (J by central differences), inverted by
 * Gauss-Jordan elimination with partial pivoting; +infinity if singular.
 */
static void sigma_pixel(const or_problem *pb, const double *obs, const double *w, double mu,
                        const double *p, double *sigma)
{
    const int nl = pb->n_lambda, ns = 4 * nl, M = or_npar(pb);
    double *model = (double *)malloc(sizeof(double) * ns);
    double *jac = (double *)malloc(sizeof(double) * ns * M);
    or_synth(pb, p, mu, model);
    const double chi2 = or_chi2(obs, model, w, nl, M);
    or_jacobian(pb, p, mu, jac);
    const double nu = (double)(4 * nl - M);
    double H[OR_MAXPAR][2 * OR_MAXPAR];
    memset(H, 0, sizeof H);
    for (int i = 0; i < ns; ++i) {
        const double ws = w[i / nl] * w[i / nl];
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b)
                H[a][b] += 2.0 / nu * ws * jac[(size_t)i * M + a] * jac[(size_t)i * M + b];
    }
    for (int a = 0; a < M; ++a) H[a][M + a] = 1.0;
    int ok = 1;
    for (int c = 0; c < M && ok; ++c) {
        int piv = c;
        for (int r = c + 1; r < M; ++r) if (fabs(H[r][c]) > fabs(H[piv][c])) piv = r;
        if (!(fabs(H[piv][c]) > 0.0)) { ok = 0; break; }
        if (piv != c)
            for (int k = 0; k < 2 * M; ++k) { double t = H[c][k]; H[c][k] = H[piv][k]; H[piv][k] = t; }
        const double d = H[c][c];
        for (int k = 0; k < 2 * M; ++k) H[c][k] /= d;
        for (int r = 0; r < M; ++r) {
            if (r == c) continue;
            const double f = H[r][c];
            for (int k = 0; k < 2 * M; ++k) H[r][k] -= f * H[c][k];
        }
    }
    for (int a = 0; a < M; ++a) {
        const double v = ok ? H[a][M + a] * chi2 / (double)M : INFINITY;
        sigma[a] = ok && v >= 0.0 ? sqrt(v) : INFINITY;
    }
    free(model); free(jac);
}

void or_lm_uncertainty(const or_problem *pb, const double *obs, const double *w, const double *mu_px,
                       double mu, int npix, const double *params, double *sigma)
{
    const int nl = pb->n_lambda;
    for (int ip = 0; ip < npix; ++ip) {
        const double *o = obs + (size_t)ip * 4 * nl;
        double wv[4];
        if (w) memcpy(wv, w + (size_t)ip * 4, sizeof wv);
        else or_weights_invmax(o, nl, wv);
        const int M = or_npar(pb);
        sigma_pixel(pb, o, wv, mu_px ? mu_px[ip] : mu, params + (size_t)ip * M, sigma + (size_t)ip * M);
    }
}

typedef struct {
    const or_problem *pb;
    const double *obs, *w, *mu_px;
    double mu;
    const double *lo, *hi;
    int iters;
    double lambda0;
    unsigned free_mask;
    double *params, *chi2;
    const double *sparams;
    double *stokes;
    int t0, t1;
} lm_job;

static void *lm_worker(void *arg)
{
    const lm_job *J = (const lm_job *)arg;
    const int nl = J->pb->n_lambda;
    for (int ip = J->t0; ip < J->t1; ++ip) {
        const double *obs = J->obs + (size_t)ip * 4 * nl;
        double w[4];
        if (J->w) memcpy(w, J->w + (size_t)ip * 4, sizeof w);
        else or_weights_invmax(obs, nl, w);
        const double mu = J->mu_px ? J->mu_px[ip] : J->mu;
        lm_pixel(J->pb, obs, w, mu, J->lo, J->hi, J->iters, J->lambda0, J->free_mask,
                 J->params + (size_t)ip * or_npar(J->pb), J->chi2 + ip);
    }
    return NULL;
}

static void *synth_worker(void *arg)
{
    const lm_job *J = (const lm_job *)arg;
    const int nl = J->pb->n_lambda;
    for (int ip = J->t0; ip < J->t1; ++ip) {
        const double mu = J->mu_px ? J->mu_px[ip] : J->mu;
        or_synth(J->pb, J->sparams + (size_t)ip * or_npar(J->pb), mu, J->stokes + (size_t)ip * 4 * nl);
    }
    return NULL;
}

static void run_threads(lm_job *base, int n, int nthreads, void *(*fn)(void *))
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = n > 0 ? n : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    lm_job *jobs = (lm_job *)malloc(sizeof(lm_job) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *base;
        jobs[t].t0 = (int)((long)n * t / nthreads);
        jobs[t].t1 = (int)((long)n * (t + 1) / nthreads);
        pthread_create(&th[t], NULL, fn, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs);
}

int or_lm_polish(const or_problem *pb, const double *obs, const double *w,
                 const double *mu_px, double mu, int npix, const double *lo,
                 const double *hi, int iters, double lambda0, unsigned free_mask,
                 double *params_inout, double *chi2_out, int nthreads)
{
    if (npix < 0 || iters < 0) return 1;
    lm_job base;
    memset(&base, 0, sizeof base);
    base.pb = pb; base.obs = obs; base.w = w; base.mu_px = mu_px; base.mu = mu;
    base.lo = lo; base.hi = hi; base.iters = iters; base.lambda0 = lambda0;
    base.free_mask = free_mask;
    base.params = params_inout; base.chi2 = chi2_out;
    run_threads(&base, npix, nthreads, lm_worker);
    return 0;
}

void or_synth_batch(const or_problem *pb, const double *params, int n,
                    const double *mu_px, double mu, double *stokes, int nthreads)
{
    lm_job base;
    memset(&base, 0, sizeof base);
    base.pb = pb; base.mu_px = mu_px; base.mu = mu;
    base.sparams = params; base.stokes = stokes;
    run_threads(&base, n, nthreads, synth_worker);
}
