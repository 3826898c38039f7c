/*
 * Oracle: Faddeeva function, Unno-Rachkovsky synthesis, weights and chi2.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_C_KMS 299792.458   /* speed of light [km/s] */
#define OR_ZEEMAN 4.6686e-13  /* e/(4 pi m c^2) in A^-1 G^-1 (textbook value) */

/*
 * Faddeeva function w(z) = exp(-z^2) erfc(-i z), z = x + i y.
 *
 * The paper evaluates the Voigt and Faraday-Voigt profiles H and F with a
 * rational approximation (Section 5, Hui et al. 1978).  The oracle uses a
 * different, published method so that it shares nothing with the GPU path:
 * the trapezoidal rule with pole correction of Matta & Reichel (1971,
 * Math. Comp. 25, 339) applied to
 *     w(z) = (i z / pi) * Integral exp(-t^2) / (z^2 - t^2) dt,   Im z > 0,
 * with step h = 0.5 on nodes t = k h, or on the shifted nodes t = (k+1/2) h
 * when x lies within h/4 of an unshifted node (this keeps every denominator
 * at least h/4 away from zero).  The poles at t = +-z add
 *     2 exp(-z^2) / (1 -+ exp(-2 pi i z / h))    for Im z < pi / h.
 * The discretisation error is of order exp(-pi^2/h^2) ~ 5e-18; 16 nodes per
 * side leave a truncation of exp(-64).  For y < 0 the reflection
 * w(z) = 2 exp(-z^2) - w(-z) is used (w is entire).
 */
static double complex faddeeva_upper(double x, double y)
{
    const double h = 0.5;
    const int nk = 16;
    const double complex z = x + I * y;
    const double complex z2 = z * z;
    const double q = x / h;
    const int shifted = fabs(q - nearbyint(q)) < 0.25;
    double complex s = 0.0;
    for (int k = 0; k <= nk; ++k) {
        double t, wt;
        if (shifted) {
            t = (k + 0.5) * h;
            wt = 1.0;
        } else {
            t = k * h;
            wt = (k == 0) ? 0.5 : 1.0;
        }
        s += wt * exp(-t * t) / (z2 - t * t);
    }
    double complex val = (2.0 * I * h / M_PI) * z * s;
    if (y < M_PI / h) {
        double complex e = cexp(-2.0 * I * M_PI * z / h);
        double complex den = shifted ? (1.0 + e) : (1.0 - e);
        val += 2.0 * cexp(-z2) / den;
    }
    return val;
}

void or_faddeeva(double x, double y, double *re, double *im)
{
    double complex w;
    if (y >= 0.0) {
        w = faddeeva_upper(x, y);
    } else {
        double complex z = x + I * y;
        w = 2.0 * cexp(-z * z) - faddeeva_upper(-x, -y);
    }
    *re = creal(w);
    *im = cimag(w);
}

/*
 * Propagation-matrix elements at one wavelength (Section 5: K = 1 + eta0 Phi).
 * The paper defers the elements of Phi to Landi Degl'Innocenti & Landolfi;
 * with the effective-triplet Zeeman pattern they are, per line l with
 * eta0_l = eta0 * r_l and phi + i psi = w(z):
 *   eta_I = 1 + sum eta0_l/2 [phi_p sin^2 t + (phi_b + phi_r)/2 (1 + cos^2 t)]
 *   eta_Q =     sum eta0_l/2 [phi_p - (phi_b + phi_r)/2] sin^2 t cos 2chi
 *   eta_U =     sum eta0_l/2 [phi_p - (phi_b + phi_r)/2] sin^2 t sin 2chi
 *   eta_V =     sum eta0_l/2 (phi_r - phi_b) cos t
 * and rho_Q, rho_U, rho_V the same with psi.  b, p, r are the sigma_blue,
 * pi and sigma_red components centred at v + v_B, v and v - v_B.
 */
static void kmatrix(const or_problem *pb, const double *p, double lam,
                    double e[7])
{
    const double deg = M_PI / 180.0;
    const double B = p[0], th = p[1] * deg, ch = p[2] * deg, vlos = p[3];
    const double dld_mA = p[4], a = p[5], eta0 = p[6];
    const double st = sin(th), ct = cos(th);
    const double s2 = st * st, c2 = ct * ct;
    const double c2x = cos(2.0 * ch), s2x = sin(2.0 * ch);
    double etaI = 1.0, etaQ = 0.0, etaU = 0.0, etaV = 0.0;
    double rhoQ = 0.0, rhoU = 0.0, rhoV = 0.0;
    for (int l = 0; l < pb->n_lines; ++l) {
        const double l0 = pb->lambda0[l];
        /* lambda - lambda_c with lambda_c = lambda0 (1 + v_LOS / c), written as
         * (lambda - lambda0) - lambda0 v_LOS / c: the first difference is exact
         * (Sterbenz), so v keeps full relative precision near the line core */
        const double dl = (lam - l0) - l0 * vlos / OR_C_KMS;
        const double dD = dld_mA * 1e-3 * l0 / pb->lambda_dop;
        const double v = dl / dD;
        const double vB = OR_ZEEMAN * pb->g[l] * l0 * l0 * B / dD;
        double phb, psb, php, psp, phr, psr;
        if (pb->pattern[l]) {
            /* full Zeeman pattern: each group is the strength-weighted sum of
             * its components, centred at v - v_L s with v_L the Larmor
             * splitting in Doppler units */
            int n[3];
            double sh[3][OR_MAX_COMP], st[3][OR_MAX_COMP];
            or_zeeman_components(pb->j_lower[l], pb->g_lower[l], pb->j_upper[l], pb->g_upper[l],
                                 n, sh, st);
            const double vL = OR_ZEEMAN * l0 * l0 * B / dD;
            double ph[3] = {0, 0, 0}, ps[3] = {0, 0, 0};
            for (int g = 0; g < 3; ++g)
                for (int i = 0; i < n[g]; ++i) {
                    double re, im;
                    or_faddeeva(v - vL * sh[g][i], a, &re, &im);
                    ph[g] += st[g][i] * re;
                    ps[g] += st[g][i] * im;
                }
            phb = ph[0]; psb = ps[0]; php = ph[1]; psp = ps[1]; phr = ph[2]; psr = ps[2];
        } else {
            or_faddeeva(v + vB, a, &phb, &psb);
            or_faddeeva(v, a, &php, &psp);
            or_faddeeva(v - vB, a, &phr, &psr);
        }
        const double h = 0.5 * eta0 * pb->eta_ratio[l];
        etaI += h * (php * s2 + 0.5 * (phb + phr) * (1.0 + c2));
        etaQ += h * (php - 0.5 * (phb + phr)) * s2 * c2x;
        etaU += h * (php - 0.5 * (phb + phr)) * s2 * s2x;
        etaV += h * (phr - phb) * ct;
        rhoQ += h * (psp - 0.5 * (psb + psr)) * s2 * c2x;
        rhoU += h * (psp - 0.5 * (psb + psr)) * s2 * s2x;
        rhoV += h * (psr - psb) * ct;
    }
    e[0] = etaI; e[1] = etaQ; e[2] = etaU; e[3] = etaV;
    e[4] = rhoQ; e[5] = rhoU; e[6] = rhoV;
}

/*
 * Milne-Eddington solution (Section 5): with S = S0 + S1 tau the emergent
 * Stokes vector is S0 e + mu S1 K^-1 e, e = (1,0,0,0); I_c = S0 + mu S1.
 * K^-1 e written out (Landi Degl'Innocenti closed form):
 *   Delta = eI^2 (eI^2 - eQ^2 - eU^2 - eV^2 + rQ^2 + rU^2 + rV^2) - Pi^2,
 *   Pi = eQ rQ + eU rU + eV rV,
 *   I = eI (eI^2 + rQ^2 + rU^2 + rV^2) / Delta,
 *   Q = -[eI^2 eQ + eI (eV rU - eU rV) + rQ Pi] / Delta, U, V cyclic.
 */
/*
 * Section 5.2 fill fraction: I <- alpha I_mag + (1 - alpha) I_nm e.  The
 * field-free part is read as the same Milne-Eddington atmosphere without a
 * field (the paper's quiet-sun CLV profile is not printed):
 *   I_nm = S0 + mu S1 / (1 + sum_l eta0_l Re w(v_l, a)),
 * v_l the unshifted profile argument of line l.
 */
static double nonmagnetic_I(const or_problem *pb, const double *p, double mu, double lam)
{
    const double vlos = p[3], dld_mA = p[4], a = p[5], eta0 = p[6];
    double eta = 1.0;
    for (int l = 0; l < pb->n_lines; ++l) {
        const double l0 = pb->lambda0[l];
        const double dl = (lam - l0) - l0 * vlos / OR_C_KMS;
        const double dD = dld_mA * 1e-3 * l0 / pb->lambda_dop;
        double re, im;
        or_faddeeva(dl / dD, a, &re, &im);
        eta += eta0 * pb->eta_ratio[l] * re;
    }
    return p[7] + mu * p[8] / eta;
}

static void apply_fill(const or_problem *pb, const double *p, double mu, double *stokes)
{
    if (!pb->fill) return;
    const int nl = pb->n_lambda;
    const double alpha = p[9];
    for (int j = 0; j < nl; ++j) {
        stokes[0 * nl + j] = alpha * stokes[0 * nl + j] + (1.0 - alpha) * nonmagnetic_I(pb, p, mu, pb->lambda[j]);
        stokes[1 * nl + j] = alpha * stokes[1 * nl + j];
        stokes[2 * nl + j] = alpha * stokes[2 * nl + j];
        stokes[3 * nl + j] = alpha * stokes[3 * nl + j];
    }
}

void or_synth(const or_problem *pb, const double *p, double mu, double *stokes)
{
    const int nl = pb->n_lambda;
    const double S0 = p[7], S1 = p[8];
    for (int j = 0; j < nl; ++j) {
        double e[7];
        kmatrix(pb, p, pb->lambda[j], e);
        const double eI = e[0], eQ = e[1], eU = e[2], eV = e[3];
        const double rQ = e[4], rU = e[5], rV = e[6];
        const double Pi = eQ * rQ + eU * rU + eV * rV;
        const double eI2 = eI * eI;
        const double Delta =
            eI2 * (eI2 - eQ * eQ - eU * eU - eV * eV + rQ * rQ + rU * rU + rV * rV)
            - Pi * Pi;
        const double f = mu * S1 / Delta;
        stokes[0 * nl + j] = S0 + f * eI * (eI2 + rQ * rQ + rU * rU + rV * rV);
        stokes[1 * nl + j] = -f * (eI2 * eQ + eI * (eV * rU - eU * rV) + rQ * Pi);
        stokes[2 * nl + j] = -f * (eI2 * eU + eI * (eQ * rV - eV * rQ) + rU * Pi);
        stokes[3 * nl + j] = -f * (eI2 * eV + eI * (eU * rQ - eQ * rU) + rV * Pi);
    }
    apply_fill(pb, p, mu, stokes);
}

/* Same Stokes vector, solving K x = e directly (Gaussian elimination with
 * partial pivoting) at every wavelength. */
void or_synth_lu(const or_problem *pb, const double *p, double mu, double *stokes)
{
    const int nl = pb->n_lambda;
    const double S0 = p[7], S1 = p[8];
    for (int j = 0; j < nl; ++j) {
        double e[7];
        kmatrix(pb, p, pb->lambda[j], e);
        const double eI = e[0], eQ = e[1], eU = e[2], eV = e[3];
        const double rQ = e[4], rU = e[5], rV = e[6];
        double K[4][5] = {
            {eI, eQ, eU, eV, 1.0},
            {eQ, eI, rV, -rU, 0.0},
            {eU, -rV, eI, rQ, 0.0},
            {eV, rU, -rQ, eI, 0.0},
        };
        for (int c = 0; c < 4; ++c) {
            int piv = c;
            for (int r = c + 1; r < 4; ++r)
                if (fabs(K[r][c]) > fabs(K[piv][c])) piv = r;
            if (piv != c)
                for (int k = 0; k < 5; ++k) {
                    double t = K[c][k]; K[c][k] = K[piv][k]; K[piv][k] = t;
                }
            for (int r = c + 1; r < 4; ++r) {
                double m = K[r][c] / K[c][c];
                for (int k = c; k < 5; ++k) K[r][k] -= m * K[c][k];
            }
        }
        double x[4];
        for (int r = 3; r >= 0; --r) {
            double s = K[r][4];
            for (int k = r + 1; k < 4; ++k) s -= K[r][k] * x[k];
            x[r] = s / K[r][r];
        }
        stokes[0 * nl + j] = S0 + mu * S1 * x[0];
        for (int s = 1; s < 4; ++s) stokes[s * nl + j] = mu * S1 * x[s];
    }
    apply_fill(pb, p, mu, stokes);
}

/*
 * Inverse-max weights (Section 5.4): w_I = 1/(I_c - I_0), w_Q = 1/max|Q|,
 * w_U = 1/max|U|, w_V = 1/max|V|.  I_c is read as the largest observed I in
 * the window and I_0 as the smallest (the line core).  Each denominator is
 * floored at 1e-6 |I_c| so that a profile that is identically zero gives a
 * large finite weight; a zero denominator (all-zero input) gives w = 0.
 */
void or_weights_invmax(const double *obs, int nl, double *w)
{
    double imax = obs[0], imin = obs[0];
    for (int j = 1; j < nl; ++j) {
        if (obs[j] > imax) imax = obs[j];
        if (obs[j] < imin) imin = obs[j];
    }
    double d[4];
    d[0] = imax - imin;
    for (int s = 1; s < 4; ++s) {
        double m = 0.0;
        for (int j = 0; j < nl; ++j) {
            double a = fabs(obs[s * nl + j]);
            if (a > m) m = a;
        }
        d[s] = m;
    }
    const double fl = 1e-6 * fabs(imax);
    for (int s = 0; s < 4; ++s) {
        double dd = d[s] > fl ? d[s] : fl;
        w[s] = dd > 0.0 ? 1.0 / dd : 0.0;
    }
}

/* Eq. chisq: chi2 = (1/nu) sum_s w_s^2 sum_j (O_sj - M_sj)^2, nu = 4 N - M. */
double or_chi2(const double *obs, const double *model, const double *w,
               int nl, int m)
{
    double tot = 0.0;
    for (int s = 0; s < 4; ++s) {
        double ss = 0.0;
        for (int j = 0; j < nl; ++j) {
            double r = obs[s * nl + j] - model[s * nl + j];
            ss += r * r;
        }
        tot += w[s] * w[s] * ss;
    }
    return tot / (double)(4 * nl - m);
}

/* w(x_i + i y_i) for n points (test convenience). */
void or_faddeeva_batch(int n, const double *x, const double *y, double *re, double *im)
{
    for (int i = 0; i < n; ++i) or_faddeeva(x[i], y[i], re + i, im + i);
}

/*
 * Section 5.1: line centre by centre of symmetry.  For candidate index i,
 * S_i = sum_{j=1..W} |I(lambda_{i+j}) - I(lambda_{i-j})| (W = half_width, in
 * grid points); lambda_sym = argmin_i S_i over i in [i_lo, i_hi] restricted to
 * [W, N-1-W] (ties: lowest index), refined by the vertex of the parabola
 * through (lambda, S) at i-1, i, i+1 when both neighbours are candidates.
 * I rows are read with the given stride (4 n_lambda for a Stokes cube).
 */
static double sym_S(const double *row, int i, int W)
{
    double s = 0.0;
    for (int j = 1; j <= W; ++j) s += fabs(row[i + j] - row[i - j]);
    return s;
}

void or_line_centre(const double *rows, int npix, int stride, int nl, const double *lam, int half_width,
                    int i_lo, int i_hi, double *lam_c, int *idx)
{
    const int W = half_width;
    const int lo = i_lo > W ? i_lo : W;
    const int hi = i_hi < nl - 1 - W ? i_hi : nl - 1 - W;
    for (int ip = 0; ip < npix; ++ip) {
        const double *row = rows + (size_t)ip * stride;
        double best = INFINITY;
        int bi = -1;
        for (int i = lo; i <= hi; ++i) {
            const double s = sym_S(row, i, W);
            if (s < best) { best = s; bi = i; }
        }
        idx[ip] = bi;
        if (bi < 0) { lam_c[ip] = NAN; continue; }
        double xc = lam[bi];
        if (bi - 1 >= lo && bi + 1 <= hi) {
            const double x0 = lam[bi - 1], x1 = lam[bi], x2 = lam[bi + 1];
            const double y0 = sym_S(row, bi - 1, W), y1 = best, y2 = sym_S(row, bi + 1, W);
            const double d0 = x1 - x0, d2 = x1 - x2, e0 = y1 - y0, e2 = y1 - y2;
            const double num = d0 * d0 * e2 - d2 * d2 * e0;
            const double den = d0 * e2 - d2 * e0;
            if (den != 0.0) xc = x1 - 0.5 * num / den;
        }
        lam_c[ip] = xc;
    }
}

/*
 * Section 2 pixel selection, the weak-field fallback and the Section 5.5
 * seeds.  Window sums run in index order; extrema take the lowest index on ties.
 *   Threshold: I_c = mean of I over the quiet window [q_lo, q_hi); sigma_s^2
 *   the (1/n) variance of s = Q, U, V there; p = sqrt(Qmax^2 + Umax^2 +
 *   Vmax^2) / I_c with X_max = max |X| over the whole grid; sigma_P = P_thresh
 *   sqrt(sigma_Q^2 + sigma_U^2 + sigma_V^2) / I_c; flag = p > sigma_P.
 *   Line window [c_lo, c_hi] (inclusive) of line `line` (g, lambda0),
 *   kz = 4.6686e-13 g lambda0^2 (Angstrom per gauss).
 *   Weak field (Auer et al. 1977): the I+V and I-V cores are argmins refined
 *   by the parabola vertex through i-1, i, i+1; B_par = (lambda(I+V) -
 *   lambda(I-V)) / (2 kz).  m = argmax of Q^2 + U^2; chi = atan2(-s U_m,
 *   -s Q_m)/2 in [0, 180) with s = -1 where I''_m < 0 (a sigma lobe: the linear
 *   polarization there has the sign opposite to the line core's), else +1; B_perp = sqrt(4 L_m / D2) / kz with L_m = sqrt(Q_m^2 + U_m^2)
 *   and D2 = max |I''| (three-point second differences); theta = atan2(B_perp,
 *   B_par) in degrees, B = sqrt(B_par^2 + B_perp^2).
 *   Polarity: +1 when the positive V lobe lies blueward of the negative one
 *   (argmax V < argmin V), -1 when redward, 0 when they coincide.
 *   Seeds (B, psi, chi) rows: 0 weak field; 1 integral form of the same
 *   relations, B_par = s int|V| / (kz TV(I)), B_perp = sqrt(4 int L / TV(I')) / kz
 *   (TV = total variation over the window, trapezoid integrals, s the polarity,
 *   +1 when 0); 2 centre of gravity of I_c - (I +- V) (Rees & Semel 1979) for
 *   B_par with the weak-field B_perp; 3 the non-magnetic solution B = 0 with
 *   the weak-field angles.  A seed whose psi lies in the other polarity's half
 *   is reflected, psi -> 180 - psi.
 * out_pol [npix][2] = (p, sigma_P); out_weak [npix][5] = (B, theta, chi,
 * B_par, B_perp); seeds [npix][4][3].
 */
static double vertex3(double x0, double x1, double x2, double y0, double y1, double y2)
{
    const double d0 = x1 - x0, d2 = x1 - x2, e0 = y1 - y0, e2 = y1 - y2;
    const double num = d0 * d0 * e2 - d2 * d2 * e0;
    const double den = d0 * e2 - d2 * e0;
    return den != 0.0 ? x1 - 0.5 * num / den : x1;
}

static double core_of(const double *row, const double *lam, int nl, int lo, int hi)
{
    int bi = lo;
    for (int i = lo + 1; i <= hi; ++i)
        if (row[i] < row[bi]) bi = i;
    if (bi - 1 >= 0 && bi + 1 < nl)
        return vertex3(lam[bi - 1], lam[bi], lam[bi + 1], row[bi - 1], row[bi], row[bi + 1]);
    return lam[bi];
}

static double second_diff(const double *lam, const double *y, int c)
{
    const double h1 = lam[c] - lam[c - 1], h2 = lam[c + 1] - lam[c];
    return 2.0 * (h1 * (y[c + 1] - y[c]) - h2 * (y[c] - y[c - 1])) / (h1 * h2 * (h1 + h2));
}

static double trap_w(const double *lam, int lo, int hi, int j)
{
    if (lo == hi) return 0.0;
    const double a = j > lo ? lam[j] - lam[j - 1] : 0.0;
    const double b = j < hi ? lam[j + 1] - lam[j] : 0.0;
    return 0.5 * (a + b);
}

static void put_seed(double *sd, double bpar, double bperp, double chi, int pol)
{
    double psi = atan2(bperp, bpar) * 180.0 / M_PI;
    if ((pol > 0 && psi > 90.0) || (pol < 0 && psi < 90.0)) psi = 180.0 - psi;
    sd[0] = sqrt(bpar * bpar + bperp * bperp);
    sd[1] = psi;
    sd[2] = chi;
}

void or_classify(const or_problem *pb, const double *obs, int npix, double p_thresh, int q_lo, int q_hi,
                 int line, int c_lo, int c_hi, int *flag, int *polarity, double *out_pol, double *out_weak,
                 double *seeds)
{
    const int nl = pb->n_lambda;
    const double *lam = pb->lambda;
    const double l0 = pb->lambda0[line], g = pb->g[line];
    const double kz = OR_ZEEMAN * g * l0 * l0;
    double *ipv = (double *)malloc(sizeof(double) * nl);
    double *imv = (double *)malloc(sizeof(double) * nl);
    for (int ip = 0; ip < npix; ++ip) {
        const double *sI = obs + (size_t)ip * 4 * nl, *sQ = sI + nl, *sU = sI + 2 * nl, *sV = sI + 3 * nl;
        /* threshold */
        const int nq = q_hi - q_lo;
        double ic = 0.0, mq = 0.0, mu = 0.0, mv = 0.0;
        for (int j = q_lo; j < q_hi; ++j) { ic += sI[j]; mq += sQ[j]; mu += sU[j]; mv += sV[j]; }
        ic /= nq; mq /= nq; mu /= nq; mv /= nq;
        double vq = 0.0, vu = 0.0, vv = 0.0;
        for (int j = q_lo; j < q_hi; ++j) {
            vq += (sQ[j] - mq) * (sQ[j] - mq);
            vu += (sU[j] - mu) * (sU[j] - mu);
            vv += (sV[j] - mv) * (sV[j] - mv);
        }
        vq /= nq; vu /= nq; vv /= nq;
        double qx = 0.0, ux = 0.0, vx = 0.0;
        for (int j = 0; j < nl; ++j) {
            if (fabs(sQ[j]) > qx) qx = fabs(sQ[j]);
            if (fabs(sU[j]) > ux) ux = fabs(sU[j]);
            if (fabs(sV[j]) > vx) vx = fabs(sV[j]);
        }
        const double p = sqrt(qx * qx + ux * ux + vx * vx) / ic;
        const double sp = p_thresh * sqrt(vq + vu + vv) / ic;
        flag[ip] = p > sp ? 1 : 0;
        out_pol[(size_t)ip * 2] = p;
        out_pol[(size_t)ip * 2 + 1] = sp;

        /* polarity from the order of the V lobes */
        int jmax = c_lo, jmin = c_lo;
        for (int j = c_lo + 1; j <= c_hi; ++j) {
            if (sV[j] > sV[jmax]) jmax = j;
            if (sV[j] < sV[jmin]) jmin = j;
        }
        const int pol = jmax < jmin ? 1 : (jmax > jmin ? -1 : 0);
        polarity[ip] = pol;

        /* weak field */
        for (int j = 0; j < nl; ++j) { ipv[j] = sI[j] + sV[j]; imv[j] = sI[j] - sV[j]; }
        const double bpar = (core_of(ipv, lam, nl, c_lo, c_hi) - core_of(imv, lam, nl, c_lo, c_hi)) / (2.0 * kz);
        double qa = 0.0, ub = 0.0, dd = 0.0;
        for (int j = c_lo > 1 ? c_lo : 1; j <= c_hi && j + 1 < nl; ++j) {
            const double d2 = second_diff(lam, sI, j);
            qa += sQ[j] * d2;
            ub += sU[j] * d2;
            dd += d2 * d2;
        }
        double chi = 0.5 * atan2(-ub, -qa) * 180.0 / M_PI;
        if (chi < 0.0) chi += 180.0;
        const double amp = sqrt(qa * qa + ub * ub);
        const double bperp = dd > 0.0 ? sqrt(4.0 * amp / dd) / kz : 0.0;
        double *wo = out_weak + (size_t)ip * 5;
        wo[0] = sqrt(bpar * bpar + bperp * bperp);
        wo[1] = atan2(bperp, bpar) * 180.0 / M_PI;
        wo[2] = chi;
        wo[3] = bpar;
        wo[4] = bperp;

        /* seeds */
        double *sd = seeds + (size_t)ip * 12;
        put_seed(sd, bpar, bperp, chi, pol);
        double av = 0.0, al = 0.0, tvi = 0.0, tvd = 0.0;
        for (int j = c_lo; j <= c_hi; ++j) {
            const double wj = trap_w(lam, c_lo, c_hi, j);
            av += wj * fabs(sV[j]);
            al += wj * sqrt(sQ[j] * sQ[j] + sU[j] * sU[j]);
        }
        for (int j = c_lo; j < c_hi; ++j) tvi += fabs(sI[j + 1] - sI[j]);
        for (int j = c_lo + 1; j < c_hi; ++j) {
            const double sl = (sI[j + 1] - sI[j]) / (lam[j + 1] - lam[j]);
            const double sr = (sI[j] - sI[j - 1]) / (lam[j] - lam[j - 1]);
            tvd += fabs(sl - sr);
        }
        const double bpi = tvi > 0.0 ? (pol < 0 ? -1.0 : 1.0) * av / (kz * tvi) : 0.0;
        const double bti = tvd > 0.0 ? sqrt(4.0 * al / tvd) / kz : 0.0;
        put_seed(sd + 3, bpi, bti, chi, pol);
        double np = 0.0, dp = 0.0, nm = 0.0, dm = 0.0;
        for (int j = c_lo; j <= c_hi; ++j) {
            const double wj = trap_w(lam, c_lo, c_hi, j);
            const double ap = wj * (ic - ipv[j]), am = wj * (ic - imv[j]);
            np += ap * lam[j]; dp += ap;
            nm += am * lam[j]; dm += am;
        }
        const double bcog = (dp != 0.0 && dm != 0.0) ? (np / dp - nm / dm) / (2.0 * kz) : 0.0;
        put_seed(sd + 6, bcog, bperp, chi, pol);
        put_seed(sd + 9, bpar, bperp, chi, pol);
        sd[9] = 0.0;
    }
    free(ipv); free(imv);
}
