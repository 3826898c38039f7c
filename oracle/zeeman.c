/*
 * Oracle: Zeeman components of a transition (the "full Zeeman pattern" the
 * paper computes at start-up, Section 5).  TEST INFRASTRUCTURE ONLY (see
 * oracle.h).
 *
 * A transition lower (J_l, g_l) -> upper (J_u, g_u) splits into components
 * M_u -> M_l with q = M_l - M_u in {-1, 0, +1}.  Component shift in units of
 * the Larmor displacement dlambda_L = 4.6686e-13 lambda0^2 B (positive = to
 * longer wavelength): s = g_l M_l - g_u M_u.  Relative strength (normalised to
 * 1 within each q): S = 3 (J_u J_l 1; M_u -M_l q)^2, a Wigner 3j symbol, here
 * evaluated with Racah's closed formula (the 3j sum rule makes each group's
 * strengths add up to 1; the pins check that).  q = -1 is the sigma_blue group, 0 the
 * pi group and +1 the sigma_red group (for a normal triplet J_u = 1 -> J_l = 0
 * this gives s = -g, 0, +g).
 */
#include <math.h>
#include <stdlib.h>

#include "oracle.h"

static double fact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* Wigner 3j symbol for integer arguments (Racah's formula). */
double or_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3)
{
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
    const double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) /
                       fact(j1 + j2 + j3 + 1);
    const double pre = sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                            fact(j3 + m3) * fact(j3 - m3));
    double sum = 0.0;
    for (int k = 0; k <= j1 + j2 + j3; ++k) {
        const int a = j3 - j2 + k + m1, b = j3 - j1 + k - m2, c = j1 + j2 - j3 - k;
        const int d = j1 - k - m1, e = j2 - k + m2;
        if (a < 0 || b < 0 || c < 0 || d < 0 || e < 0) continue;
        const double t = 1.0 / (fact(k) * fact(a) * fact(b) * fact(c) * fact(d) * fact(e));
        sum += (k % 2 ? -t : t);
    }
    const int ph = j1 - j2 - m3;
    return ((ph % 2 + 2) % 2 ? -1.0 : 1.0) * pre * sum;
}

int or_zeeman_components(int j_lower, double g_lower, int j_upper, double g_upper,
                         int n[3], double shift[3][OR_MAX_COMP], double strength[3][OR_MAX_COMP])
{
    if (j_lower < 0 || j_upper < 0 || abs(j_lower - j_upper) > 1 || (j_lower == 0 && j_upper == 0))
        return 1;
    for (int q = -1; q <= 1; ++q) {
        const int gi = q + 1;
        n[gi] = 0;
        for (int mu = -j_upper; mu <= j_upper; ++mu) {
            const int ml = mu + q;
            if (ml < -j_lower || ml > j_lower) continue;
            const double w3 = or_wigner3j(j_upper, j_lower, 1, mu, -ml, q);
            const double s = 3.0 * w3 * w3;
            if (s <= 0.0) continue;
            if (n[gi] >= OR_MAX_COMP) return 2;
            shift[gi][n[gi]] = g_lower * ml - g_upper * mu;
            strength[gi][n[gi]] = s;
            ++n[gi];
        }
    }
    return 0;
}
