// Device-side Milne-Eddington synthesis for sm_103a.
//
// Section 5 of Harker & Mighell (2012): K = 1 + eta0 Phi, the emergent Stokes
// vector S0 e + mu S1 K^-1 e, with Voigt / Faraday-Voigt profiles for the
// sigma_b, pi and sigma_r components of every line.  All templates take the
// arithmetic type R (float or double).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "genesis.h"

namespace genesis {

constexpr double kSpeedOfLight = 299792.458;  // km/s
constexpr double kZeeman = 4.6686e-13;        // A^-1 G^-1 (e / 4 pi m c^2)
constexpr double kDeg = 3.14159265358979323846 / 180.0;

// ------------------------------------------------------------ launch params
struct KLine {
    double lam0;       // rest wavelength [A]
    double lam0_c;     // lambda0 / c [A per km/s]
    double dscale;     // 1e-3 lambda0 / lambda_dop: Doppler width [A] per mA of param 4
    double zfac;       // 4.6686e-13 g_eff lambda0^2 [A / G] (effective triplet)
    double half_eta;   // eta_ratio / 2
    double zfacL;      // 4.6686e-13 lambda0^2 [A / G]: Larmor displacement per gauss
    int ncomp[3];      // full Zeeman pattern: components per group (0 = effective triplet)
    double cshift[3][ME_MAX_COMP];  // component shifts [Larmor units, + = red]
    double cstr[3][ME_MAX_COMP];    // component strengths (sum 1 per group)
    float cshift32[3][ME_MAX_COMP];
    float cstr32[3][ME_MAX_COMP];
    float2 qs2;        // FP32 pair path: half_eta / sqrt(pi) in both lanes
    float2 wq2[17];    // FP32 pair path: Weideman coefficients 2 a_n times half_eta, in both lanes
};

template <class R> __device__ __forceinline__ R comp_shift(const KLine &ln, int g, int i);
template <> __device__ __forceinline__ float comp_shift<float>(const KLine &ln, int g, int i) { return ln.cshift32[g][i]; }
template <> __device__ __forceinline__ double comp_shift<double>(const KLine &ln, int g, int i) { return ln.cshift[g][i]; }
template <class R> __device__ __forceinline__ R comp_str(const KLine &ln, int g, int i);
template <> __device__ __forceinline__ float comp_str<float>(const KLine &ln, int g, int i) { return ln.cstr32[g][i]; }
template <> __device__ __forceinline__ double comp_str<double>(const KLine &ln, int g, int i) { return ln.cstr[g][i]; }

// Everything a synthesis needs, passed by value in the kernel parameters
// (about 6.4 KB, within the 32 KB parameter space of sm_70+).
struct KProblem {
    int n_lines;
    int n_lambda;
    int fill;                   // 1: parameter 9 is the fill fraction alpha
    double mu;
    KLine line[ME_MAX_LINES];
    double lam[ME_MAX_LAMBDA];  // wavelength grid [A]
};

// Weideman coefficient tables (filled per device at library initialisation).
struct FaddeevaTables {
    float w32[17];     // Weideman a_1..a_16 (index n = 1..16), N = 16
    float2 w32x2[17];  // the same doubled (the series' factor 2, exact), in both lanes for packed FP32x2 use
    float L32;
    double w64[37];    // Weideman N = 36
    double L64;
};

// k-th convergent of the Laplace continued fraction of w(z), computed at
// compile time: t_{k+1} = z, t_m = z - (m/2)/t_m+1, w = (i/sqrt(pi))/t_1.
// With t_m = A_m/B_m: A_m = z A_{m+1} - (m/2) B_{m+1}, B_m = A_{m+1}.  For odd
// k, A_1 = a(u) is even and B_1 = z b(u) odd in z (u = z^2), both monic:
// a has degree (k+1)/2, b degree (k-1)/2; coefficients ascend in u.
template <int K> struct CfPoly {
    double a[(K + 1) / 2 + 1];
    double b[(K - 1) / 2 + 1];
    constexpr CfPoly() : a(), b()
    {
        double A[K + 3] = {}, B[K + 3] = {}, An[K + 3] = {};
        A[1] = 1.0;  // z
        B[0] = 1.0;  // 1
        for (int m = K; m >= 1; --m) {
            for (int i = 0; i < K + 3; ++i) An[i] = 0.0;
            for (int i = 0; i + 1 < K + 3; ++i) An[i + 1] += A[i];
            for (int i = 0; i < K + 3; ++i) An[i] -= 0.5 * m * B[i];
            for (int i = 0; i < K + 3; ++i) { B[i] = A[i]; A[i] = An[i]; }
        }
        for (int i = 0; i <= (K + 1) / 2; ++i) a[i] = A[2 * i];
        for (int i = 0; i <= (K - 1) / 2; ++i) b[i] = B[2 * i + 1];
    }
};

// Each translation unit holds its own copy; genesis::upload_tables() fills all.
static __constant__ FaddeevaTables c_fad;

template <class R> struct FadCfg;
template <> struct FadCfg<float> {
    static constexpr int N = 16;        // Weideman terms
    static constexpr int K = 3;         // continued-fraction depth
    static constexpr float R2 = 36.0f;  // |z|^2 above which the continued fraction is used
};
template <> struct FadCfg<double> {
    static constexpr int N = 36;
    static constexpr int K = 9;
    static constexpr double R2 = 64.0;
};


template <class R> struct C2 { R x, y; };

// MUFU reciprocal (relative error < 2^-23), one instruction.
__device__ __forceinline__ float fast_rcp(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double fast_rcp(double v) { return 1.0 / v; }

template <class R> __device__ __forceinline__ R weid(int n);
template <> __device__ __forceinline__ float weid<float>(int n) { return c_fad.w32[n]; }
template <> __device__ __forceinline__ double weid<double>(int n) { return c_fad.w64[n]; }
template <class R> __device__ __forceinline__ R weidL();
template <> __device__ __forceinline__ float weidL<float>() { return c_fad.L32; }
template <> __device__ __forceinline__ double weidL<double>() { return c_fad.L64; }

// Exterior branch: k-th convergent of the Laplace continued fraction,
// w = (i/sqrt(pi)) z b(u) / a(u) with u = z^2 and monic a, b.  a2 = y^2.
template <class R>
__device__ __forceinline__ C2<R> faddeeva_exterior(R x, R y, R a2)
{
    constexpr int NA = (FadCfg<R>::K + 1) / 2, NB = (FadCfg<R>::K - 1) / 2;
    constexpr CfPoly<FadCfg<R>::K> P{};
    const R ux = x * x - a2, uy = R(2) * x * y;
    // monic Horner: start from u + c_{n-1}
    R ax = ux + R(P.a[NA - 1]), ay = uy;
#pragma unroll
    for (int n = NA - 2; n >= 0; --n) {
        const R tx = ax * ux - ay * uy + R(P.a[n]);
        ay = ax * uy + ay * ux;
        ax = tx;
    }
    R bx = R(1), by = R(0);
    if (NB >= 1) {
        bx = ux + R(P.b[NB - 1]);
        by = uy;
    }
#pragma unroll
    for (int n = NB - 2; n >= 0; --n) {
        const R tx = bx * ux - by * uy + R(P.b[n]);
        by = bx * uy + by * ux;
        bx = tx;
    }
    // num = z b(u); w = (i/sqrt(pi)) num / a(u)
    const R nx = x * bx - y * by, ny = x * by + y * bx;
    const R inv = fast_rcp(ax * ax + ay * ay) * R(0.56418958354775628695);  // 1/sqrt(pi)
    C2<R> w;
    w.x = (nx * ay - ny * ax) * inv;
    w.y = (nx * ax + ny * ay) * inv;
    return w;
}

// Interior branch: Weideman's rational series.  The real-coefficient
// polynomial p(Z) = sum_{n=1}^{N} a_n Z^{n-1} is evaluated at the complex
// point Z by synthetic division by the real quadratic with roots Z and
// conj(Z), Z^2 - r Z - s (r = 2 Re Z, s = -|Z|^2): b_{N-1} = a_N,
// b_{N-2} = a_{N-1} + r b_{N-1}, b_j = a_{j+1} + r b_{j+1} + s b_{j+2}, and
// p(Z) = b_1 Z + a_1 + s b_2 (two real FMAs per coefficient).
template <class R>
__device__ __forceinline__ C2<R> faddeeva_interior(R x, R y)
{
    constexpr int N = FadCfg<R>::N;
    const R L = weidL<R>();
    // d = L - i z = (L + y) - i x;  r = 1/d
    const R dx = L + y, dy = -x;
    const R inv = fast_rcp(dx * dx + dy * dy);
    const R rx = dx * inv, ry = -dy * inv;
    // Z = (L + i z) r = ((L - y) + i x) r
    const R mx = L - y, my = x;
    const R Zx = mx * rx - my * ry, Zy = mx * ry + my * rx;
    const R r = R(2) * Zx, sq = -(Zx * Zx + Zy * Zy);
    R b2 = weid<R>(N);
    R b1 = weid<R>(N - 1) + r * b2;
#pragma unroll
    for (int j = N - 3; j >= 1; --j) {
        const R b0 = weid<R>(j + 1) + r * b1 + sq * b2;
        b2 = b1;
        b1 = b0;
    }
    const R px = weid<R>(1) + sq * b2 + b1 * Zx, py = b1 * Zy;
    const R r2x = rx * rx - ry * ry, r2y = R(2) * rx * ry;
    const R s = R(0.56418958354775628695);
    C2<R> w;
    w.x = R(2) * (px * r2x - py * r2y) + rx * s;
    w.y = R(2) * (px * r2y + py * r2x) + ry * s;
    return w;
}

// w(z) = exp(-z^2) erfc(-i z) for z = x + i y, y >= 0.
//
// Interior |z| <= R: Weideman's (1994) rational series
//     w(z) = 2 p(Z) / (L - i z)^2 + (1/sqrt(pi)) / (L - i z),
//     Z = (L + i z) / (L - i z),  p(Z) = sum_{n=1}^{N} a_n Z^{n-1},
// with a_n the Fourier coefficients of (L^2 + t^2) exp(-t^2) under
// t = L tan(theta/2) (computed on the host from that integral).
// Exterior |z| > R: the k-th convergent of the Laplace continued fraction
//     w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/(z - ...)))),
// written as a ratio of polynomials in u = z^2.  Both branches need one
// reciprocal.  Absolute error: FP32 ~1e-7 (N = 16, k = 3, R = 6), FP64 ~2e-15
// (N = 36, k = 9, R = 8).  r2 = x^2 + y^2 is passed in so that every caller
// takes the same branch decision.
template <class R>
__device__ __forceinline__ C2<R> faddeeva_r2(R x, R y, R a2, R r2)
{
    if (r2 > FadCfg<R>::R2) return faddeeva_exterior<R>(x, y, a2);
    return faddeeva_interior<R>(x, y);
}

template <class R>
__device__ __forceinline__ C2<R> faddeeva(R x, R y)
{
    const R a2 = y * y;
    return faddeeva_r2<R>(x, y, a2, x * x + a2);
}

// The three Zeeman components of one line at one wavelength: sigma_b at
// v + v_B, pi at v, sigma_r at v - v_B (each x = doff/D + offset, one FMA).
// When |v| - |v_B| = m > 0 the smallest |x| is m, so m^2 + a^2 > R^2 puts all
// three outside |z| = R; they are then evaluated without branches and their
// continued fractions overlap.  Otherwise each component picks its branch.
template <class R>
__device__ __forceinline__ bool triplet_exterior(R v, R vB, R a2)
{
    const R m = fabs(v) - fabs(vB);
    return m > R(0) && m * m + a2 > FadCfg<R>::R2;
}

template <class R>
__device__ __forceinline__ void faddeeva_triplet(R xb, R v, R xr, R vB, R a, R a2, C2<R> &wb,
                                                 C2<R> &wp, C2<R> &wr)
{
    if (triplet_exterior<R>(v, vB, a2)) {
        wb = faddeeva_exterior<R>(xb, a, a2);
        wp = faddeeva_exterior<R>(v, a, a2);
        wr = faddeeva_exterior<R>(xr, a, a2);
    } else {
        wb = faddeeva_r2<R>(xb, a, a2, xb * xb + a2);
        wp = faddeeva_r2<R>(v, a, a2, v * v + a2);
        wr = faddeeva_r2<R>(xr, a, a2, xr * xr + a2);
    }
}

// ------------------------------------------------------ per-model geometry
template <class R> struct Geo {
    R a, a2;            // damping, damping^2
    R kIp, kIs;         // eta0 sin^2 t, eta0 (1 + cos^2 t)/2
    R kQ, kU, kV;       // eta0 sin^2 t cos 2chi, eta0 sin^2 t sin 2chi, eta0 cos t
    R kIp2, kV2;        // kIp^2, kV^2
    R kUV, kQV;         // kU kV, kQ kV
    R S0, muS1;
    R eta0, alpha;          // line strength; fill fraction (1 without one)
    // FP32 pair path: |x| thresholds of the far, outer-shell, continued-
    // fraction and middle regions (|x| > t <=> x^2 + a^2 > R^2; -1 when
    // a^2 >= R^2); a triplet is wholly beyond one when |v| - |v_B| is
    R tfar, t80, text, tmid;
    unsigned vmask;     // pair path: the lanes that evaluate together (votes)
    R shift[ME_MAX_LINES];  // lambda0 v_LOS / c [A]
    R invD[ME_MAX_LINES];   // 1 / Doppler width [1/A]
    R vB[ME_MAX_LINES];     // Zeeman splitting in Doppler units
    R cp[ME_MAX_LINES];     // -shift / D: x_pi = doff / D + cp
    R vL[ME_MAX_LINES];     // Larmor displacement in Doppler units (full patterns)
};

__device__ __forceinline__ void sincos_deg(float d, float *s, float *c)
{
    sincospif(d * (1.0f / 180.0f), s, c);
}
__device__ __forceinline__ void sincos_deg(double d, double *s, double *c)
{
    sincospi(d * (1.0 / 180.0), s, c);
}

// Geometry of one parameter vector p (Section 5 model vector), in R.
// FILL: p[9] is the fill fraction alpha of Section 5.2.
template <class R, int NL, bool FILL = false>
__device__ __forceinline__ Geo<R> make_geo(const KProblem &pb, int nlines, const R *p, R mu)
{
    Geo<R> g;
    R st, ct, s2c, c2c;
    sincos_deg(p[1], &st, &ct);
    sincos_deg(R(2) * p[2], &s2c, &c2c);
    const R eta0 = p[6];
    const R s2 = st * st;
    g.a = p[5];
    g.a2 = g.a * g.a;
    g.kIp = eta0 * s2;
    g.kIs = eta0 * R(0.5) * (R(1) + ct * ct);
    g.kQ = eta0 * s2 * c2c;
    g.kU = eta0 * s2 * s2c;
    g.kV = eta0 * ct;
    g.kIp2 = g.kIp * g.kIp;
    g.kV2 = g.kV * g.kV;
    g.kUV = g.kU * g.kV;
    g.kQV = g.kQ * g.kV;
    g.S0 = p[7];
    g.muS1 = mu * p[8];
    g.eta0 = eta0;
    if constexpr (FILL) g.alpha = p[9];
    else g.alpha = R(1);
    const int nl = NL > 0 ? NL : nlines;
#pragma unroll
    for (int l = 0; l < (NL > 0 ? NL : ME_MAX_LINES); ++l) {
        if (l < nl) {
            const KLine &ln = pb.line[l];
            g.shift[l] = R(ln.lam0_c) * p[3];
            g.invD[l] = R(1) / (p[4] * R(ln.dscale));
            g.vB[l] = R(ln.zfac) * p[0] * g.invD[l];
            g.cp[l] = -g.shift[l] * g.invD[l];
            g.vL[l] = R(ln.zfacL) * p[0] * g.invD[l];
        }
    }
    return g;
}

template <class R> struct Stokes4 { R I, Q, U, V; };

// Section 5.2 fill fraction: Stokes <- alpha Stokes + (1 - alpha) I_nm e with
// the field-free I_nm = S0 + mu S1 / (1 + eta0 sum_l eta_ratio_l Re w0_l)
// (w0 the unshifted profile); P0 = sum_l (eta_ratio_l / 2) Re w0_l.
template <class R>
__device__ __forceinline__ void fill_mix(Stokes4<R> &s, const Geo<R> &g, R P0)
{
    const R inm = g.muS1 * fast_rcp(R(1) + R(2) * g.eta0 * P0);
    s.I = g.S0 + g.alpha * (s.I - g.S0) + (R(1) - g.alpha) * inm;
    s.Q *= g.alpha;
    s.U *= g.alpha;
    s.V *= g.alpha;
}

// Group profiles (sigma_b, pi, sigma_r) of a line with a full Zeeman pattern:
// each is the strength-weighted sum of its components' w(x_i + i a), with
// x_i = doff / D + cp - v_L s_i.
template <class R>
__device__ __forceinline__ void pattern_profiles(const KLine &ln, R dinv, R cp, R vL, R a, R a2,
                                                 C2<R> &wb, C2<R> &wp, C2<R> &wr)
{
    C2<R> out[3];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        R px = R(0), py = R(0);
        const int n = ln.ncomp[g];
        for (int i = 0; i < n; ++i) {
            const R x = dinv + (cp - vL * comp_shift<R>(ln, g, i));
            const C2<R> wi = faddeeva_r2<R>(x, a, a2, x * x + a2);
            const R st = comp_str<R>(ln, g, i);
            px += st * wi.x;
            py += st * wi.y;
        }
        out[g].x = px;
        out[g].y = py;
    }
    wb = out[0];
    wp = out[1];
    wr = out[2];
}

// Stokes vector at one wavelength.  doff[l] = lambda_j - lambda0_l (exact in
// FP64, rounded to R), half_eta[l] = eta_ratio_l / 2.
// PAT = false compiles out full-pattern lines (problems with effective
// triplets only); PAT = true checks each line at run time.
// FILL mixes in the field-free profile with the fill fraction g.alpha.
template <class R, int NL, bool PAT = true, bool FILL = false>
__device__ __forceinline__ Stokes4<R> me_point(const Geo<R> &g, const R *doff, const R *half_eta,
                                               int nlines, const KLine *lines)
{
    R P = 0, Sg = 0, T = 0, Dd = 0, Ti = 0, Di = 0, P0 = 0;
    const int nl = NL > 0 ? NL : nlines;
#pragma unroll
    for (int l = 0; l < (NL > 0 ? NL : ME_MAX_LINES); ++l) {
        if (l < nl) {
            C2<R> wb, wp, wr;
            if (!PAT || lines[l].ncomp[0] == 0) {
                const R v = doff[l] * g.invD[l] + g.cp[l];
                const R xb = doff[l] * g.invD[l] + (g.cp[l] + g.vB[l]);
                const R xr = doff[l] * g.invD[l] + (g.cp[l] - g.vB[l]);
                faddeeva_triplet<R>(xb, v, xr, g.vB[l], g.a, g.a2, wb, wp, wr);
                if (FILL) P0 += half_eta[l] * wp.x;  // the pi profile is unshifted
            } else {
                pattern_profiles<R>(lines[l], doff[l] * g.invD[l], g.cp[l], g.vL[l], g.a, g.a2, wb, wp, wr);
                if (FILL) P0 += half_eta[l] * faddeeva<R>(doff[l] * g.invD[l] + g.cp[l], g.a).x;
            }
            const R q = half_eta[l];
            const R sx = wb.x + wr.x, sy = wb.y + wr.y;
            P += q * wp.x;
            Sg += q * sx;
            T += q * (wp.x - R(0.5) * sx);
            Ti += q * (wp.y - R(0.5) * sy);
            Dd += q * (wr.x - wb.x);
            Di += q * (wr.y - wb.y);
        }
    }
    // eta_Q, eta_U share the profile sum T and rho_Q, rho_U share Ti
    // (eta_Q = kQ T, eta_U = kU T, rho_Q = kQ Ti, rho_U = kU Ti, kQ^2 + kU^2 =
    // kIp^2), so the closed form of K^-1 e simplifies exactly to
    //   E2 = eQ^2+eU^2+eV^2 = kIp^2 T^2 + kV^2 Dd^2,  rho2 = kIp^2 Ti^2 + kV^2 Di^2,
    //   Pi = kIp^2 T Ti + kV^2 Dd Di,  A = eI^2 T + Ti Pi,  C = Dd Ti - T Di,
    //   Q = -f (kQ A + kU kV eI C),  U = -f (kU A - kQ kV eI C),
    //   V = -f kV (eI^2 Dd + Di Pi)   (the eI (eU rQ - eQ rU) term vanishes).
    const R eI = R(1) + g.kIp * P + g.kIs * Sg;
    const R pT = g.kIp2 * T, pTi = g.kIp2 * Ti, vD = g.kV2 * Dd, vDi = g.kV2 * Di;
    const R E2 = pT * T + vD * Dd;
    const R rho2 = pTi * Ti + vDi * Di;
    const R Pi = pT * Ti + vD * Di;
    const R eI2 = eI * eI;
    const R Delta = eI2 * (eI2 - E2 + rho2) - Pi * Pi;
    const R f = g.muS1 * fast_rcp(Delta);
    const R A = eI2 * T + Ti * Pi;
    const R eIC = eI * (Dd * Ti - T * Di);
    Stokes4<R> s;
    s.I = g.S0 + f * eI * (eI2 + rho2);
    s.Q = -f * (g.kQ * A + g.kUV * eIC);
    s.U = -f * (g.kU * A - g.kQV * eIC);
    s.V = -f * g.kV * (eI2 * Dd + Di * Pi);
    if (FILL) fill_mix(s, g, P0);
    return s;
}

// Number of Faddeeva evaluations at one wavelength that take the interior
// (Weideman) branch; the same test as faddeeva().  Used only by the counting
// instantiation of the GA kernel, to turn branch counts into flops.
template <class R, int NL, bool PAT = true>
__device__ __forceinline__ unsigned count_interior(const Geo<R> &g, const R *doff, int nlines,
                                                   const KLine *lines)
{
    unsigned c = 0;
    const int nl = NL > 0 ? NL : nlines;
#pragma unroll
    for (int l = 0; l < (NL > 0 ? NL : ME_MAX_LINES); ++l) {
        if (PAT && l < nl && lines[l].ncomp[0] != 0) {
            const R dinv = doff[l] * g.invD[l];
            for (int gg = 0; gg < 3; ++gg)
                for (int i = 0; i < lines[l].ncomp[gg]; ++i) {
                    const R x = dinv + (g.cp[l] - g.vL[l] * comp_shift<R>(lines[l], gg, i));
                    c += (x * x + g.a2 > FadCfg<R>::R2) ? 0u : 1u;
                }
        } else if (l < nl) {
            const R v = doff[l] * g.invD[l] + g.cp[l];
            const R xb = doff[l] * g.invD[l] + (g.cp[l] + g.vB[l]);
            const R xr = doff[l] * g.invD[l] + (g.cp[l] - g.vB[l]);
            const R a2 = g.a2;
            if (!triplet_exterior<R>(v, g.vB[l], a2)) {
                c += (xb * xb + a2 > FadCfg<R>::R2) ? 0u : 1u;
                c += (v * v + a2 > FadCfg<R>::R2) ? 0u : 1u;
                c += (xr * xr + a2 > FadCfg<R>::R2) ? 0u : 1u;
            }
        }
    }
    return c;
}

}  // namespace genesis
