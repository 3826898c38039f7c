// FP32 synthesis of two wavelength points at once with packed FP32x2 arithmetic
// (sm_100+ FFMA2/FMUL2/FADD2): the same formulas as me_point<float>, with the
// .x lane holding wavelength j and the .y lane wavelength j+1.  One packed
// instruction does the work of two scalar ones, which halves the issue slots
// of the GA's fitness loop (an issue-bound loop of FP32 arithmetic).
//
// Branches are uniform across the warp.  A Zeeman component takes the
// far-field approximant when every lane's pair of points is beyond
// |z|^2 = 360, the even (three-node) convergent of the continued fraction when
// every pair is beyond |z|^2 = 80, the 3rd convergent beyond 36, the 5th
// beyond 21, and Weideman's series otherwise.  Each branch is accurate
// wherever it is taken: the convergents and the far field to 1.3e-7 or better
// beyond their thresholds, the series everywhere (truncation error 4.3e-8 for
// |x| <= 1e4, 0 <= y <= 1; near the line centre, where |w| is about 1, FP32
// rounding of the series is the larger term, about 1e-6 relative).  A point's
// value can therefore depend on its partner's and its warp's regions, always
// within that budget.
// An effective triplet is tested as a whole first: wholly far, all three
// components take the far field; wholly beyond 80 the even convergent, wholly
// beyond 36 the 3rd convergent; otherwise (near a line core) each component
// tests the regions from the inside out.  A warp-uniform choice costs one branch where a
// per-lane choice would run both for a mixed warp.  A region test is one
// comparison of the pair's nearer |x| with a per-individual threshold, and
// the vote reuses the fitness call's lane mask: the loop's issue slots, not
// its flops, set its speed.
#pragma once

#include "me_device.cuh"

namespace genesis {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(fast_rcp(a.x), fast_rcp(a.y)); }
// A shared-memory vector load the compiler keeps where it is written (not
// hoisted out of the loop that contains it).
__device__ __forceinline__ float4 lds4(const float4 *p)
{
    float4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// Every branch returns a weighted profile value q w(z) as qi (nx + i ny): the
// caller adds qi nx and qi ny into its sums with one FMA each.  The rational
// branches leave their numerator unnormalised and put q / (sqrt(pi) |A|^2)
// into qi (qs = q / sqrt(pi) is passed in), which saves the two multiplies of
// a normalised w; the series returns w itself with qi = q.  For an effective
// triplet the series instead adds q w into the sums itself (fad_int2_acc,
// with the line's coefficients scaled by q on the host).

// Continued-fraction branch (K-th convergent, monic a(u), b(u)) for a pair of
// real arguments x and a common damping y (a2 = y^2).
template <int K>
__device__ __forceinline__ void fad_cf2(float2 x, float y, float a2, float2 qs, float2 &wx, float2 &wy,
                                        float2 &qi)
{
    constexpr int NA = (K + 1) / 2, NB = (K - 1) / 2;
    constexpr CfPoly<K> P{};
    const float2 ux = fma2(x, x, f2(-a2));
    const float2 uy = mul2(x, f2(2.0f * y));
    float2 ax = add2(ux, f2((float)P.a[NA - 1])), ay = uy;
#pragma unroll
    for (int n = NA - 2; n >= 0; --n) {
        const float2 tx = fma2(ax, ux, fma2(neg2(ay), uy, f2((float)P.a[n])));
        ay = fma2(ax, uy, mul2(ay, ux));
        ax = tx;
    }
    float2 bx = f2(1.0f), by = f2(0.0f);
    if (NB >= 1) {
        bx = add2(ux, f2((float)P.b[NB - 1]));
        by = uy;
    }
#pragma unroll
    for (int n = NB - 2; n >= 0; --n) {
        const float2 tx = fma2(bx, ux, fma2(neg2(by), uy, f2((float)P.b[n])));
        by = fma2(bx, uy, mul2(by, ux));
        bx = tx;
    }
    // num = z b(u), z = x + i y;  w = (i/sqrt(pi)) num conj(a(u)) / |a(u)|^2
    const float2 nx = fma2(x, bx, mul2(f2(-y), by));
    const float2 ny = fma2(x, by, mul2(f2(y), bx));
    qi = mul2(qs, rcp2(fma2(ax, ax, mul2(ay, ay))));
    wx = fma2(nx, ay, neg2(mul2(ny, ax)));
    wy = fma2(nx, ax, mul2(ny, ay));
}
// The 3rd convergent w = (i/sqrt(pi)) z (z^2 - 5/2) / (z^4 - 3 z^2 + 3/4) for
// R2 < |z|^2 <= kEven2R2, written in s = |z|^2 for real x: with N = z (z^2 - 5/2),
// D = z^4 - 3 z^2 + 3/4 and z = x + i y,
//   i N conj(D) = y (s^3 - 4.5 s^2 + c1 s + c0) + i x (s^3 - 5.5 s^2 + (c1 + 3) s - c0),
//   |D|^2 = s^4 - 6 s^3 + d2 s^2 + (6 - d2) s + d0,
// c1 = 5.25 + 10 y^2, c0 = 1.875 + 3 y^2, d2 = 10.5 + 12 y^2,
// d0 = 12 y^4 + 9 y^2 + 0.5625 (per individual), 14 packed operations where
// the complex polynomials take 19.
__device__ __forceinline__ void fad_ext2(float2 x, float y, float a2, float2 qs, float2 &wx, float2 &wy,
                                         float2 &qi)
{
    static_assert(FadCfg<float>::K == 3, "the s-form is the 3rd convergent");
    const float c1 = fmaf(10.0f, a2, 5.25f), c0 = fmaf(3.0f, a2, 1.875f);
    const float d2 = fmaf(12.0f, a2, 10.5f), d0 = fmaf(fmaf(12.0f, a2, 9.0f), a2, 0.5625f);
    const float2 s = fma2(x, x, f2(a2));
    const float2 pr = fma2(fma2(s, add2(s, f2(-4.5f)), f2(c1)), s, f2(c0));
    const float2 pi = fma2(fma2(s, add2(s, f2(-5.5f)), f2(c1 + 3.0f)), s, f2(-c0));
    const float2 den = fma2(fma2(fma2(add2(s, f2(-6.0f)), s, f2(d2)), s, f2(6.0f - d2)), s, f2(d0));
    qi = mul2(qs, rcp2(den));
    wx = mul2(f2(y), pr);
    wy = mul2(x, pi);
}
// Middle shell kMidR2 < |z|^2 <= R2: the 5th convergent (six-node rule),
// |error| <= 1.04e-7 there (at the boundary), about half the work of
// Weideman's series.
constexpr float kMidR2 = 21.0f;

// Outer shell kEven2R2 < |z|^2 <= kFarR2: the even convergent
// w = (i/sqrt(pi)) (z^2 - 1) / (z (z^2 - 3/2)) of the Laplace continued fraction
// (the three-node Gauss-Hermite rule), |error| <= 1.13e-7 in FP32 there (at
// the boundary; it falls outward), within the 1.3e-7 of the 3rd convergent.
constexpr float kEven2R2 = 80.0f;
__device__ __forceinline__ void fad_even2(float2 x, float y, float a2, float2 qs, float2 &wx, float2 &wy,
                                          float2 &qi)
{
    // With N = z^2 - 1, D = z (z^2 - 3/2), z = x + i y and s = |z|^2 = x^2 + y^2
    // (x real, y the damping): i N conj(D) = y P + i x (P - s) with
    // P = s^2 - 1.5 s + 4 y^2 + 1.5, and |D|^2 = s (s^2 - 3 s + 6 y^2 + 9/4).
    // In m = s - 3/2 (one FMA from x, like s): P = m s + 4 y^2 + 1.5 and
    // s^2 - 3 s + 6 y^2 + 9/4 = m^2 + 6 y^2, nine packed operations in all.
    const float2 s = fma2(x, x, f2(a2));
    const float2 m = fma2(x, x, f2(a2 - 1.5f));
    const float2 pr = fma2(m, s, f2(4.0f * a2 + 1.5f));
    const float2 u = fma2(m, m, f2(6.0f * a2));
    qi = mul2(qs, rcp2(mul2(s, u)));
    wx = mul2(f2(y), pr);
    wy = mul2(x, sub2(pr, s));
}

// Far field (|z|^2 > kFarR2): the first non-trivial convergent of the Laplace
// continued fraction (the two-node Gauss-Hermite rule), w = (i/sqrt(pi)) z /
// (z^2 - 1/2); |error| <= 1.23e-7 in FP32 there (at the boundary; it falls
// as |z|^-5 outward), within the 1.3e-7 of the 3rd convergent at |z|^2 = 36.
constexpr float kFarR2 = 360.0f;
__device__ __forceinline__ void fad_far2(float2 x, float y, float a2, float2 qs, float2 &wx, float2 &wy,
                                         float2 &qi)
{
    // With z = x + i y and s = |z|^2 (x real): i z conj(z^2 - 1/2) =
    // y (s + 1/2) + i x (s - 1/2) and |z^2 - 1/2|^2 = (s - 1/2)^2 + 2 y^2, all
    // three in u = s - 1/2 (one FMA from x): five packed operations.
    const float2 u = fma2(x, x, f2(a2 - 0.5f));
    qi = mul2(qs, rcp2(fma2(u, u, f2(2.0f * a2))));
    wx = fma2(f2(y), u, f2(y));
    wy = mul2(x, u);
}

// Interior branch (Weideman N = 16, real-quadratic synthetic division) for a
// pair of real arguments x and common damping y.
__device__ __forceinline__ void fad_int2(float2 x, float y, float2 q, float2 &wx, float2 &wy, float2 &qi)
{
    qi = q;
    constexpr int N = FadCfg<float>::N;
    const float L = c_fad.L32;
    // 1/(L - i z) = (dx + i x) / (dx^2 + x^2), dx = L + y
    const float dx = L + y;
    const float2 inv = rcp2(fma2(x, x, f2(dx * dx)));
    const float2 rx = mul2(f2(dx), inv), ry = mul2(x, inv);
    // Z = ((L - y) + i x) / ((L + y) - i x) = ((L^2 - y^2 - x^2) + i 2 L x) inv
    const float2 Zx = mul2(fma2(neg2(x), x, f2((L - y) * dx)), inv);
    const float2 Zy = mul2(ry, f2(2.0f * L));
    const float2 r = add2(Zx, Zx), sq = neg2(fma2(Zx, Zx, mul2(Zy, Zy)));
    float2 b2 = c_fad.w32x2[N];
    float2 b1 = fma2(r, b2, c_fad.w32x2[N - 1]);
#pragma unroll
    for (int j = N - 3; j >= 1; --j) {
        const float2 b0 = fma2(r, b1, fma2(sq, b2, c_fad.w32x2[j + 1]));
        b2 = b1;
        b1 = b0;
    }
    const float2 px = fma2(sq, b2, fma2(b1, Zx, c_fad.w32x2[1])), py = mul2(b1, Zy);
    // w = (2 p(Z) r + 1/sqrt(pi)) r with r = 1/(L - i z) = rx + i ry
    const float2 ux = fma2(px, rx, fma2(neg2(py), ry, f2(0.56418958354775628695f)));
    const float2 uy = fma2(px, ry, mul2(py, rx));
    wx = fma2(ux, rx, neg2(mul2(uy, ry)));
    wy = fma2(ux, ry, mul2(uy, rx));
}


// Weideman's series for an effective triplet's component, added into the
// caller's sums: the line's coefficients arrive scaled by its strength q
// (wq = q 2 a_n) and qs = q / sqrt(pi), so (p r + qs) r is q w itself and its
// product with r goes straight into the sums (Ax, Ay) += q w.
__device__ __forceinline__ void fad_int2_acc(float2 x, float y, const float2 *wq, float2 qs, float2 &Ax,
                                             float2 &Ay)
{
    constexpr int N = FadCfg<float>::N;
    const float L = c_fad.L32;
    const float dx = L + y;
    const float2 inv = rcp2(fma2(x, x, f2(dx * dx)));
    const float2 rx = mul2(f2(dx), inv), ry = mul2(x, inv);
    const float2 Zx = mul2(fma2(neg2(x), x, f2((L - y) * dx)), inv);
    const float2 Zy = mul2(ry, f2(2.0f * L));
    const float2 r = add2(Zx, Zx), sq = neg2(fma2(Zx, Zx, mul2(Zy, Zy)));
    float2 b2 = wq[N];
    float2 b1 = fma2(r, b2, wq[N - 1]);
#pragma unroll
    for (int j = N - 3; j >= 1; --j) {
        const float2 b0 = fma2(r, b1, fma2(sq, b2, wq[j + 1]));
        b2 = b1;
        b1 = b0;
    }
    const float2 px = fma2(sq, b2, fma2(b1, Zx, wq[1])), py = mul2(b1, Zy);
    const float2 ux = fma2(px, rx, fma2(neg2(py), ry, qs));
    const float2 uy = fma2(px, ry, mul2(py, rx));
    Ax = fma2(ux, rx, fma2(neg2(uy), ry, Ax));
    Ay = fma2(ux, ry, fma2(uy, rx, Ay));
}

// |x| threshold of a region x^2 + a^2 > R2 (once per individual).
__device__ __forceinline__ float region_threshold(float R2, float a2) { return a2 >= R2 ? -1.0f : sqrtf(R2 - a2); }
// Fill the pair path's thresholds of a geometry (once per individual).
__device__ __forceinline__ void pair_thresholds(Geo<float> &g, int)
{
    g.tfar = region_threshold(kFarR2, g.a2);
    g.t80 = region_threshold(kEven2R2, g.a2);
    g.text = region_threshold(FadCfg<float>::R2, g.a2);
    g.tmid = region_threshold(kMidR2, g.a2);
}
// Nearer |x| of a pair: the pair is beyond a threshold t when this is.
__device__ __forceinline__ float pair_min_abs(float2 x) { return fminf(fabsf(x.x), fabsf(x.y)); }
// A predicate that holds for every lane of mask, the lanes that evaluate
// together.  The vote only chooses among branches that are each accurate for
// every lane they are taken by (a lane takes a cheaper branch only if its own
// points qualify), so it is correct for any set of voting lanes.  The fitness
// loop takes the mask once per call (__activemask() on entry): its branches
// are all warp-uniform, so the set of lanes does not change inside it, and a
// caller that runs divergent (the GA's restarts evaluate only part of a
// warp) votes over just its active lanes.
__device__ __forceinline__ bool warp_all(bool p, unsigned mask) { return __all_sync(mask, p); }

// 1 / sqrt(pi), the factor of the rational branches.
constexpr float kInvSqrtPi = 0.56418958354775628695f;

// One component for the pair, weighted by q (qs = q / sqrt(pi)), the branch
// chosen uniformly across the warp.
__device__ __forceinline__ void fad_pair(float2 x, const Geo<float> &g, float2 q, float2 qs, float2 &wx,
                                         float2 &wy, float2 &qi)
{
    const float m = pair_min_abs(x);
    if (warp_all(m > g.tfar, g.vmask)) fad_far2(x, g.a, g.a2, qs, wx, wy, qi);
    else if (warp_all(m > g.t80, g.vmask)) fad_even2(x, g.a, g.a2, qs, wx, wy, qi);
    else if (warp_all(m > g.text, g.vmask)) fad_ext2(x, g.a, g.a2, qs, wx, wy, qi);
    else if (warp_all(m > g.tmid, g.vmask)) fad_cf2<5>(x, g.a, g.a2, qs, wx, wy, qi);
    else fad_int2(x, g.a, q, wx, wy, qi);
}

// Work counts of the algorithm proper: each real point's evaluation classified
// by its own region (Weideman interior, middle shell, 3rd convergent, outer
// shell, far field), whatever branch its pair and warp took.
struct EvalCount {
    unsigned interior, mid, even2, far;
};
__device__ __forceinline__ void count_point(float x, float a2, EvalCount &n)
{
    const float r = x * x + a2;
    n.interior += r > kMidR2 ? 0u : 1u;
    n.mid += (r > kMidR2 && r <= FadCfg<float>::R2) ? 1u : 0u;
    n.even2 += (r > kEven2R2 && r <= kFarR2) ? 1u : 0u;
    n.far += r > kFarR2 ? 1u : 0u;
}
__device__ __forceinline__ void count_pair(float2 x, float a2, bool y_real, EvalCount &n)
{
    count_point(x.x, a2, n);
    if (y_real) count_point(x.y, a2, n);
}

struct Stokes4x2 {
    float2 I, Q, U, V;
};

// Full Zeeman pattern for a pair of points: each group's strength-weighted sum
// of components (see pattern_profiles).
template <bool COUNT>
__device__ __forceinline__ void pattern_profiles_x2(const KLine &ln, float2 dinv, float cp, float vL,
                                                    const Geo<float> &geo, float2 w[6], bool y_real,
                                                    EvalCount &ncount)
{
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        float2 px = f2(0.f), py = f2(0.f);
        const int n = ln.ncomp[g];
        for (int i = 0; i < n; ++i) {
            const float2 x = add2(dinv, f2(cp - vL * ln.cshift32[g][i]));
            if (COUNT) count_pair(x, geo.a2, y_real, ncount);
            const float st = ln.cstr32[g][i];
            float2 wx, wy, qi;
            fad_pair(x, geo, f2(st), f2(st * kInvSqrtPi), wx, wy, qi);
            px = fma2(qi, wx, px);
            py = fma2(qi, wy, py);
        }
        w[2 * g] = px;
        w[2 * g + 1] = py;
    }
}

// One component near a line core: the same branches tested from the inside
// out, for components that mostly need the inner ones.
__device__ __forceinline__ void fad_pair_in(float2 x, const Geo<float> &g, float2 q, float2 qs, float2 &wx,
                                            float2 &wy, float2 &qi)
{
    const float m = pair_min_abs(x);
    if (!warp_all(m > g.tmid, g.vmask)) fad_int2(x, g.a, q, wx, wy, qi);
    else if (!warp_all(m > g.text, g.vmask)) fad_cf2<5>(x, g.a, g.a2, qs, wx, wy, qi);
    else if (!warp_all(m > g.t80, g.vmask)) fad_ext2(x, g.a, g.a2, qs, wx, wy, qi);
    else fad_even2(x, g.a, g.a2, qs, wx, wy, qi);
}

// Adds qi (wx + i wy) into (Ax, Ay).
__device__ __forceinline__ void acc_w(float2 qi, float2 wx, float2 wy, float2 &Ax, float2 &Ay)
{
    Ax = fma2(qi, wx, Ax);
    Ay = fma2(qi, wy, Ay);
}

// One effective-triplet component near a line core, added into (Ax, Ay):
// the branches of fad_pair_in, the series with the line's scaled coefficients.
__device__ __forceinline__ void fad_pair_in_acc(float2 x, const Geo<float> &g, const float2 *wq, float2 qs,
                                                float2 &Ax, float2 &Ay)
{
    const float m = pair_min_abs(x);
    if (!warp_all(m > g.tmid, g.vmask)) {
        fad_int2_acc(x, g.a, wq, qs, Ax, Ay);
        return;
    }
    float2 wx, wy, qi;
    if (!warp_all(m > g.text, g.vmask)) fad_cf2<5>(x, g.a, g.a2, qs, wx, wy, qi);
    else if (!warp_all(m > g.t80, g.vmask)) fad_ext2(x, g.a, g.a2, qs, wx, wy, qi);
    else fad_even2(x, g.a, g.a2, qs, wx, wy, qi);
    acc_w(qi, wx, wy, Ax, Ay);
}

// One component at a known level, added into (Ax, Ay): 3 = every lane's pair
// is in the far field, 2 = beyond the outer shell's threshold (the even
// convergent, accurate there, also where a component is already far), 1 =
// beyond the continued-fraction threshold (the 3rd convergent, likewise), 0 =
// anywhere (cheaper than testing each component).
template <int LEVEL>
__device__ __forceinline__ void fad_level_acc(float2 x, const Geo<float> &g, const float2 *wq, float2 qs,
                                              float2 &Ax, float2 &Ay)
{
    if (LEVEL == 0) {
        fad_pair_in_acc(x, g, wq, qs, Ax, Ay);
        return;
    }
    float2 wx, wy, qi;
    if (LEVEL == 3) fad_far2(x, g.a, g.a2, qs, wx, wy, qi);
    else if (LEVEL == 2) fad_even2(x, g.a, g.a2, qs, wx, wy, qi);
    else fad_ext2(x, g.a, g.a2, qs, wx, wy, qi);
    acc_w(qi, wx, wy, Ax, Ay);
}

// One effective triplet's contribution to a pair's profile sums, each
// component added as soon as it is evaluated (EXT: the level of fad_level_acc
// that every lane's triplet reaches as a whole).  The sigma components go
// into sums of their own (Sb, Sbi blue, Sr, Sri red); their sum and
// difference are formed once per point after the last line.
template <int EXT, bool FILL>
__device__ __forceinline__ void triplet_acc(float2 xb, float2 v, float2 xr, const Geo<float> &g,
                                            const float2 *wq, float2 qs, float2 &P, float2 &Pim, float2 &Sb,
                                            float2 &Sbi, float2 &Sr, float2 &Sri, float2 &P0)
{
    fad_level_acc<EXT>(xb, g, wq, qs, Sb, Sbi);
    if (FILL) {  // the pi profile is unshifted: its real part also feeds P0
        float2 tx = f2(0.f), ty = f2(0.f);
        fad_level_acc<EXT>(v, g, wq, qs, tx, ty);
        P = add2(P, tx);
        Pim = add2(Pim, ty);
        P0 = add2(P0, tx);
    } else {
        fad_level_acc<EXT>(v, g, wq, qs, P, Pim);
    }
    fad_level_acc<EXT>(xr, g, wq, qs, Sr, Sri);
}

// The branch level of an effective triplet for a pair, voted across the warp
// from its pi arguments v (the sigma arguments are v +- v_B): 3 when every
// lane's triplet is wholly in the far field (|v| > t_far + |v_B|), 2 when
// wholly beyond the outer shell's threshold, 1 when wholly beyond the
// continued-fraction threshold, 0 near a line core.
__device__ __forceinline__ int triplet_level(float2 v, const Geo<float> &g, int l)
{
    // the nearest component's |x| is at least |v| - |v_B|
    const float m = pair_min_abs(v) - fabsf(g.vB[l]);
    if (!warp_all(m > g.text, g.vmask)) return 0;
    if (warp_all(m > g.tfar, g.vmask)) return 3;
    return warp_all(m > g.t80, g.vmask) ? 2 : 1;
}

// Residuals o - Stokes at two wavelength points (the synthesis of Section
// 5 and the difference of Eq. chisq).  doff2[l] holds (lambda_j -
// lambda0_l, lambda_{j+1} - lambda0_l); op points at the pair's staged
// observed values (I, I', Q, Q', U, U', V, V' in shared memory), read only
// where the residuals are formed.  An effective triplet's q / sqrt(pi) and
// its series coefficients scaled by q come from the kernel parameters
// (lines[l].qs2, wq2), so they are constant-bank operands.  FILL mixes in the field-free
// profile with the fill fraction (Section 5.2, see fill_mix).  kc points at
// the individual's shared-memory slots (stride nt float4): (kIs, kIp, kIp2,
// kV2), (muS1, S0, kQ, kUV), (kU, kQV, kV, w_I), the last three weighted as
// fitness_pairs stores them; wI receives w_I.
template <int NL, bool COUNT, bool PAT, bool FILL = false>
__device__ __forceinline__ Stokes4x2 resid_x2(const Geo<float> &g, const float2 *doff2, const float *op,
                                              const float *half_eta, int nlines, bool y_real,
                                              EvalCount &ncount, const KLine *lines, const float4 *kc, int nt,
                                              float &wI)
{
    // profile sums over the lines: P, Pim = sum q phi_p, q psi_p; Sb, Sbi =
    // sum q phi_b, q psi_b; Sr, Sri = sum q phi_r, q psi_r.  Once per point:
    // Sg, Sgi = Sb + Sr, Sbi + Sri; Dd, Di = Sr - Sb, Sri - Sbi; T = P - Sg/2
    // and Ti = Pim - Sgi/2
    float2 P = f2(0.f), Pim = f2(0.f), Sb = f2(0.f), Sbi = f2(0.f), Sr = f2(0.f), Sri = f2(0.f);
    float2 P0 = f2(0.f);
    const int nl = NL > 0 ? NL : nlines;
#pragma unroll
    for (int l = 0; l < (NL > 0 ? NL : ME_MAX_LINES); ++l) {
        if (PAT && l < nl && lines[l].ncomp[0] != 0) {
            float2 w[6];
            pattern_profiles_x2<COUNT>(lines[l], mul2(doff2[l], f2(g.invD[l])), g.cp[l], g.vL[l], g, w, y_real,
                                       ncount);
            if (FILL) {
                float2 ux, uy, qi;
                fad_pair(fma2(doff2[l], f2(g.invD[l]), f2(g.cp[l])), g, f2(half_eta[l]),
                         f2(half_eta[l] * kInvSqrtPi), ux, uy, qi);
                P0 = fma2(qi, ux, P0);
            }
            const float2 q = f2(half_eta[l]);
            P = fma2(q, w[2], P);
            Pim = fma2(q, w[3], Pim);
            Sb = fma2(q, w[0], Sb);
            Sbi = fma2(q, w[1], Sbi);
            Sr = fma2(q, w[4], Sr);
            Sri = fma2(q, w[5], Sri);
        } else if (l < nl) {
            const float2 id = f2(g.invD[l]);
            const float2 v = fma2(doff2[l], id, f2(g.cp[l]));
            const float2 xb = add2(v, f2(g.vB[l]));
            const float2 xr = sub2(v, f2(g.vB[l]));
            if (COUNT) {
                count_pair(xb, g.a2, y_real, ncount);
                count_pair(v, g.a2, y_real, ncount);
                count_pair(xr, g.a2, y_real, ncount);
            }
            const float2 *wq = lines[l].wq2;
            const float2 qs = lines[l].qs2;
            const int lev = triplet_level(v, g, l);
            if (lev == 3)
                triplet_acc<3, FILL>(xb, v, xr, g, wq, qs, P, Pim, Sb, Sbi, Sr, Sri, P0);
            else if (lev == 2)
                triplet_acc<2, FILL>(xb, v, xr, g, wq, qs, P, Pim, Sb, Sbi, Sr, Sri, P0);
            else if (lev == 1)
                triplet_acc<1, FILL>(xb, v, xr, g, wq, qs, P, Pim, Sb, Sbi, Sr, Sri, P0);
            else
                triplet_acc<0, FILL>(xb, v, xr, g, wq, qs, P, Pim, Sb, Sbi, Sr, Sri, P0);
        }
    }
    // the sigma sums and differences, once per point
    const float2 Sg = add2(Sb, Sr), Sgi = add2(Sbi, Sri), Dd = sub2(Sr, Sb), Di = sub2(Sri, Sbi);
    // closed form of K^-1 e (see me_point), with G = eI^2 + rho^2 shared by
    // Delta = eI^2 (G - E2) - Pi^2 and I = S0 + f eI G.  The individual's
    // constants are read from its shared-memory slot here, once per pair, so
    // that they hold no registers across the profile evaluations.
    const float4 k0 = lds4(kc), k1 = lds4(kc + nt), k2 = lds4(kc + 2 * nt);
    const float kIs = k0.x, kIp = k0.y, kIp2 = k0.z, kV2 = k0.w;
    const float muS1 = k1.x, S0 = k1.y, kQ = k1.z, kUV = k1.w;
    const float kU = k2.x, kQV = k2.y, kV = k2.z;
    wI = k2.w;
    const float2 T = fma2(f2(-0.5f), Sg, P), Ti = fma2(f2(-0.5f), Sgi, Pim);
    const float2 eI = fma2(f2(kIs), Sg, fma2(f2(kIp), P, f2(1.0f)));
    const float2 pT = mul2(f2(kIp2), T), pTi = mul2(f2(kIp2), Ti);
    const float2 vD = mul2(f2(kV2), Dd), vDi = mul2(f2(kV2), Di);
    const float2 E2 = fma2(pT, T, mul2(vD, Dd));
    const float2 rho2 = fma2(pTi, Ti, mul2(vDi, Di));
    const float2 Pi = fma2(pT, Ti, mul2(vD, Di));
    const float2 eI2 = mul2(eI, eI);
    const float2 G = add2(eI2, rho2);
    const float2 Delta = fma2(eI2, sub2(G, E2), neg2(mul2(Pi, Pi)));
    const float2 f = mul2(f2(muS1), rcp2(Delta));
    const float2 A = fma2(eI2, T, mul2(Ti, Pi));
    const float2 C = fma2(Dd, Ti, neg2(mul2(T, Di)));
    // Q, U, V = -f X: the residual o - (-f X) is formed by FMAs on o, with f
    // applied once to A and to eI C.  FILL scales the polarised model by
    // alpha and mixes the field-free I.
    const float2 fq = FILL ? mul2(f, f2(g.alpha)) : f;
    const float2 fqeI = mul2(fq, eI);
    const float2 fA = mul2(fq, A), fC = mul2(fqeI, C);
    // the observed pair, read here rather than held through the evaluations
    const float4 o0 = lds4((const float4 *)op), o1 = lds4((const float4 *)(op + 4));
    const Stokes4x2 o = {make_float2(o0.x, o0.y), make_float2(o0.z, o0.w), make_float2(o1.x, o1.y),
                         make_float2(o1.z, o1.w)};
    Stokes4x2 r;
    if (FILL) {
        const float2 inm = mul2(f2(muS1), rcp2(fma2(f2(2.0f * g.eta0), P0, f2(1.0f))));
        const float2 base = fma2(f2(1.0f - g.alpha), inm, f2(S0));
        r.I = sub2(o.I, fma2(fqeI, G, base));
    } else {
        r.I = sub2(o.I, fma2(fqeI, G, f2(S0)));
    }
    r.Q = fma2(f2(kQ), fA, fma2(f2(kUV), fC, o.Q));
    r.U = fma2(f2(kU), fA, fma2(f2(-kQV), fC, o.U));
    r.V = fma2(mul2(fq, f2(kV)), fma2(eI2, Dd, mul2(Di, Pi)), o.V);
    return r;
}

}  // namespace genesis
