// Analytic Jacobian of the Milne-Eddington Stokes vector (sm_103a).
//
// Differentiates Section 5's solution S0 e + mu S1 K^-1 e through the closed
// form of K^-1 e, the propagation-matrix elements and the Faddeeva profiles,
// using w'(z) = -2 z w(z) + 2 i / sqrt(pi) and dw/da = i w'(z).
#pragma once

#include "me_device.cuh"

namespace genesis {

template <class R> struct GeoJ {
    Geo<R> g;
    R eta0, invDpar;                 // eta0, 1 / (param 4)
    R uIp, uIs, uQ, uU, uV;          // kIp..kV per unit eta0
    R dIp_th, dIs_th, dQ_th, dU_th, dV_th;  // d k / d theta [per deg]
    R dQ_ch, dU_ch;                         // d k / d chi [per deg]
    R mu;
    R kv[ME_MAX_LINES];              // d x / d v_LOS = -kv (lambda0 / c / Doppler width)
    R kB[ME_MAX_LINES];              // d v_B / d B
    R kL[ME_MAX_LINES];              // d v_L / d B (Larmor displacement, full patterns)
};

template <class R, int NL, bool FILL = false>
__device__ __forceinline__ GeoJ<R> make_geoj(const KProblem &pb, int nlines, const R *p, R mu)
{
    GeoJ<R> G;
    G.g = make_geo<R, NL, FILL>(pb, nlines, p, mu);
    R st, ct, s2c, c2c;
    sincos_deg(p[1], &st, &ct);
    sincos_deg(R(2) * p[2], &s2c, &c2c);
    const R eta0 = p[6], s2 = st * st, kd = R(kDeg);
    G.eta0 = eta0;
    G.invDpar = R(1) / p[4];
    G.uIp = s2;
    G.uIs = R(0.5) * (R(1) + ct * ct);
    G.uQ = s2 * c2c;
    G.uU = s2 * s2c;
    G.uV = ct;
    const R ds2 = R(2) * st * ct * kd;    // d sin^2 / d theta
    G.dIp_th = eta0 * ds2;
    G.dIs_th = -eta0 * st * ct * kd;
    G.dQ_th = eta0 * ds2 * c2c;
    G.dU_th = eta0 * ds2 * s2c;
    G.dV_th = -eta0 * st * kd;
    G.dQ_ch = -eta0 * s2 * R(2) * s2c * kd;
    G.dU_ch = eta0 * s2 * R(2) * c2c * kd;
    G.mu = mu;
    const int nl = NL > 0 ? NL : nlines;
#pragma unroll
    for (int l = 0; l < (NL > 0 ? NL : ME_MAX_LINES); ++l) {
        if (l < nl) {
            G.kv[l] = R(pb.line[l].lam0_c) * G.g.invD[l];
            G.kB[l] = R(pb.line[l].zfac) * G.g.invD[l];
            G.kL[l] = R(pb.line[l].zfacL) * G.g.invD[l];
        }
    }
    return G;
}

// Profile sums per unit eta0 and their derivatives along B, v_LOS, D, a.
template <class R> struct Sums {
    R P, Sg, T, Ti, Dd, Di;
    R dP[4], dSg[4], dT[4], dTi[4], dDd[4], dDi[4];
};

// Near a line core the sigma-minus-pi combinations of a weakly split
// effective triplet, T = w(v) - (w(v + d) + w(v - d)) / 2 and its
// derivatives, lose their relative precision to cancellation in FP32 (about
// 1e-7 / d^2 at d = v_B).  There they are formed instead from Taylor series
// in d about the pi point z = v + i a:
//   h  = (w(v+d) + w(v-d)) / 2 - w(v)    = sum_k d^2k / (2k)! w^(2k)(z),
//   hp = (w'(v+d) + w'(v-d)) / 2 - w'(v) = sum_k d^2k / (2k)! w^(2k+1)(z),
//   g1 = (w'(v+d) - w'(v-d)) / 2         = sum_k d^(2k-1) / (2k-1)! w^(2k)(z),
// k = 1..5, with the derivatives of w from w^(n+1) = -2 z w^(n) - 2 n w^(n-1)
// (the derivative of w' = -2 z w + 2i/sqrt(pi)).  The caller takes this form
// for |d| <= 0.25 and |z|^2 <= 16, and for |d| <= 0.1 and |z|^2 <= 36: there the
// recurrence loses at most a factor 2 |z|^2 / (n + 1) per step, which the
// factors d^m / m! absorb (w'' itself to about 6e-8 (2/3) |z|^4 relative), and
// the first omitted term is below 1e-8 of the sums.  w1 = w'(z).
template <class R>
__device__ __forceinline__ void split_series(R v, R a, R d, C2<R> w0, C2<R> w1, C2<R> &h, C2<R> &hp,
                                             C2<R> &g1)
{
    C2<R> wm = w0, wc = w1;  // w^(n-1), w^(n)
    R c = d;                 // d^n / n!
    h = hp = g1 = C2<R>{R(0), R(0)};
#pragma unroll
    for (int n = 1; n <= 10; ++n) {
        const C2<R> wn = {R(-2) * (v * wc.x - a * wc.y) - R(2 * n) * wm.x,
                          R(-2) * (v * wc.y + a * wc.x) - R(2 * n) * wm.y};  // w^(n+1)
        const R cn = c * d * R(1.0 / (n + 1));                                // d^(n+1) / (n+1)!
        if ((n + 1) % 2 == 0) {
            h.x += cn * wn.x;
            h.y += cn * wn.y;
            g1.x += c * wn.x;
            g1.y += c * wn.y;
        } else {
            hp.x += c * wn.x;
            hp.y += c * wn.y;
        }
        wm = wc;
        wc = wn;
        c = cn;
    }
}

// Stokes vector and J[s][k] = d Stokes_s / d p_k at one wavelength.
// FILL: Section 5.2 fill fraction, p[9] = alpha, J has a 10th column.
template <class R, int NL, bool FILL = false>
__device__ __forceinline__ void me_point_jac(const GeoJ<R> &G, const R *doff, const R *half_eta,
                                             int nlines, const KLine *lines, Stokes4<R> &out,
                                             R J[4][ME_NPAR + (FILL ? 1 : 0)])
{
    const Geo<R> &g = G.g;
    Sums<R> S;
    S.P = S.Sg = S.T = S.Ti = S.Dd = S.Di = R(0);
#pragma unroll
    for (int d = 0; d < 4; ++d) S.dP[d] = S.dSg[d] = S.dT[d] = S.dTi[d] = S.dDd[d] = S.dDi[d] = R(0);
    // field-free profile sum P0 = sum (eta_ratio / 2) Re w0 and its
    // derivatives along v_LOS, D, a (FILL only)
    R P0 = R(0), dP0[4] = {R(0), R(0), R(0), R(0)};
    const R two_isp = R(1.12837916709551257390);  // 2 / sqrt(pi)
    const int nl = NL > 0 ? NL : nlines;
#pragma unroll
    for (int l = 0; l < (NL > 0 ? NL : ME_MAX_LINES); ++l) {
        if (l < nl) {
            const R q = half_eta[l];
            C2<R> w[3], wd[3][4];
            const R sv = -G.kv[l];
            // T + i Ti of this line and its derivatives, when the series form applies
            C2<R> tc{R(0), R(0)}, dtc[4];
            bool series = false;
            if (lines[l].ncomp[0] == 0) {
                const R xs[3] = {doff[l] * g.invD[l] + (g.cp[l] + g.vB[l]),  // blue
                                 doff[l] * g.invD[l] + g.cp[l],              // pi
                                 doff[l] * g.invD[l] + (g.cp[l] - g.vB[l])}; // red
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    w[c] = faddeeva<R>(xs[c], g.a);
                    // w' = -2 z w + 2i/sqrt(pi)
                    const R dx = R(-2) * (xs[c] * w[c].x - g.a * w[c].y);
                    const R dy = R(-2) * (xs[c] * w[c].y + g.a * w[c].x) + two_isp;
                    const R sB = c == 0 ? G.kB[l] : (c == 2 ? -G.kB[l] : R(0));
                    const R sD = -xs[c] * G.invDpar;
                    wd[c][0] = {dx * sB, dy * sB};   // d/dB
                    wd[c][1] = {dx * sv, dy * sv};   // d/dv_LOS
                    wd[c][2] = {dx * sD, dy * sD};   // d/dD
                    wd[c][3] = {-dy, dx};            // d/da = i w'
                }
                if constexpr (sizeof(R) == 4) {
                    // a weakly split triplet near its core: T and its
                    // derivatives without the cancellation of the three
                    // profiles (split_series)
                    const R v = xs[1], d = g.vB[l], ad = fabs(d), r2 = v * v + g.a2;
                    if ((ad <= R(0.25) && r2 <= R(16)) || (ad <= R(0.1) && r2 <= FadCfg<R>::R2)) {
                        C2<R> h, hp, g1;
                        split_series<R>(v, g.a, d, w[1], C2<R>{wd[1][3].y, -wd[1][3].x}, h, hp, g1);
                        tc = C2<R>{-h.x, -h.y};
                        dtc[0] = C2<R>{-G.kB[l] * g1.x, -G.kB[l] * g1.y};               // d/dB
                        dtc[1] = C2<R>{-sv * hp.x, -sv * hp.y};                         // d/dv_LOS
                        dtc[2] = C2<R>{G.invDpar * (v * hp.x + d * g1.x),
                                       G.invDpar * (v * hp.y + d * g1.y)};              // d/dD
                        dtc[3] = C2<R>{hp.y, -hp.x};                                    // d/da
                        series = true;
                    }
                }
                if (FILL) {  // the pi component is unshifted
                    P0 += q * w[1].x;
#pragma unroll
                    for (int d = 1; d < 4; ++d) dP0[d] += q * wd[1][d].x;
                }
            } else {
                // full pattern: strength-weighted sums over each group's
                // components x_i = doff/D + cp - v_L s_i, dx_i/dB = -s_i k_L
                const R dinv = doff[l] * g.invD[l];
                for (int c = 0; c < 3; ++c) {
                    w[c] = {R(0), R(0)};
                    for (int d = 0; d < 4; ++d) wd[c][d] = {R(0), R(0)};
                    for (int i = 0; i < lines[l].ncomp[c]; ++i) {
                        const R sh = comp_shift<R>(lines[l], c, i), st = comp_str<R>(lines[l], c, i);
                        const R x = dinv + (g.cp[l] - g.vL[l] * sh);
                        const C2<R> wi = faddeeva<R>(x, g.a);
                        const R dx = R(-2) * (x * wi.x - g.a * wi.y);
                        const R dy = R(-2) * (x * wi.y + g.a * wi.x) + two_isp;
                        const R sB = -sh * G.kL[l], sD = -x * G.invDpar;
                        w[c].x += st * wi.x;
                        w[c].y += st * wi.y;
                        wd[c][0].x += st * dx * sB;
                        wd[c][0].y += st * dy * sB;
                        wd[c][1].x += st * dx * sv;
                        wd[c][1].y += st * dy * sv;
                        wd[c][2].x += st * dx * sD;
                        wd[c][2].y += st * dy * sD;
                        wd[c][3].x -= st * dy;
                        wd[c][3].y += st * dx;
                    }
                }
                if (FILL) {  // the field-free profile needs its own, unshifted evaluation
                    const R x = dinv + g.cp[l];
                    const C2<R> w0 = faddeeva<R>(x, g.a);
                    const R dx = R(-2) * (x * w0.x - g.a * w0.y);
                    const R dy = R(-2) * (x * w0.y + g.a * w0.x) + two_isp;
                    P0 += q * w0.x;
                    dP0[1] += q * dx * sv;
                    dP0[2] += q * dx * (-x * G.invDpar);
                    dP0[3] -= q * dy;
                }
            }
            const R sx = w[0].x + w[2].x, sy = w[0].y + w[2].y;
            S.P += q * w[1].x;
            S.Sg += q * sx;
            S.T += q * (series ? tc.x : w[1].x - R(0.5) * sx);
            S.Ti += q * (series ? tc.y : w[1].y - R(0.5) * sy);
            S.Dd += q * (w[2].x - w[0].x);
            S.Di += q * (w[2].y - w[0].y);
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const R bx = wd[0][d].x + wd[2][d].x, by = wd[0][d].y + wd[2][d].y;
                S.dP[d] += q * wd[1][d].x;
                S.dSg[d] += q * bx;
                S.dT[d] += q * (series ? dtc[d].x : wd[1][d].x - R(0.5) * bx);
                S.dTi[d] += q * (series ? dtc[d].y : wd[1][d].y - R(0.5) * by);
                S.dDd[d] += q * (wd[2][d].x - wd[0][d].x);
                S.dDi[d] += q * (wd[2][d].y - wd[0][d].y);
            }
        }
    }
    // propagation-matrix elements e = (eI, eQ, eU, eV, rQ, rU, rV)
    const R eI = R(1) + g.kIp * S.P + g.kIs * S.Sg;
    const R eQ = g.kQ * S.T, eU = g.kU * S.T, eV = g.kV * S.Dd;
    const R rQ = g.kQ * S.Ti, rU = g.kU * S.Ti, rV = g.kV * S.Di;
    const R eI2 = eI * eI;
    const R rho2 = rQ * rQ + rU * rU + rV * rV;
    const R E2 = eQ * eQ + eU * eU + eV * eV;
    const R Pi = eQ * rQ + eU * rU + eV * rV;
    const R Delta = eI2 * (eI2 - E2 + rho2) - Pi * Pi;
    const R iD = R(1) / Delta;
    const R f = g.muS1 * iD;
    const R nI = eI * (eI2 + rho2);
    const R nQ = eI2 * eQ + eI * (eV * rU - eU * rV) + rQ * Pi;
    const R nU = eI2 * eU + eI * (eQ * rV - eV * rQ) + rU * Pi;
    const R nV = eI2 * eV + eI * (eU * rQ - eQ * rU) + rV * Pi;
    out.I = g.S0 + f * nI;
    out.Q = -f * nQ;
    out.U = -f * nU;
    out.V = -f * nV;

    // d Delta / d e
    const R dDe[7] = {R(2) * eI * (R(2) * eI2 - E2 + rho2),
                      R(-2) * (eI2 * eQ + Pi * rQ), R(-2) * (eI2 * eU + Pi * rU),
                      R(-2) * (eI2 * eV + Pi * rV),
                      R(2) * (eI2 * rQ - Pi * eQ), R(2) * (eI2 * rU - Pi * eU),
                      R(2) * (eI2 * rV - Pi * eV)};
    // d n_s / d e
    const R dnI[7] = {R(3) * eI2 + rho2, R(0), R(0), R(0), R(2) * eI * rQ, R(2) * eI * rU,
                      R(2) * eI * rV};
    const R dnQ[7] = {R(2) * eI * eQ + eV * rU - eU * rV, eI2 + rQ * rQ, -eI * rV + rQ * rU,
                      eI * rU + rQ * rV, Pi + rQ * eQ, eI * eV + rQ * eU, -eI * eU + rQ * eV};
    const R dnU[7] = {R(2) * eI * eU + eQ * rV - eV * rQ, eI * rV + rU * rQ, eI2 + rU * rU,
                      -eI * rQ + rU * rV, -eI * eV + rU * eQ, Pi + rU * eU, eI * eQ + rU * eV};
    const R dnV[7] = {R(2) * eI * eV + eU * rQ - eQ * rU, -eI * rU + rV * rQ, eI * rQ + rV * rU,
                      eI2 + rV * rV, eI * eU + rV * eQ, -eI * eQ + rV * eU, Pi + rV * eV};
    // G[s][e] = d Stokes_s / d e
    R Gm[4][7];
    const R xI = nI * iD, xQ = nQ * iD, xU = nU * iD, xV = nV * iD;
#pragma unroll
    for (int e = 0; e < 7; ++e) {
        Gm[0][e] = f * (dnI[e] - xI * dDe[e]);
        Gm[1][e] = -f * (dnQ[e] - xQ * dDe[e]);
        Gm[2][e] = -f * (dnU[e] - xU * dDe[e]);
        Gm[3][e] = -f * (dnV[e] - xV * dDe[e]);
    }
    // E[e] = d e / d p_k for k = 0..6, then J = G E
    const int dirs[4] = {0, 3, 4, 5};  // B, v_LOS, D, a
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        R E[7];
        E[0] = g.kIp * S.dP[d] + g.kIs * S.dSg[d];
        E[1] = g.kQ * S.dT[d];
        E[2] = g.kU * S.dT[d];
        E[3] = g.kV * S.dDd[d];
        E[4] = g.kQ * S.dTi[d];
        E[5] = g.kU * S.dTi[d];
        E[6] = g.kV * S.dDi[d];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            R acc = R(0);
#pragma unroll
            for (int e = 0; e < 7; ++e) acc += Gm[s][e] * E[e];
            J[s][dirs[d]] = acc;
        }
    }
    {   // theta
        R E[7];
        E[0] = G.dIp_th * S.P + G.dIs_th * S.Sg;
        E[1] = G.dQ_th * S.T;
        E[2] = G.dU_th * S.T;
        E[3] = G.dV_th * S.Dd;
        E[4] = G.dQ_th * S.Ti;
        E[5] = G.dU_th * S.Ti;
        E[6] = G.dV_th * S.Di;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            R acc = R(0);
#pragma unroll
            for (int e = 0; e < 7; ++e) acc += Gm[s][e] * E[e];
            J[s][1] = acc;
        }
    }
    {   // chi: only eQ, eU, rQ, rU depend on it
#pragma unroll
        for (int s = 0; s < 4; ++s)
            J[s][2] = Gm[s][1] * G.dQ_ch * S.T + Gm[s][2] * G.dU_ch * S.T +
                      Gm[s][4] * G.dQ_ch * S.Ti + Gm[s][5] * G.dU_ch * S.Ti;
    }
    {   // eta0
        R E[7];
        E[0] = G.uIp * S.P + G.uIs * S.Sg;
        E[1] = G.uQ * S.T;
        E[2] = G.uU * S.T;
        E[3] = G.uV * S.Dd;
        E[4] = G.uQ * S.Ti;
        E[5] = G.uU * S.Ti;
        E[6] = G.uV * S.Di;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            R acc = R(0);
#pragma unroll
            for (int e = 0; e < 7; ++e) acc += Gm[s][e] * E[e];
            J[s][6] = acc;
        }
    }
    // source function: d/dS0 = e, d/dS1 = mu K^-1 e
    J[0][7] = R(1);
    J[1][7] = J[2][7] = J[3][7] = R(0);
    J[0][8] = G.mu * xI;
    J[1][8] = -G.mu * xQ;
    J[2][8] = -G.mu * xU;
    J[3][8] = -G.mu * xV;
    if constexpr (FILL) {
        // Stokes = alpha S_mag + (1 - alpha) I_nm e, I_nm = S0 + mu S1 / eta_nm,
        // eta_nm = 1 + 2 eta0 P0
        const R inv = R(1) / (R(1) + R(2) * G.eta0 * P0);
        const R inm = g.muS1 * inv;
        const R c = -g.muS1 * inv * inv * R(2);  // d I_nm / d (eta0 P0)
        const R al = g.alpha, om = R(1) - g.alpha;
        R dnm[ME_NPAR] = {R(0), R(0), R(0), c * G.eta0 * dP0[1], c * G.eta0 * dP0[2], c * G.eta0 * dP0[3],
                          c * P0, R(1), G.mu * inv};
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int k = 0; k < ME_NPAR; ++k) J[s][k] = al * J[s][k] + (s == 0 ? om * dnm[k] : R(0));
        J[0][ME_NPAR] = (out.I - g.S0) - inm;  // I_mag - I_nm
        J[1][ME_NPAR] = out.Q;
        J[2][ME_NPAR] = out.U;
        J[3][ME_NPAR] = out.V;
        out.I = g.S0 + al * (out.I - g.S0) + om * inm;
        out.Q *= al;
        out.U *= al;
        out.V *= al;
    }
}

}  // namespace genesis
