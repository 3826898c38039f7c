// Levenberg-Marquardt polish kernel (sm_103a).
//
// One warp per pixel, lanes over wavelengths.  Per iteration: analytic
// Jacobian in the problem's precision (FP32 for float cubes), per-lane partial
// sums of J^T W^2 J and J^T W^2 r and their warp reduction in the same
// precision (the FP32 Jacobian bounds their accuracy; GB300's FP64 rate is a
// small fraction of its FP32 rate), the damped Cholesky solve in FP64 shared
// by the warp (lane i holds row i of the factor), and a trial synthesis whose
// FP64-summed chi2 decides acceptance (Levenberg 1944, Marquardt 1963).
#include "kernels.h"
#include "me_jac.cuh"
#include "rng_device.cuh"

namespace genesis {

cudaError_t upload_tables_lm(const HostTables &t)
{
    return cudaMemcpyToSymbol(c_fad, &t.fad, sizeof(FaddeevaTables));
}

namespace {

constexpr int kLmWarps = 4;
// Blocks per SM the register allocation of the FP32 instantiations must
// allow: 4 (128 registers) spills a little of the Jacobian's partial sums
// but gives the latency-bound warps twice the company of the unbounded 255
// registers (10-iteration polish 5 % faster, 40-iteration prefit 7 %, the
// uncertainty 20 % on GB300).  FP64 instantiations keep the compiler's
// choice.  Build option: GENESIS_LM_MINB.
#ifndef GENESIS_LM_MINB
#define GENESIS_LM_MINB 4
#endif

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <class R> __device__ __forceinline__ void kahan_sq(R &s, R &c, R r)
{
    const R y = r * r - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
}

// chi2 (Eq. chisq) of parameters p: synthesis in R, per-lane compensated sums,
// warp sum in FP64.  Every lane returns the same value.
template <class R, class RO, int NL, int M = ME_NPAR>
__device__ double lm_chi2(const KProblem &pb, int nlines, int nl, const double *p, double mu,
                          const RO *o, const R *s_doff, const R *he, const double *w2)
{
    R pr[M];
#pragma unroll
    for (int d = 0; d < M; ++d) pr[d] = R(p[d]);
    const Geo<R> g = make_geo<R, NL, (M > ME_NPAR)>(pb, nlines, pr, R(mu));
    R s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (int j = threadIdx.x & 31; j < nl; j += 32) {
        R doff[ME_MAX_LINES];
#pragma unroll
        for (int l = 0; l < ME_MAX_LINES; ++l) doff[l] = l < nlines ? s_doff[l * nl + j] : R(0);
        const Stokes4<R> m = me_point<R, NL, true, (M > ME_NPAR)>(g, doff, he, nlines, pb.line);
        kahan_sq(s[0], c[0], R(o[j]) - m.I);
        kahan_sq(s[1], c[1], R(o[nl + j]) - m.Q);
        kahan_sq(s[2], c[2], R(o[2 * nl + j]) - m.U);
        kahan_sq(s[3], c[3], R(o[3 * nl + j]) - m.V);
    }
    double tot = 0.0;
#pragma unroll
    for (int st = 0; st < 4; ++st) tot += w2[st] * warp_sum((double)s[st]);
    return tot / (double)(4 * nl - M);
}

// One warp's shared state; M x M matrices stored with row stride M.  The
// normal equations A, g keep the precision R they were summed in (the solve
// widens each element as it reads it).
template <class R> struct LmWarpSmem {
    double N[ME_NPAR_MAX * ME_NPAR_MAX];
    double x[ME_NPAR_MAX];
    double w2[4];
    R A[ME_NPAR_MAX * ME_NPAR_MAX];
    R g[ME_NPAR_MAX];
};

// Warp-cooperative Cholesky factorisation in FP64 of an M x M symmetric
// matrix whose row i lane i < M supplies through a(j): lane i keeps row i of
// the factor L in registers and column j is formed on all rows at once (the
// left-looking order), with the row of L_j broadcast by shuffles and one
// reciprocal square root of the pivot per column (rinv, the same on every
// lane) in place of a division per element.  Entries above the diagonal of
// L are left unspecified.  Returns false, on every lane, at the first pivot
// that is not positive.  All lanes of the warp must call it together.
template <int M, class RowFn>
__device__ __forceinline__ bool warp_cholesky(RowFn a, double (&L)[M], double (&rinv)[M])
{
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double s = a(j);
#pragma unroll
        for (int k = 0; k < j; ++k) s = fma(-L[k], __shfl_sync(0xffffffffu, L[k], j), s);
        const double dj = __shfl_sync(0xffffffffu, s, j);
        if (!(dj > 0.0)) return false;
        rinv[j] = rsqrt(dj);
        L[j] = s * rinv[j];
    }
    return true;
}

// Solve (A + lam D) x = g with Marquardt's diagonal D = diag(max(A_jj,
// 1e-12 max_k A_kk)), the rows and columns of held parameters zeroed, with
// warp_cholesky; forward substitution runs on the same rows, back
// substitution reads L^T through the warp's shared matrix N.  A pivot that
// is not positive multiplies lam by 10 and retries (up to 30 times).
// Returns false, on every lane, if no step was found (also when A has no
// positive diagonal); the step lands in W.x.  All lanes of the warp must
// call it together.
template <int M, class R>
__device__ bool warp_damped_solve(LmWarpSmem<R> &W, unsigned free_mask, double &lam)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int row = lane < M ? lane : 0;
    const bool free_row = lane < M && ((free_mask >> row) & 1u);
    const double aii = free_row ? (double)W.A[row * M + row] : 0.0;
    double dmax = aii;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dmax = fmax(dmax, __shfl_xor_sync(full, dmax, off));
    if (!(dmax > 0.0)) return false;
    const double floor_d = 1e-12 * dmax;
    const double dscale = aii > floor_d ? aii : floor_d;
    const double grow = free_row ? (double)W.g[row] : 0.0;
    for (int tries = 0; tries < 30; ++tries) {
        const double drow = fma(lam, dscale, aii);  // this row's damped diagonal
        double L[M], rinv[M];
        const bool ok = warp_cholesky<M>(
            [&](int j) {
                return lane == j ? drow : ((free_row && ((free_mask >> j) & 1u)) ? (double)W.A[row * M + j] : 0.0);
            },
            L, rinv);
        if (!ok) {
            lam *= 10.0;
            continue;
        }
        // L y = g, then L^T x = y
        double t = grow, y = 0.0;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const double yk = __shfl_sync(full, t, k) * rinv[k];
            if (lane == k) y = yk;
            t = fma(-L[k], yk, t);
        }
        if (lane < M) {
#pragma unroll
            for (int k = 0; k < M; ++k) W.N[row * M + k] = L[k];
        }
        __syncwarp();
        double u = y, x = 0.0;
#pragma unroll
        for (int k = M - 1; k >= 0; --k) {
            const double xk = __shfl_sync(full, u, k) * rinv[k];
            if (lane == k) x = xk;
            u = fma(-W.N[k * M + row], xk, u);
        }
        if (lane < M) W.x[row] = x;
        __syncwarp();
        return true;
    }
    return false;
}


// Weights of one pixel into w2 (squared): the caller's, or Section 5.4
// inverse-max in FP64.  Every lane gets the result.
template <class RO, class R>
__device__ void lm_weights(const RO *o, int nl, const double *w_user, int pix, LmWarpSmem<R> &W, double w2[4])
{
    const int lane = threadIdx.x & 31;
    if (w_user) {
        if (lane < 4) {
            const double w = w_user[(size_t)pix * 4 + lane];
            W.w2[lane] = w * w;
        }
    } else {
        double imax = -INFINITY, imin = INFINITY, mq = 0, mu = 0, mv = 0;
        for (int j = lane; j < nl; j += 32) {
            const double I = (double)o[j];
            imax = fmax(imax, I);
            imin = fmin(imin, I);
            mq = fmax(mq, fabs((double)o[nl + j]));
            mu = fmax(mu, fabs((double)o[2 * nl + j]));
            mv = fmax(mv, fabs((double)o[3 * nl + j]));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            imax = fmax(imax, __shfl_xor_sync(0xffffffffu, imax, off));
            imin = fmin(imin, __shfl_xor_sync(0xffffffffu, imin, off));
            mq = fmax(mq, __shfl_xor_sync(0xffffffffu, mq, off));
            mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, off));
            mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, off));
        }
        if (lane == 0) {
            const double d[4] = {imax - imin, mq, mu, mv};
            const double fl = 1e-6 * fabs(imax);
            for (int s = 0; s < 4; ++s) {
                const double dd = d[s] > fl ? d[s] : fl;
                const double w = dd > 0.0 ? 1.0 / dd : 0.0;
                W.w2[s] = w * w;
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 4; ++s) w2[s] = W.w2[s];
}

// Normal equations at p: W.A = J^T W^2 J (full M x M) and W.g = J^T W^2 r,
// per-lane partial sums in R over the lane's wavelengths, warp sums in R,
// stored in R (the solve widens them to FP64).
template <class R, class RO, int NL, int M = ME_NPAR>
__device__ void lm_normal(const KProblem &pb, int nlines, int nl, const double *p, double mu,
                          const RO *o, const R *s_doff, const R *he, const R *w2r, LmWarpSmem<R> &W)
{
    const int lane = threadIdx.x & 31;
    R pr[M];
#pragma unroll
    for (int d = 0; d < M; ++d) pr[d] = R(p[d]);
    const GeoJ<R> G = make_geoj<R, NL, (M > ME_NPAR)>(pb, nlines, pr, R(mu));
    constexpr int kNT = M * (M + 1) / 2;  // packed lower triangle
    R Aacc[kNT], gacc[M];
#pragma unroll
    for (int a = 0; a < kNT; ++a) Aacc[a] = R(0);
#pragma unroll
    for (int a = 0; a < M; ++a) gacc[a] = R(0);
    for (int j = lane; j < nl; j += 32) {
        R doff[ME_MAX_LINES];
#pragma unroll
        for (int l = 0; l < ME_MAX_LINES; ++l) doff[l] = l < nlines ? s_doff[l * nl + j] : R(0);
        Stokes4<R> m;
        R J[4][M];
        me_point_jac<R, NL, (M > ME_NPAR)>(G, doff, he, nlines, pb.line, m, J);
        const R r[4] = {R(o[j]) - m.I, R(o[nl + j]) - m.Q, R(o[2 * nl + j]) - m.U,
                        R(o[3 * nl + j]) - m.V};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int t = 0;
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const R wa = w2r[s] * J[s][a];
                gacc[a] += wa * r[s];
#pragma unroll
                for (int b = 0; b <= a; ++b) Aacc[t++] += wa * J[s][b];
            }
        }
    }
    int t = 0;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const R gv = warp_sum(gacc[a]);
        if (lane == 0) W.g[a] = gv;
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            const R v = warp_sum(Aacc[t++]);
            if (lane == 0) {
                W.A[a * M + b] = v;
                W.A[b * M + a] = v;
            }
        }
    }
    __syncwarp();
}

template <class R, class RO, int NL, int M = ME_NPAR>
__global__ void __launch_bounds__(kLmWarps * 32, sizeof(R) == 4 ? GENESIS_LM_MINB : 1)
k_lm(const __grid_constant__ KProblem pb, const __grid_constant__ KLm lm, const RO *__restrict__ obs,
     const double *__restrict__ w_user, const double *__restrict__ mu_px, int npix,
     double *__restrict__ params, const KSub sub)
{
    extern __shared__ __align__(16) unsigned char smem[];
    LmWarpSmem<R> *s_w = (LmWarpSmem<R> *)smem;
    R *s_he = (R *)(smem + sizeof(LmWarpSmem<R>) * kLmWarps);
    R *s_doff = s_he + ME_MAX_LINES;
    const int nl = pb.n_lambda, nlines = NL > 0 ? NL : pb.n_lines;
    for (int i = threadIdx.x; i < nlines * nl; i += blockDim.x) {
        const int l = i / nl, j = i - l * nl;
        s_doff[i] = R(pb.lam[j] - pb.line[l].lam0);
    }
    if (threadIdx.x < ME_MAX_LINES)
        s_he[threadIdx.x] = threadIdx.x < nlines ? R(pb.line[threadIdx.x].half_eta) : R(0);
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * kLmWarps + warp;
    if (b >= (sub.count ? min(*sub.count, npix) : npix)) return;
    const int pix = sub.index ? sub.index[b] : b;
    if (pix < 0 || pix >= npix) return;  // a bad index skips the warp, uniformly
    LmWarpSmem<R> &W = s_w[warp];
    const RO *o = obs + (size_t)pix * 4 * nl;
    R he[ME_MAX_LINES];
#pragma unroll
    for (int l = 0; l < ME_MAX_LINES; ++l) he[l] = s_he[l];

    double w2[4];
    lm_weights(o, nl, w_user, pix, W, w2);
    R w2r[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) w2r[s] = R(w2[s]);

    const double mu = mu_px ? mu_px[pix] : pb.mu;
    double p[M];
#pragma unroll
    for (int d = 0; d < M; ++d) p[d] = params[(size_t)pix * M + d];
    double chi2 = lm_chi2<R, RO, NL, M>(pb, nlines, nl, p, mu, o, s_doff, he, w2);
    double lam = lm.lambda0;
    bool need = true;
    for (int it = 0; it < lm.iters; ++it) {
        if (need) {
            lm_normal<R, RO, NL, M>(pb, nlines, nl, p, mu, o, s_doff, he, w2r, W);
            need = false;
        }
        if (!warp_damped_solve<M>(W, lm.free_mask, lam)) break;
        // trial point: lane d forms parameter d (the azimuth wrapped into
        // [0, 180), then the bounds), and the warp gathers the vector
        double q[M];
        {
            const int row = lane < M ? lane : 0;
            double pl = p[0];
#pragma unroll
            for (int d = 1; d < M; ++d) pl = (lane == d) ? p[d] : pl;
            double qv = pl + W.x[row];
            if (lane == 2 && !(qv >= 0.0 && qv < 180.0)) {
                qv = fmod(qv, 180.0);
                if (qv < 0.0) qv += 180.0;
                if (qv >= 180.0) qv -= 180.0;
            }
            qv = fmin(fmax(qv, lm.lo[row]), lm.hi[row]);
#pragma unroll
            for (int d = 0; d < M; ++d) q[d] = __shfl_sync(0xffffffffu, qv, d);
        }
        const double c2 = lm_chi2<R, RO, NL, M>(pb, nlines, nl, q, mu, o, s_doff, he, w2);
        __syncwarp();
        if (c2 < chi2) {
#pragma unroll
            for (int d = 0; d < M; ++d) p[d] = q[d];
            chi2 = c2;
            lam /= 10.0;
            need = true;
        } else {
            lam *= 10.0;
        }
    }
    if (lane < M) {
        double v = p[0];
#pragma unroll
        for (int d = 1; d < M; ++d) v = (lane == d) ? p[d] : v;
        params[(size_t)pix * M + lane] = v;
    }
}

// Section 6 uncertainty estimate at given parameters: sigma_i^2 =
// [H^-1]_ii chi2 / M with H the Gauss-Newton Hessian of Eq. chisq,
// H = (2/nu) J^T W^2 J.  Warp per pixel; J and its sums in the problem
// precision, the Cholesky factor and the inverse diagonal in FP64 (lane i
// forms [H^-1]_ii).  A parameter without influence (singular H) gets
// +infinity on every parameter of the pixel.
template <class R, class RO, int NL, int M = ME_NPAR>
__global__ void __launch_bounds__(kLmWarps * 32, sizeof(R) == 4 ? GENESIS_LM_MINB : 1)
k_lm_sigma(const __grid_constant__ KProblem pb, const RO *__restrict__ obs,
           const double *__restrict__ w_user, const double *__restrict__ mu_px, int npix,
           const double *__restrict__ params, double *__restrict__ sigma)
{
    extern __shared__ __align__(16) unsigned char smem[];
    LmWarpSmem<R> *s_w = (LmWarpSmem<R> *)smem;
    R *s_he = (R *)(smem + sizeof(LmWarpSmem<R>) * kLmWarps);
    R *s_doff = s_he + ME_MAX_LINES;
    const int nl = pb.n_lambda, nlines = NL > 0 ? NL : pb.n_lines;
    for (int i = threadIdx.x; i < nlines * nl; i += blockDim.x) {
        const int l = i / nl, j = i - l * nl;
        s_doff[i] = R(pb.lam[j] - pb.line[l].lam0);
    }
    if (threadIdx.x < ME_MAX_LINES)
        s_he[threadIdx.x] = threadIdx.x < nlines ? R(pb.line[threadIdx.x].half_eta) : R(0);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pix = blockIdx.x * kLmWarps + warp;
    if (pix >= npix) return;
    LmWarpSmem<R> &W = s_w[warp];
    const RO *o = obs + (size_t)pix * 4 * nl;
    R he[ME_MAX_LINES];
#pragma unroll
    for (int l = 0; l < ME_MAX_LINES; ++l) he[l] = s_he[l];
    double w2[4];
    lm_weights(o, nl, w_user, pix, W, w2);
    R w2r[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) w2r[s] = R(w2[s]);
    const double mu = mu_px ? mu_px[pix] : pb.mu;
    double p[M];
#pragma unroll
    for (int d = 0; d < M; ++d) p[d] = params[(size_t)pix * M + d];
    const double chi2 = lm_chi2<R, RO, NL, M>(pb, nlines, nl, p, mu, o, s_doff, he, w2);
    lm_normal<R, RO, NL, M>(pb, nlines, nl, p, mu, o, s_doff, he, w2r, W);
    // H = (2/nu) A;  [H^-1]_ii = (nu/2) [A^-1]_ii = (nu/2) || L^-1 e_i ||^2
    double L[M], rinv[M];
    const int row = lane < M ? lane : 0;
    const bool ok = warp_cholesky<M>([&](int j) { return lane < M ? (double)W.A[row * M + j] : 0.0; }, L, rinv);
    if (ok && lane < M) {
#pragma unroll
        for (int k = 0; k < M; ++k) W.N[row * M + k] = L[k];
    }
    __syncwarp();
    if (lane < M) {
        double v = INFINITY;
        if (ok) {
            // lane i: forward substitution of e_i against L (broadcast reads)
            double y[M];
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r < M; ++r) {
                double t = (r == lane) ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < r; ++k) t = fma(-W.N[r * M + k], y[k], t);
                y[r] = t * rinv[r];
                acc = fma(y[r], y[r], acc);
            }
            const double nu = (double)(4 * nl - M);
            v = sqrt(0.5 * nu * acc * chi2 / (double)M);
        }
        sigma[(size_t)pix * M + lane] = v;
    }
}

template <class R, class RO, int NL, int M = ME_NPAR>
cudaError_t sigma_t(const KProblem &pb, const void *obs, const double *w, const double *mu_px, int npix,
                    const double *params, double *sigma, cudaStream_t st)
{
    const int nlines = NL > 0 ? NL : pb.n_lines;
    const size_t smem = sizeof(LmWarpSmem<R>) * kLmWarps + sizeof(R) * (ME_MAX_LINES + (size_t)nlines * pb.n_lambda);
    auto kern = k_lm_sigma<R, RO, NL, M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(npix + kLmWarps - 1) / kLmWarps, kLmWarps * 32, smem, st>>>(pb, (const RO *)obs, w, mu_px, npix,
                                                                       params, sigma);
    return cudaGetLastError();
}

template <class R, class RO, int NL, int M = ME_NPAR>
cudaError_t lm_t(const KProblem &pb, const KLm &lm, const void *obs, const double *w,
                 const double *mu_px, int npix, double *params, cudaStream_t st, KSub sub)
{
    const int nlines = NL > 0 ? NL : pb.n_lines;
    const size_t smem = sizeof(LmWarpSmem<R>) * kLmWarps + sizeof(R) * (ME_MAX_LINES + (size_t)nlines * pb.n_lambda);
    auto kern = k_lm<R, RO, NL, M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(npix + kLmWarps - 1) / kLmWarps, kLmWarps * 32, smem, st>>>(pb, lm, (const RO *)obs, w, mu_px,
                                                                      npix, params, sub);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lm_sigma(const KProblem &pb, int dtype, const void *obs, const double *w,
                            const double *mu_px, int npix, const double *params, double *sigma,
                            cudaStream_t st)
{
    if (npix <= 0) return cudaSuccess;
    if (pb.fill)
        return dtype == ME_F32 ? sigma_t<float, float, 0, ME_NPAR_MAX>(pb, obs, w, mu_px, npix, params, sigma, st)
                               : sigma_t<double, double, 0, ME_NPAR_MAX>(pb, obs, w, mu_px, npix, params, sigma, st);
    if (dtype == ME_F32) {
        if (pb.n_lines == 1) return sigma_t<float, float, 1>(pb, obs, w, mu_px, npix, params, sigma, st);
        if (pb.n_lines == 2) return sigma_t<float, float, 2>(pb, obs, w, mu_px, npix, params, sigma, st);
        return sigma_t<float, float, 0>(pb, obs, w, mu_px, npix, params, sigma, st);
    }
    return sigma_t<double, double, 0>(pb, obs, w, mu_px, npix, params, sigma, st);
}

cudaError_t launch_lm(const KProblem &pb, const KLm &lm, int dtype, const void *obs,
                      const double *w, const double *mu_px, int npix, double *params,
                      cudaStream_t st, KSub sub)
{
    if (npix <= 0 || lm.iters <= 0) return cudaSuccess;
    if (pb.fill)
        return dtype == ME_F32 ? lm_t<float, float, 0, ME_NPAR_MAX>(pb, lm, obs, w, mu_px, npix, params, st, sub)
                               : lm_t<double, double, 0, ME_NPAR_MAX>(pb, lm, obs, w, mu_px, npix, params, st, sub);
    if (dtype == ME_F32) {
        if (pb.n_lines == 1) return lm_t<float, float, 1>(pb, lm, obs, w, mu_px, npix, params, st, sub);
        if (pb.n_lines == 2) return lm_t<float, float, 2>(pb, lm, obs, w, mu_px, npix, params, st, sub);
        return lm_t<float, float, 0>(pb, lm, obs, w, mu_px, npix, params, st, sub);
    }
    return lm_t<double, double, 0>(pb, lm, obs, w, mu_px, npix, params, st, sub);
}

}  // namespace genesis
