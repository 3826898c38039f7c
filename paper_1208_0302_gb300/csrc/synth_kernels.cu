// Stokes synthesis, Jacobian, adjoint and FP64 chi-square kernels (sm_103a).
#include "kernels.h"
#include "me_jac.cuh"
#include "rng_device.cuh"

namespace genesis {

cudaError_t upload_tables_synth(const HostTables &t)
{
    return cudaMemcpyToSymbol(c_fad, &t.fad, sizeof(FaddeevaTables));
}

namespace {

constexpr int kSynthBlock = 128;

// Fill s_doff[l * nl + j] = lambda_j - lambda0_l for all lines (exact in FP64,
// rounded to R) and s_he[l] = eta_ratio_l / 2.
template <class R>
__device__ __forceinline__ void stage_offsets(const KProblem &pb, int nlines, R *s_doff, R *s_he)
{
    const int nl = pb.n_lambda;
    for (int i = threadIdx.x; i < nlines * nl; i += blockDim.x) {
        const int l = i / nl, j = i - l * nl;
        s_doff[i] = R(pb.lam[j] - pb.line[l].lam0);
    }
    if (threadIdx.x < ME_MAX_LINES)
        s_he[threadIdx.x] = threadIdx.x < nlines ? R(pb.line[threadIdx.x].half_eta) : R(0);
}

// One thread per (model, wavelength).
template <class R, int NL, bool FILL = false>
__global__ void __launch_bounds__(kSynthBlock)
k_synth(const __grid_constant__ KProblem pb, const double *__restrict__ params,
        const double *__restrict__ mu_px, int n, R *__restrict__ stokes)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nl = pb.n_lambda, nlines = NL > 0 ? NL : pb.n_lines;
    R *s_he = (R *)smem;
    R *s_doff = s_he + ME_MAX_LINES;
    stage_offsets<R>(pb, nlines, s_doff, s_he);
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * nl) return;
    const int m = (int)(i / nl), j = (int)(i - (long long)m * nl);
    constexpr int M = kNpar<FILL>;
    R p[M];
#pragma unroll
    for (int d = 0; d < M; ++d) p[d] = R(params[(size_t)m * M + d]);
    const R mu = mu_px ? R(mu_px[m]) : R(pb.mu);
    const Geo<R> g = make_geo<R, NL, FILL>(pb, nlines, p, mu);
    R doff[ME_MAX_LINES], he[ME_MAX_LINES];
#pragma unroll
    for (int l = 0; l < ME_MAX_LINES; ++l) {
        doff[l] = l < nlines ? s_doff[l * nl + j] : R(0);
        he[l] = s_he[l];
    }
    const Stokes4<R> s = me_point<R, NL, true, FILL>(g, doff, he, nlines, pb.line);
    R *o = stokes + (size_t)m * 4 * nl;
    o[j] = s.I;
    o[nl + j] = s.Q;
    o[2 * nl + j] = s.U;
    o[3 * nl + j] = s.V;
}

template <class R, int NL, bool FILL = false>
__global__ void __launch_bounds__(kSynthBlock)
k_jac(const __grid_constant__ KProblem pb, const double *__restrict__ params,
      const double *__restrict__ mu_px, int n, R *__restrict__ stokes, R *__restrict__ jac)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nl = pb.n_lambda, nlines = NL > 0 ? NL : pb.n_lines;
    R *s_he = (R *)smem;
    R *s_doff = s_he + ME_MAX_LINES;
    stage_offsets<R>(pb, nlines, s_doff, s_he);
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * nl) return;
    const int m = (int)(i / nl), j = (int)(i - (long long)m * nl);
    constexpr int M = kNpar<FILL>;
    R p[M];
#pragma unroll
    for (int d = 0; d < M; ++d) p[d] = R(params[(size_t)m * M + d]);
    const R mu = mu_px ? R(mu_px[m]) : R(pb.mu);
    const GeoJ<R> G = make_geoj<R, NL, FILL>(pb, nlines, p, mu);
    R doff[ME_MAX_LINES], he[ME_MAX_LINES];
#pragma unroll
    for (int l = 0; l < ME_MAX_LINES; ++l) {
        doff[l] = l < nlines ? s_doff[l * nl + j] : R(0);
        he[l] = s_he[l];
    }
    Stokes4<R> s;
    R J[4][M];
    me_point_jac<R, NL, FILL>(G, doff, he, nlines, pb.line, s, J);
    if (stokes) {
        R *o = stokes + (size_t)m * 4 * nl;
        o[j] = s.I;
        o[nl + j] = s.Q;
        o[2 * nl + j] = s.U;
        o[3 * nl + j] = s.V;
    }
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        R *o = jac + (((size_t)m * 4 + st) * nl + j) * M;
#pragma unroll
        for (int k = 0; k < M; ++k) o[k] = J[st][k];
    }
}

// One warp per model: grad_params[m] = sum_{s, j} J[s][j][:] * grad_stokes[m][s][j].
template <class R, int NL, bool FILL = false>
__global__ void __launch_bounds__(kSynthBlock)
k_vjp(const __grid_constant__ KProblem pb, const double *__restrict__ params,
      const double *__restrict__ mu_px, int n, const R *__restrict__ gs, double *__restrict__ gp)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nl = pb.n_lambda, nlines = NL > 0 ? NL : pb.n_lines;
    R *s_he = (R *)smem;
    R *s_doff = s_he + ME_MAX_LINES;
    stage_offsets<R>(pb, nlines, s_doff, s_he);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (m >= n) return;
    constexpr int M = kNpar<FILL>;
    R p[M];
#pragma unroll
    for (int d = 0; d < M; ++d) p[d] = R(params[(size_t)m * M + d]);
    const R mu = mu_px ? R(mu_px[m]) : R(pb.mu);
    const GeoJ<R> G = make_geoj<R, NL, FILL>(pb, nlines, p, mu);
    R he[ME_MAX_LINES];
#pragma unroll
    for (int l = 0; l < ME_MAX_LINES; ++l) he[l] = s_he[l];
    R acc[M];
#pragma unroll
    for (int k = 0; k < M; ++k) acc[k] = R(0);
    const R *g = gs + (size_t)m * 4 * nl;
    for (int j = lane; j < nl; j += 32) {
        R doff[ME_MAX_LINES];
#pragma unroll
        for (int l = 0; l < ME_MAX_LINES; ++l) doff[l] = l < nlines ? s_doff[l * nl + j] : R(0);
        Stokes4<R> s;
        R J[4][M];
        me_point_jac<R, NL, FILL>(G, doff, he, nlines, pb.line, s, J);
#pragma unroll
        for (int st = 0; st < 4; ++st) {
            const R gv = g[st * nl + j];
#pragma unroll
            for (int k = 0; k < M; ++k) acc[k] += J[st][k] * gv;
        }
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        double v = (double)acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) gp[(size_t)m * M + k] = v;
    }
}

// FP64 chi-square (Eq. chisq) of given parameters, one block per pixel,
// threads over wavelengths.  Inverse-max weights (Section 5.4) are formed in
// FP64 from the observed values when w is NULL.
// NL > 0 with PAT = false: problems with NL effective-triplet lines (the
// loops over lines unrolled, the full-pattern code compiled out; the same
// arithmetic in the same order as the generic form, 4.6 % faster on the
// two-line map, where the pass is bound by the FP64 pipe).
template <class RO, bool FILL = false, int NL = 0, bool PAT = true>
__global__ void __launch_bounds__(kSynthBlock)
k_chi2_f64(const __grid_constant__ KProblem pb, const RO *__restrict__ obs,
           const double *__restrict__ w_user, const double *__restrict__ mu_px, int npix,
           const double *__restrict__ params, double *__restrict__ chi2, const KSub sub)
{
    __shared__ double s_red[kSynthBlock / 32][4];
    __shared__ double s_w2[4];
    const int nl = pb.n_lambda, nlines = pb.n_lines;
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (sub.count && b >= *sub.count) return;
    const int pix = sub.index ? sub.index[b] : b;
    if (pix < 0 || pix >= npix) return;
    const RO *o = obs + (size_t)pix * 4 * nl;
    if (w_user) {
        if (threadIdx.x < 4) {
            const double w = w_user[(size_t)pix * 4 + threadIdx.x];
            s_w2[threadIdx.x] = w * w;
        }
    } else if (warp == 0) {
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
                s_w2[s] = w * w;
            }
        }
    }
    constexpr int M = kNpar<FILL>;
    // the pixel's geometry, built once per block (FP64 trigonometry and
    // divisions) and read by every thread from shared memory
    __shared__ __align__(16) unsigned char s_geo_raw[sizeof(Geo<double>)];
    Geo<double> &s_geo = *reinterpret_cast<Geo<double> *>(s_geo_raw);
    if (threadIdx.x == 0) {
        double p[M];
#pragma unroll
        for (int d = 0; d < M; ++d) p[d] = params[(size_t)pix * M + d];
        const double mu = mu_px ? mu_px[pix] : pb.mu;
        s_geo = make_geo<double, NL, FILL>(pb, nlines, p, mu);
    }
    __syncthreads();
    const Geo<double> &g = s_geo;
    double he[ME_MAX_LINES];
#pragma unroll
    for (int l = 0; l < ME_MAX_LINES; ++l) he[l] = l < nlines ? pb.line[l].half_eta : 0.0;
    double ss[4] = {0, 0, 0, 0};
    for (int j = threadIdx.x; j < nl; j += blockDim.x) {
        double doff[ME_MAX_LINES];
#pragma unroll
        for (int l = 0; l < ME_MAX_LINES; ++l) doff[l] = l < nlines ? pb.lam[j] - pb.line[l].lam0 : 0.0;
        const Stokes4<double> s = me_point<double, NL, PAT, FILL>(g, doff, he, nlines, pb.line);
        const double r0 = (double)o[j] - s.I, r1 = (double)o[nl + j] - s.Q;
        const double r2 = (double)o[2 * nl + j] - s.U, r3 = (double)o[3 * nl + j] - s.V;
        ss[0] += r0 * r0;
        ss[1] += r1 * r1;
        ss[2] += r2 * r2;
        ss[3] += r3 * r3;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss[s] += __shfl_xor_sync(0xffffffffu, ss[s], off);
    }
    if (lane == 0)
        for (int s = 0; s < 4; ++s) s_red[warp][s] = ss[s];
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int s = 0; s < 4; ++s) {
            double a = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += s_red[w][s];
            tot += s_w2[s] * a;
        }
        chi2[pix] = tot / (double)(4 * nl - M);
    }
}

// Section 5.1 centre of symmetry, one warp per pixel: lanes scan candidates,
// each sums |I(i+j) - I(i-j)| in FP64 in increasing j; warp argmin (ties to
// the lowest index); lane 0 refines with the three-point parabola vertex,
// written without contraction.
template <class RO>
__global__ void __launch_bounds__(kSynthBlock)
k_line_centre(const __grid_constant__ KProblem pb, const RO *__restrict__ obs, int npix, int W, int lo,
              int hi, double *__restrict__ lam_c, int *__restrict__ idx)
{
    const int lane = threadIdx.x & 31;
    const int pix = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pix >= npix) return;
    const int nl = pb.n_lambda;
    const RO *I = obs + (size_t)pix * 4 * nl;
    auto S = [&](int i) {
        double s = 0.0;
        for (int j = 1; j <= W; ++j) s = __dadd_rn(s, fabs(__dsub_rn((double)I[i + j], (double)I[i - j])));
        return s;
    };
    double best = INFINITY;
    int bi = 0x7fffffff;
    for (int i = lo + lane; i <= hi; i += 32) {
        const double s = S(i);
        if (s < best || (s == best && i < bi)) { best = s; bi = i; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double os = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (os < best || (os == best && oi < bi)) { best = os; bi = oi; }
    }
    if (lane != 0) return;
    if (bi == 0x7fffffff) {
        lam_c[pix] = NAN;
        if (idx) idx[pix] = -1;
        return;
    }
    double xc = pb.lam[bi];
    if (bi - 1 >= lo && bi + 1 <= hi) {
        const double x0 = pb.lam[bi - 1], x1 = pb.lam[bi], x2 = pb.lam[bi + 1];
        const double y0 = S(bi - 1), y1 = best, y2 = S(bi + 1);
        const double d0 = __dsub_rn(x1, x0), d2 = __dsub_rn(x1, x2);
        const double e0 = __dsub_rn(y1, y0), e2 = __dsub_rn(y1, y2);
        const double num = __dsub_rn(__dmul_rn(__dmul_rn(d0, d0), e2), __dmul_rn(__dmul_rn(d2, d2), e0));
        const double den = __dsub_rn(__dmul_rn(d0, e2), __dmul_rn(d2, e0));
        if (den != 0.0) xc = __dsub_rn(x1, __dmul_rn(0.5, __ddiv_rn(num, den)));
    }
    lam_c[pix] = xc;
    if (idx) idx[pix] = bi;
}

template <class R> size_t offsets_smem(const KProblem &pb)
{
    return sizeof(R) * (ME_MAX_LINES + (size_t)pb.n_lines * pb.n_lambda);
}

template <class R, int NL, bool FILL = false>
cudaError_t synth_t(const KProblem &pb, const double *params, const double *mu_px, int n,
                    void *stokes, cudaStream_t st)
{
    const long long tot = (long long)n * pb.n_lambda;
    const int blocks = (int)((tot + kSynthBlock - 1) / kSynthBlock);
    k_synth<R, NL, FILL><<<blocks, kSynthBlock, offsets_smem<R>(pb), st>>>(pb, params, mu_px, n, (R *)stokes);
    return cudaGetLastError();
}

template <class R, int NL, bool FILL = false>
cudaError_t jac_t(const KProblem &pb, const double *params, const double *mu_px, int n,
                  void *stokes, void *jac, cudaStream_t st)
{
    const long long tot = (long long)n * pb.n_lambda;
    const int blocks = (int)((tot + kSynthBlock - 1) / kSynthBlock);
    k_jac<R, NL, FILL><<<blocks, kSynthBlock, offsets_smem<R>(pb), st>>>(pb, params, mu_px, n, (R *)stokes,
                                                                  (R *)jac);
    return cudaGetLastError();
}

template <class R, int NL, bool FILL = false>
cudaError_t vjp_t(const KProblem &pb, const double *params, const double *mu_px, int n,
                  const void *gs, double *gp, cudaStream_t st)
{
    const int per = kSynthBlock / 32;
    k_vjp<R, NL, FILL><<<(n + per - 1) / per, kSynthBlock, offsets_smem<R>(pb), st>>>(pb, params, mu_px, n,
                                                                               (const R *)gs, gp);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_synth(const KProblem &pb, int dtype, const double *params, const double *mu_px,
                         int n, void *stokes, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (pb.fill)
        return dtype == ME_F32 ? synth_t<float, 0, true>(pb, params, mu_px, n, stokes, st)
                               : synth_t<double, 0, true>(pb, params, mu_px, n, stokes, st);
    if (dtype == ME_F32) {
        if (pb.n_lines == 1) return synth_t<float, 1>(pb, params, mu_px, n, stokes, st);
        if (pb.n_lines == 2) return synth_t<float, 2>(pb, params, mu_px, n, stokes, st);
        return synth_t<float, 0>(pb, params, mu_px, n, stokes, st);
    }
    return synth_t<double, 0>(pb, params, mu_px, n, stokes, st);
}

cudaError_t launch_jac(const KProblem &pb, int dtype, const double *params, const double *mu_px,
                       int n, void *stokes, void *jac, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (pb.fill)
        return dtype == ME_F32 ? jac_t<float, 0, true>(pb, params, mu_px, n, stokes, jac, st)
                               : jac_t<double, 0, true>(pb, params, mu_px, n, stokes, jac, st);
    if (dtype == ME_F32) {
        if (pb.n_lines == 1) return jac_t<float, 1>(pb, params, mu_px, n, stokes, jac, st);
        if (pb.n_lines == 2) return jac_t<float, 2>(pb, params, mu_px, n, stokes, jac, st);
        return jac_t<float, 0>(pb, params, mu_px, n, stokes, jac, st);
    }
    return jac_t<double, 0>(pb, params, mu_px, n, stokes, jac, st);
}

cudaError_t launch_vjp(const KProblem &pb, int dtype, const double *params, const double *mu_px,
                       int n, const void *gs, double *gp, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (pb.fill)
        return dtype == ME_F32 ? vjp_t<float, 0, true>(pb, params, mu_px, n, gs, gp, st)
                               : vjp_t<double, 0, true>(pb, params, mu_px, n, gs, gp, st);
    if (dtype == ME_F32) {
        if (pb.n_lines == 1) return vjp_t<float, 1>(pb, params, mu_px, n, gs, gp, st);
        if (pb.n_lines == 2) return vjp_t<float, 2>(pb, params, mu_px, n, gs, gp, st);
        return vjp_t<float, 0>(pb, params, mu_px, n, gs, gp, st);
    }
    return vjp_t<double, 0>(pb, params, mu_px, n, gs, gp, st);
}

cudaError_t launch_line_centre(const KProblem &pb, int dtype, const void *obs, int npix, int W, int lo,
                               int hi, double *lam_c, int *idx, cudaStream_t st)
{
    if (npix <= 0) return cudaSuccess;
    const int per = kSynthBlock / 32;
    if (dtype == ME_F32)
        k_line_centre<float><<<(npix + per - 1) / per, kSynthBlock, 0, st>>>(pb, (const float *)obs, npix, W, lo,
                                                                            hi, lam_c, idx);
    else
        k_line_centre<double><<<(npix + per - 1) / per, kSynthBlock, 0, st>>>(pb, (const double *)obs, npix, W,
                                                                             lo, hi, lam_c, idx);
    return cudaGetLastError();
}

cudaError_t launch_chi2_f64(const KProblem &pb, int dtype, const void *obs, const double *w,
                            const double *mu_px, int npix, const double *params, double *chi2,
                            cudaStream_t st, KSub sub)
{
    if (npix <= 0) return cudaSuccess;
    if (dtype == ME_F32 && pb.fill)
        k_chi2_f64<float, true><<<npix, kSynthBlock, 0, st>>>(pb, (const float *)obs, w, mu_px, npix, params,
                                                              chi2, sub);
    else if (dtype == ME_F32 && !has_pattern(pb) && pb.n_lines == 2)
        k_chi2_f64<float, false, 2, false><<<npix, kSynthBlock, 0, st>>>(pb, (const float *)obs, w, mu_px, npix,
                                                                        params, chi2, sub);
    else if (dtype == ME_F32 && !has_pattern(pb) && pb.n_lines == 1)
        k_chi2_f64<float, false, 1, false><<<npix, kSynthBlock, 0, st>>>(pb, (const float *)obs, w, mu_px, npix,
                                                                        params, chi2, sub);
    else if (dtype == ME_F32)
        k_chi2_f64<float><<<npix, kSynthBlock, 0, st>>>(pb, (const float *)obs, w, mu_px, npix, params, chi2,
                                                        sub);
    else if (pb.fill)
        k_chi2_f64<double, true><<<npix, kSynthBlock, 0, st>>>(pb, (const double *)obs, w, mu_px, npix, params,
                                                               chi2, sub);
    else
        k_chi2_f64<double><<<npix, kSynthBlock, 0, st>>>(pb, (const double *)obs, w, mu_px, npix, params,
                                                         chi2, sub);
    return cudaGetLastError();
}

}  // namespace genesis
