// Verification kernels of the GA's fitness path (sm_103a): the fitness and
// its residuals for caller-given individuals, launched the way the GA
// evaluates them, and the FP32 pair path's w(z) branches for caller-given
// arguments.  They run the same device functions as k_ga_evolve (staging,
// weights, the pair path of me_pair.cuh and its warp votes), so that the
// arithmetic the GA ranks its population by can be compared with an
// independent FP64 evaluation of Section 5's synthesis and Eq. chisq.
#include "ga_evolve.cuh"

namespace genesis {

cudaError_t upload_tables_check(const HostTables &t)
{
    return cudaMemcpyToSymbol(c_fad, &t.fad, sizeof(FaddeevaTables));
}

namespace {

// One block per pixel, thread k = individual k of npop.  Threads k < nactive
// evaluate inside a divergent branch, as the GA's restarts do, so the pair
// path's votes run over exactly those lanes.
template <class R, int NL, int MAXT, bool PAT, int M>
__global__ void GENESIS_GA_BOUNDS(MAXT, R, NL, PAT)
k_ga_fitness(const __grid_constant__ KProblem pb, int weight_mode, const R *__restrict__ obs,
             const double *__restrict__ w_user, const double *__restrict__ mu_px, int nactive,
             const double *__restrict__ params, double *__restrict__ fit, R *__restrict__ res)
{
    constexpr bool FILL = M > ME_NPAR;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nl = pb.n_lambda;
    const int nlines = NL > 0 ? NL : pb.n_lines;
    const int npop = blockDim.x, k = threadIdx.x, pix = blockIdx.x;
    const GaSmem L = ga_smem_layout<R>(nl, nlines, npop, M);
    R *s_obs = (R *)(smem + L.obs);
    R *s_doff = (R *)(smem + L.doff);
    R *s_w2 = (R *)(smem + L.w2);
    R *s_he = (R *)(smem + L.he);
    float4 *s_kc = (float4 *)(smem + L.kc);
    const R inv_nu = R(1) / R(4 * nl - M);
    stage_offsets_ga<R>(pb, nlines, nl, k, s_doff, s_he);
    stage_obs<R>(obs + (size_t)pix * 4 * nl, nl, k, s_obs);
    __syncthreads();
    stage_weights<R>(weight_mode, w_user, pix, s_obs, nl, k, s_w2);
    __syncthreads();
    if (sizeof(R) == 4) {
        weight_obs_rows<R>(s_obs, nl, k, s_w2);
        __syncthreads();
    }
    R he[ME_MAX_LINES];
#pragma unroll
    for (int l = 0; l < ME_MAX_LINES; ++l) he[l] = s_he[l];
    const R mu = mu_px ? R(mu_px[pix]) : R(pb.mu);
    if (k < nactive) {
        const size_t ind = (size_t)pix * npop + k;
        R p[M];
#pragma unroll
        for (int d = 0; d < M; ++d) p[d] = R(params[ind * M + d]);
        WorkCount wc{};
        const R f = fitness<R, NL, false, PAT, FILL, true>(pb, nlines, nl, p, mu, s_obs, s_doff, he, s_w2, inv_nu,
                                                           wc, s_kc, res ? res + ind * 4 * nl : nullptr);
        fit[ind] = double(f);
    }
}

template <class R, int NL, int MAXT, bool PAT, int M>
cudaError_t launch_fitness_t(const KProblem &pb, int weight_mode, const void *obs, const double *w,
                             const double *mu_px, int npix, int npop, int nactive, const double *params,
                             double *fit, void *res, cudaStream_t st)
{
    const int nlines = NL > 0 ? NL : pb.n_lines;
    const GaSmem L = ga_smem_layout<R>(pb.n_lambda, nlines, npop, M);
    auto kern = k_ga_fitness<R, NL, MAXT, PAT, M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    kern<<<npix, npop, L.total, st>>>(pb, weight_mode, (const R *)obs, w, mu_px, nactive, params, fit, (R *)res);
    return cudaGetLastError();
}

// FP32 pair path w(z) for caller-given pairs: thread i (32 to a warp, in
// index order) holds pair i; lanes beyond n have exited, so the last warp of
// a ragged n votes over its remaining lanes, as a partial warp of the GA does.
// mode 0: one component with the outside-in tests (fad_pair); 1: inside-out
// (fad_pair_in); 2: an effective triplet with pi arguments x and splitting
// vB, its level voted as a whole (triplet_level) and its components added
// into the profile sums with unit strength (triplet_acc), out = (P, Pim, Sg,
// Sgi, Dd, Di) per point.
__global__ void k_fad_probe(const float2 *__restrict__ x, const float *__restrict__ a,
                            const float *__restrict__ vB, int n, int mode, float *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Geo<float> g = {};
    g.a = a[i];
    g.a2 = g.a * g.a;
    g.vB[0] = mode == 2 ? vB[i] : 0.0f;
    pair_thresholds(g, 1);
    g.vmask = __activemask();
    const float2 v = x[i];
    if (mode == 2) {
        const float2 xb = add2(v, f2(g.vB[0])), xr = sub2(v, f2(g.vB[0]));
        // unit strength: the series' doubled coefficients as they are
        const float2 *wq = c_fad.w32x2, qs = f2(kInvSqrtPi);
        float2 P = f2(0.f), Pim = f2(0.f), Sb = f2(0.f), Sbi = f2(0.f), Sr = f2(0.f), Sri = f2(0.f), P0 = f2(0.f);
        const int lev = triplet_level(v, g, 0);
        if (lev == 3)
            triplet_acc<3, false>(xb, v, xr, g, wq, qs, P, Pim, Sb, Sbi, Sr, Sri, P0);
        else if (lev == 2)
            triplet_acc<2, false>(xb, v, xr, g, wq, qs, P, Pim, Sb, Sbi, Sr, Sri, P0);
        else if (lev == 1)
            triplet_acc<1, false>(xb, v, xr, g, wq, qs, P, Pim, Sb, Sbi, Sr, Sri, P0);
        else
            triplet_acc<0, false>(xb, v, xr, g, wq, qs, P, Pim, Sb, Sbi, Sr, Sri, P0);
        // the sums and differences of the sigma profiles, as the fitness forms them
        const float2 o[6] = {P, Pim, add2(Sb, Sr), add2(Sbi, Sri), sub2(Sr, Sb), sub2(Sri, Sbi)};
        float *r = out + (size_t)i * 12;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            r[c] = o[c].x;
            r[6 + c] = o[c].y;
        }
        return;
    }
    float2 wx, wy, qi;
    if (mode == 0) fad_pair(v, g, f2(1.0f), f2(kInvSqrtPi), wx, wy, qi);
    else fad_pair_in(v, g, f2(1.0f), f2(kInvSqrtPi), wx, wy, qi);
    wx = mul2(qi, wx);  // w itself: the unit-weight profile
    wy = mul2(qi, wy);
    float *r = out + (size_t)i * 4;
    r[0] = wx.x;
    r[1] = wy.x;
    r[2] = wx.y;
    r[3] = wy.y;
}

}  // namespace

// The instantiation ga_invert_batch would use for this problem.
cudaError_t launch_ga_fitness(const KProblem &pb, int dtype, int weight_mode, const void *obs, const double *w,
                              const double *mu_px, int npix, int npop, int nactive, const double *params,
                              double *fit, void *res, cudaStream_t st)
{
    if (npix <= 0) return cudaSuccess;
    const bool pat = has_pattern(pb);
#define GENESIS_FIT(R, NL, MAXT, PAT, M) \
    launch_fitness_t<R, NL, MAXT, PAT, M>(pb, weight_mode, obs, w, mu_px, npix, npop, nactive, params, fit, res, st)
    if (pb.fill) {
        constexpr int M = ME_NPAR_MAX;
        if (dtype == ME_F32) return npop <= 256 ? GENESIS_FIT(float, 0, 256, true, M) : GENESIS_FIT(float, 0, 1024, true, M);
        return npop <= 256 ? GENESIS_FIT(double, 0, 256, true, M) : GENESIS_FIT(double, 0, 1024, true, M);
    }
    constexpr int M = ME_NPAR;
    if (dtype == ME_F32 && pat)
        return npop <= 256 ? GENESIS_FIT(float, 0, 256, true, M) : GENESIS_FIT(float, 0, 1024, true, M);
    if (dtype == ME_F32) {
        if (npop <= 256) {
            if (pb.n_lines == 1) return GENESIS_FIT(float, 1, 256, false, M);
            if (pb.n_lines == 2) return GENESIS_FIT(float, 2, 256, false, M);
            return GENESIS_FIT(float, 0, 256, false, M);
        }
        return GENESIS_FIT(float, 0, 1024, false, M);
    }
    return npop <= 256 ? GENESIS_FIT(double, 0, 256, true, M) : GENESIS_FIT(double, 0, 1024, true, M);
#undef GENESIS_FIT
}

cudaError_t launch_fad_probe(const float *x, const float *a, const float *vB, int n, int mode, float *out,
                             cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_fad_probe<<<(n + 127) / 128, 128, 0, st>>>((const float2 *)x, a, vB, n, mode, out);
    return cudaGetLastError();
}

}  // namespace genesis
