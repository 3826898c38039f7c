// Fused genetic-algorithm inversion kernel for sm_103a (Section 3, Algorithm 1;
// Section 5.6), plus the operator-only kernels used to verify it.
//
// One thread block per pixel, one thread per individual.  The pixel's
// observed Stokes profiles, its wavelength offsets, the population's uint16
// genotypes (double-buffered) and fitness stay in shared memory for all
// generations; no host round trip happens between generations.  Each thread
// walks the wavelength grid for its own individual, so every lane of a warp
// reads the same shared-memory word (broadcast) and the chi2 sum needs no
// cross-thread reduction.
#include "ga_evolve.cuh"

namespace genesis {

cudaError_t upload_tables_ga(const HostTables &t)
{
    cudaError_t e = cudaMemcpyToSymbol(c_fad, &t.fad, sizeof(FaddeevaTables));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_sobol, t.sobol, sizeof(t.sobol));
}

namespace {

// ------------------------------------------------- operator-only kernels
template <int M>
__global__ void k_ga_breed(const __grid_constant__ KGa ga, const uint16_t *__restrict__ genes,
                           const double *__restrict__ fit, int gen, uint16_t *__restrict__ child,
                           int *__restrict__ elite_out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int npop = ga.npop, k = threadIdx.x, prob = blockIdx.x;
    double *s_fit = (double *)smem;
    double *s_wmin = s_fit + npop;
    int *s_widx = (int *)(s_wmin + 32);
    uint16_t *s_cur = (uint16_t *)(s_widx + 32);
    uint16_t *s_new = s_cur + npop * M;
    const size_t base = (size_t)prob * npop;
    s_fit[k] = clean_fit(fit[base + k]);
#pragma unroll
    for (int d = 0; d < M; ++d) s_cur[k * M + d] = genes[(base + k) * M + d];
    __syncthreads();
    const int elite = block_argmin<double>(s_fit, s_wmin, s_widx);
    uint16_t g[M];
    breed_one<double, M>(ga, ga.pixel_id0 + (uint64_t)prob, gen, k, npop, s_fit, s_cur, elite,
                      s_new + k * M, g);
#pragma unroll
    for (int d = 0; d < M; ++d) child[(base + k) * M + d] = g[d];
    if (k == 0 && elite_out) elite_out[prob] = elite;
}

template <int M>
__global__ void k_ga_restart(int npop, uint16_t *__restrict__ genes, const double *__restrict__ fit,
                             uint64_t sobol_next)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_fit = (double *)smem;
    const int k = threadIdx.x, prob = blockIdx.x;
    const size_t base = (size_t)prob * npop;
    s_fit[k] = clean_fit(fit[base + k]);
    __syncthreads();
    const int rank = stable_rank<double>(s_fit, npop, k);
    if (rank >= npop / 2) {
        const uint64_t n = sobol_next + (uint64_t)(rank - npop / 2);
#pragma unroll
        for (int d = 0; d < M; ++d)
            genes[(base + k) * M + d] = (uint16_t)(sobol_point(n, d) >> 16);
    }
}

__global__ void k_philox(const uint32_t *__restrict__ ctr, int n, uint64_t key, uint32_t *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    U4 c = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    const U4 r = philox4x32_10(c, (uint32_t)key, (uint32_t)(key >> 32));
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

__global__ void k_sobol(uint64_t first, int n, int ndim, uint32_t *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * ndim) return;
    const int pt = i / ndim, d = i - pt * ndim;
    out[i] = sobol_point(first + (uint64_t)pt, d);
}

}  // namespace

bool has_pattern(const KProblem &pb)
{
    for (int l = 0; l < pb.n_lines; ++l)
        if (pb.line[l].ncomp[0] != 0) return true;
    return false;
}

cudaError_t launch_ga_evolve(const KProblem &pb, const KGa &ga, int dtype, const void *obs,
                             const double *w, const double *mu_px, int npix, double *best,
                             uint16_t *best_genes, cudaStream_t st, KSeed sd, KSub sub)
{
    if (npix <= 0) return cudaSuccess;
    if (pb.fill) return launch_ga_evolve_fill(pb, ga, dtype, obs, w, mu_px, npix, best, best_genes, st, sd, sub);
    const bool pat = has_pattern(pb);
#define GENESIS_EVOLVE(R, NL, MAXT, PAT) \
    launch_evolve_t<R, NL, MAXT, false, PAT>(pb, ga, obs, w, mu_px, npix, best, best_genes, st, nullptr, sd, sub)
    if (dtype == ME_F32 && pat) {
        if (ga.npop <= 256) return GENESIS_EVOLVE(float, 0, 256, true);
        return GENESIS_EVOLVE(float, 0, 1024, true);
    }
    if (dtype == ME_F32) {
        if (ga.npop <= 256) {
            if (pb.n_lines == 1) return GENESIS_EVOLVE(float, 1, 256, false);
            if (pb.n_lines == 2) return GENESIS_EVOLVE(float, 2, 256, false);
            return GENESIS_EVOLVE(float, 0, 256, false);
        }
        return GENESIS_EVOLVE(float, 0, 1024, false);
    }
    if (ga.npop <= 256) return GENESIS_EVOLVE(double, 0, 256, true);
    return GENESIS_EVOLVE(double, 0, 1024, true);
#undef GENESIS_EVOLVE
}

cudaError_t launch_ga_count(const KProblem &pb, const KGa &ga, int dtype, const void *obs,
                            const double *w, const double *mu_px, int npix, double *best,
                            unsigned long long *counts, cudaStream_t st)
{
    if (npix <= 0) return cudaSuccess;
    if (dtype == ME_F32 && ga.npop <= 256 && !pb.fill) {
        if (has_pattern(pb))
            return launch_evolve_t<float, 0, 256, true, true>(pb, ga, obs, w, mu_px, npix, best, nullptr, st, counts);
        if (pb.n_lines == 2)
            return launch_evolve_t<float, 2, 256, true, false>(pb, ga, obs, w, mu_px, npix, best, nullptr, st, counts);
        return launch_evolve_t<float, 0, 256, true, false>(pb, ga, obs, w, mu_px, npix, best, nullptr, st, counts);
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_ga_breed(const KGa &ga, int npar, const uint16_t *genes, const double *fit, int nprob,
                            int gen, uint16_t *child, int *elite, cudaStream_t st)
{
    if (nprob <= 0) return cudaSuccess;
    const int smem = ga.npop * 8 + 32 * 8 + 32 * 4 + 2 * ga.npop * npar * 2;
    if (npar == ME_NPAR_MAX)
        k_ga_breed<ME_NPAR_MAX><<<nprob, ga.npop, smem, st>>>(ga, genes, fit, gen, child, elite);
    else
        k_ga_breed<ME_NPAR><<<nprob, ga.npop, smem, st>>>(ga, genes, fit, gen, child, elite);
    return cudaGetLastError();
}

cudaError_t launch_ga_restart(int npop, int npar, uint16_t *genes, const double *fit, int nprob,
                              uint64_t sobol_next, cudaStream_t st)
{
    if (nprob <= 0) return cudaSuccess;
    if (npar == ME_NPAR_MAX)
        k_ga_restart<ME_NPAR_MAX><<<nprob, npop, npop * 8, st>>>(npop, genes, fit, sobol_next);
    else
        k_ga_restart<ME_NPAR><<<nprob, npop, npop * 8, st>>>(npop, genes, fit, sobol_next);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, int n, uint64_t key, uint32_t *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_philox<<<(n + 127) / 128, 128, 0, st>>>(ctr, n, key, out);
    return cudaGetLastError();
}

cudaError_t launch_sobol(uint64_t first, int n, int ndim, uint32_t *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int tot = n * ndim;
    k_sobol<<<(tot + 127) / 128, 128, 0, st>>>(first, n, ndim, out);
    return cudaGetLastError();
}

}  // namespace genesis
