// The fill-fraction instantiations of the GA kernel (Section 5.2: ten
// parameters, the tenth the magnetic fill fraction), built in a translation
// unit of their own so that the library's units compile in parallel.
#include "ga_evolve.cuh"

namespace genesis {

cudaError_t upload_tables_ga_fill(const HostTables &t)
{
    cudaError_t e = cudaMemcpyToSymbol(c_fad, &t.fad, sizeof(FaddeevaTables));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_sobol, t.sobol, sizeof(t.sobol));
}

// Every line may carry a full pattern here (run-time check per line).
cudaError_t launch_ga_evolve_fill(const KProblem &pb, const KGa &ga, int dtype, const void *obs,
                                  const double *w, const double *mu_px, int npix, double *best,
                                  uint16_t *best_genes, cudaStream_t st, KSeed sd, KSub sub)
{
    if (npix <= 0) return cudaSuccess;
    constexpr int M = ME_NPAR_MAX;
    if (dtype == ME_F32) {
        if (ga.npop <= 256)
            return launch_evolve_t<float, 0, 256, false, true, M>(pb, ga, obs, w, mu_px, npix, best, best_genes,
                                                                  st, nullptr, sd, sub);
        return launch_evolve_t<float, 0, 1024, false, true, M>(pb, ga, obs, w, mu_px, npix, best, best_genes,
                                                               st, nullptr, sd, sub);
    }
    if (ga.npop <= 256)
        return launch_evolve_t<double, 0, 256, false, true, M>(pb, ga, obs, w, mu_px, npix, best, best_genes,
                                                               st, nullptr, sd, sub);
    return launch_evolve_t<double, 0, 1024, false, true, M>(pb, ga, obs, w, mu_px, npix, best, best_genes,
                                                            st, nullptr, sd, sub);
}

}  // namespace genesis
