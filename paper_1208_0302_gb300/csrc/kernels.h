// Internal launch interface between the C-ABI layer and the kernel units.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "me_device.cuh"

namespace genesis {

// GA launch parameters (Section 3 operators, Section 5.6 restarts).
struct KGa {
    int npop, ngen, nsamp, weight_mode;
    uint64_t seed, pixel_id0;
    uint64_t t_cross;       // crossover iff u32 < t_cross
    // mutation thresholds: t_mut[b (b + 1) / 2 + c] = floor(2^32 (1 - prod_{d=c..b}
    // (1 - q_d))) for c <= b, q_d the flip probability of bit d (0 = MSB): the
    // probability that a flip falls among bits c..b of a word
    uint64_t t_mut[136];
    uint32_t rk[10][2];     // Philox4x32-10 round keys of seed: (k0, k1) + r (W0, W1)
    double lo[ME_NPAR_MAX], hi[ME_NPAR_MAX];
};

// Round keys of Philox4x32-10 for a 64-bit seed (k0 = low word, k1 = high):
// round r uses (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85) mod 2^32.
inline void philox_round_keys(uint64_t seed, uint32_t rk[10][2])
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[r][0] = k0;
        rk[r][1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Parameters per model: 9, or 10 with the fill fraction of Section 5.2.
template <bool FILL> constexpr int kNpar = ME_NPAR + (FILL ? 1 : 0);

// Section 5.5 seeds and polarity restriction: seeds [npix][nseed][3] of
// (B, psi, chi), NaN = keep the Sobol gene; polarity [npix] of -1, 0, +1;
// per-pixel bounds [npix][2][M] of Section 5.3 (NULL = the launch's).
struct KSeed {
    const double *seeds;
    int nseed;
    const int *polarity;
    const double *bounds_px;
};

// A subset of a map: block b processes pixel index[b] for b < *count (both
// on the device; NULL index = identity, NULL count = all npix).
struct KSub {
    const int *index;
    const int *count;
};

struct KLm {
    int iters;
    double lambda0;
    unsigned free_mask;  // bit k set: parameter k is fitted, else held
    double lo[ME_NPAR_MAX], hi[ME_NPAR_MAX];
};

// Section 5.3 bound rule around a prefit (margins per parameter).
struct KPrefitBounds {
    int npar;
    double lo[ME_NPAR_MAX], hi[ME_NPAR_MAX], lower[ME_NPAR_MAX], upper[ME_NPAR_MAX];
};

// Coefficient tables, computed once on the host.
struct HostTables {
    FaddeevaTables fad;
    uint32_t sobol[10][32];
};
const HostTables &host_tables();

// Per translation unit: copy the tables into that unit's __constant__ copy
// on the current device.
cudaError_t upload_tables_ga(const HostTables &t);
cudaError_t upload_tables_synth(const HostTables &t);
cudaError_t upload_tables_lm(const HostTables &t);
cudaError_t upload_tables_ga_fill(const HostTables &t);
cudaError_t upload_tables_check(const HostTables &t);

// ga_kernels.cu
cudaError_t launch_ga_evolve(const KProblem &pb, const KGa &ga, int dtype, const void *obs,
                             const double *w, const double *mu_px, int npix, double *best,
                             uint16_t *best_genes, cudaStream_t st, KSeed sd = {}, KSub sub = {});
// ga_fill_kernels.cu: the same for problems with the fill fraction
cudaError_t launch_ga_evolve_fill(const KProblem &pb, const KGa &ga, int dtype, const void *obs,
                                  const double *w, const double *mu_px, int npix, double *best,
                                  uint16_t *best_genes, cudaStream_t st, KSeed sd, KSub sub);
cudaError_t launch_ga_count(const KProblem &pb, const KGa &ga, int dtype, const void *obs,
                            const double *w, const double *mu_px, int npix, double *best,
                            unsigned long long *counts, cudaStream_t st);
// true when a line of the problem carries its full Zeeman pattern
bool has_pattern(const KProblem &pb);
// ga_check_kernels.cu: the GA's fitness on given individuals and the pair
// path's w(z) branches (verification entry points)
cudaError_t launch_ga_fitness(const KProblem &pb, int dtype, int weight_mode, const void *obs, const double *w,
                              const double *mu_px, int npix, int npop, int nactive, const double *params,
                              double *fit, void *res, cudaStream_t st);
cudaError_t launch_fad_probe(const float *x, const float *a, const float *vB, int n, int mode, float *out,
                             cudaStream_t st);
cudaError_t launch_ga_breed(const KGa &ga, int npar, const uint16_t *genes, const double *fit, int nprob,
                            int gen, uint16_t *child, int *elite, cudaStream_t st);
cudaError_t launch_ga_restart(int npop, int npar, uint16_t *genes, const double *fit, int nprob,
                              uint64_t sobol_next, cudaStream_t st);
cudaError_t launch_philox(const uint32_t *ctr, int n, uint64_t key, uint32_t *out, cudaStream_t st);
cudaError_t launch_sobol(uint64_t first, int n, int ndim, uint32_t *out, cudaStream_t st);

// synth_kernels.cu
cudaError_t launch_synth(const KProblem &pb, int dtype, const double *params, const double *mu_px,
                         int n, void *stokes, cudaStream_t st);
cudaError_t launch_jac(const KProblem &pb, int dtype, const double *params, const double *mu_px,
                       int n, void *stokes, void *jac, cudaStream_t st);
cudaError_t launch_vjp(const KProblem &pb, int dtype, const double *params, const double *mu_px,
                       int n, const void *grad_stokes, double *grad_params, cudaStream_t st);
cudaError_t launch_chi2_f64(const KProblem &pb, int dtype, const void *obs, const double *w,
                            const double *mu_px, int npix, const double *params, double *chi2,
                            cudaStream_t st, KSub sub = {});

// Section 2 selection, weak-field estimate and Section 5.5 seeds.
struct KClassify {
    double p_thresh, kz;  // kz = 4.6686e-13 g lambda0^2 of the chosen line
    int q_lo, q_hi, c_lo, c_hi, npar;
    int *flag, *polarity;
    double *pol, *weak, *seeds, *best;
};
cudaError_t launch_classify(const KProblem &pb, int dtype, const void *obs, int npix, const KClassify &c,
                            cudaStream_t st);
cudaError_t launch_prefit_bounds(const double *p_hat, int npix, const KPrefitBounds &r, double *out,
                                 cudaStream_t st);
// Order-preserving selection of the pixels whose flag equals want.
size_t select_scratch_bytes(int npix);
// Address and size of the file-scope tile array of me_select_static.
cudaError_t select_static_scratch(void **ptr, size_t *bytes);
cudaError_t launch_select(const int *flag, int npix, int want, int *index, int *count, void *scratch,
                          cudaStream_t st);

cudaError_t launch_line_centre(const KProblem &pb, int dtype, const void *obs, int npix, int W, int lo,
                               int hi, double *lam_c, int *idx, cudaStream_t st);

// lm_kernels.cu
cudaError_t launch_lm_sigma(const KProblem &pb, int dtype, const void *obs, const double *w,
                            const double *mu_px, int npix, const double *params, double *sigma,
                            cudaStream_t st);
cudaError_t launch_lm(const KProblem &pb, const KLm &lm, int dtype, const void *obs,
                      const double *w, const double *mu_px, int npix, double *params,
                      cudaStream_t st, KSub sub = {});

// peak_kernels.cu: FP32 FMA-pipe throughput probe (measurement only)
double fma_peak_flops(int packed, int nblocks, int iters);
int fma_peak_threads();
cudaError_t launch_fma_peak(int packed, int nblocks, int iters, float *out, cudaStream_t st);

// api.cu: argument validation shared by the C entry points and the serving
// loop.  Each returns ME_OK or an ME_E* code with the thread-local message set.
extern thread_local std::string g_last_error;
int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *where);
int ensure_device();
int make_problem(const me_problem *pb, KProblem &k);
int npar_of(const me_problem *pb);  // 9, or 10 with the fill fraction
int check_bounds(const me_bounds *b, int npar);
int make_ga(const ga_config *cfg, const me_bounds *b, uint64_t pid0, KGa &g, int npar);
cudaStream_t as_stream(void *s);

// Decode of Eq. decode in FP64 without contraction, the same expression the
// reference evaluation uses: lo + (hi - lo) * (g / 65535).
__device__ __forceinline__ double decode64(uint16_t g, double lo, double hi)
{
    return __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), __ddiv_rn((double)g, 65535.0)));
}

// Nearest gene of a seed value (Section 5.5), the inverse of the decode:
// t = (x - lo) / (hi - lo) clamped to [0, 1], g = floor(65535 t + 1/2).
__device__ __forceinline__ uint16_t encode64(double x, double lo, double hi)
{
    double t = __ddiv_rn(__dsub_rn(x, lo), __dsub_rn(hi, lo));
    if (!(t > 0.0)) t = 0.0;
    if (t > 1.0) t = 1.0;
    return (uint16_t)floor(__dadd_rn(__dmul_rn(t, 65535.0), 0.5));
}

// Section 5.5 polarity restriction of the inclination domain [lo, hi]:
// +1 keeps [lo, min(hi, 90)], -1 keeps [max(lo, 90), hi]; 0, or a half
// that would be empty, keeps [lo, hi].
__host__ __device__ __forceinline__ void polarity_bounds(int pol, double lo, double hi, double &a,
                                                         double &b)
{
    a = lo;
    b = hi;
    if (pol > 0 && hi > 90.0) b = 90.0;
    if (pol < 0 && lo < 90.0) a = 90.0;
    if (!(a < b)) {
        a = lo;
        b = hi;
    }
}

}  // namespace genesis
