// C-ABI entry points of libgenesis (see include/genesis.h): argument
// validation, launch-parameter assembly and per-device table upload.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "genesis.h"
#include "kernels.h"

namespace genesis {

thread_local std::string g_last_error;

namespace {

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    return fail(ME_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------- coefficient tables

// Weideman (1994) coefficients a_0..a_N of (L^2 + t^2) exp(-t^2) in the basis
// ((L + i t)/(L - i t))^n, i.e. the Fourier cosine coefficients of
// f(theta) = L^2 sec^2(theta/2) exp(-L^2 tan^2(theta/2)) on (-pi, pi),
// integrated with the (spectrally accurate) midpoint rule.
std::vector<double> weideman_coefficients(int N, double L)
{
    const int K = 8192;
    std::vector<double> a(N + 1, 0.0);
    for (int k = 0; k < K; ++k) {
        const double th = -M_PI + 2.0 * M_PI * (k + 0.5) / K;
        const double t = L * std::tan(0.5 * th);
        const double f = std::exp(-t * t) * (L * L + t * t);
        for (int n = 0; n <= N; ++n) a[n] += f * std::cos(n * th);
    }
    for (int n = 0; n <= N; ++n) a[n] /= K;
    return a;
}

// Sobol direction numbers (Section 5.6; Sobol 1967, Bratley & Fox 1988):
// dimension 0 is van der Corput; dimension d >= 1 takes the d-th primitive
// polynomial over GF(2) (ordered by degree, then by integer encoding) and
// initial numbers m_k = 2^k - 1, extended by the Sobol recurrence.
bool gf2_primitive(unsigned poly, int deg)
{
    // x must have multiplicative order exactly 2^deg - 1 modulo poly
    const unsigned period = (1u << deg) - 1u;
    unsigned r = 1u;
    for (unsigned e = 1; e <= period; ++e) {
        r <<= 1;
        if (r >> deg) r ^= poly;
        if (r == 1u) return e == period;
    }
    return false;
}

void sobol_directions(uint32_t out[10][32])
{
    for (int k = 0; k < 32; ++k) out[0][k] = 1u << (31 - k);
    int dim = 1;
    for (int deg = 1; dim < 10; ++deg) {
        for (unsigned poly = (1u << deg) | 1u; poly < (2u << deg) && dim < 10; poly += 2u) {
            if (!gf2_primitive(poly, deg)) continue;
            uint64_t m[33];
            for (int k = 1; k <= deg; ++k) m[k] = (1ull << k) - 1ull;
            for (int k = deg + 1; k <= 32; ++k) {
                uint64_t v = m[k - deg] ^ (m[k - deg] << deg);
                for (int i = 1; i < deg; ++i)
                    if ((poly >> (deg - i)) & 1u) v ^= m[k - i] << i;
                m[k] = v;
            }
            for (int k = 1; k <= 32; ++k) out[dim][k - 1] = (uint32_t)(m[k] << (32 - k));
            ++dim;
        }
    }
}

HostTables build_tables()
{
    HostTables t;
    std::memset(&t, 0, sizeof t);
    {
        const double L = 4.0;
        const std::vector<double> a = weideman_coefficients(16, L);
        for (int n = 0; n <= 16; ++n) {
            t.fad.w32[n] = (float)a[n];
            t.fad.w32x2[n] = make_float2(2.0f * (float)a[n], 2.0f * (float)a[n]);
        }
        t.fad.L32 = (float)L;
    }
    {
        const double L = 5.0;
        const std::vector<double> a = weideman_coefficients(36, L);
        for (int n = 0; n <= 36; ++n) t.fad.w64[n] = a[n];
        t.fad.L64 = L;
    }
    sobol_directions(t.sobol);
    return t;
}

}  // namespace

std::mutex g_init_mu;
bool g_dev_ready[256];

// Per device: the address of me_select_static's file-scope tile array,
// looked up once at set-up.
static void *g_select_static[256];
static size_t g_select_static_bytes = 0;

int ensure_device()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 256) return fail(ME_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (g_dev_ready[dev]) return ME_OK;
    const HostTables &t = host_tables();
    if ((e = upload_tables_ga(t)) != cudaSuccess) return cuda_fail(e, "upload tables");
    if ((e = upload_tables_synth(t)) != cudaSuccess) return cuda_fail(e, "upload tables");
    if ((e = upload_tables_lm(t)) != cudaSuccess) return cuda_fail(e, "upload tables");
    if ((e = upload_tables_ga_fill(t)) != cudaSuccess) return cuda_fail(e, "upload tables");
    if ((e = upload_tables_check(t)) != cudaSuccess) return cuda_fail(e, "upload tables");
    if ((e = select_static_scratch(&g_select_static[dev], &g_select_static_bytes)) != cudaSuccess)
        return cuda_fail(e, "select scratch address");
    g_dev_ready[dev] = true;
    return ME_OK;
}

// ------------------------------------------------------------- validation
int zeeman_pattern(int jl, double gl, int ju, double gu, int n[3], double sh[3][ME_MAX_COMP],
                   double st[3][ME_MAX_COMP]);

int make_problem(const me_problem *pb, KProblem &k)
{
    if (!pb) return fail(ME_EINVAL, "problem is NULL");
    if (pb->n_lines < 1 || pb->n_lines > ME_MAX_LINES) return fail(ME_EINVAL, "n_lines must be 1..4");
    if (pb->n_lambda < 1 || pb->n_lambda > ME_MAX_LAMBDA)
        return fail(ME_EINVAL, "n_lambda must be 1..ME_MAX_LAMBDA");
    if (pb->fill_fraction != 0 && pb->fill_fraction != 1) return fail(ME_EINVAL, "fill_fraction must be 0 or 1");
    if (4 * pb->n_lambda <= npar_of(pb))
        return fail(ME_EINVAL, "n_lambda too small: 4 n_lambda must exceed the parameter count");
    if (!pb->lambda_A) return fail(ME_EINVAL, "lambda_A is NULL");
    if (pb->dtype != ME_F32 && pb->dtype != ME_F64) return fail(ME_EINVAL, "dtype must be ME_F32 or ME_F64");
    if (!(pb->lambda_dop_A > 0.0) || !std::isfinite(pb->lambda_dop_A))
        return fail(ME_EINVAL, "lambda_dop_A must be positive");
    if (!std::isfinite(pb->mu)) return fail(ME_EINVAL, "mu must be finite");
    std::memset(&k, 0, sizeof k);
    k.n_lines = pb->n_lines;
    k.n_lambda = pb->n_lambda;
    k.fill = pb->fill_fraction;
    k.mu = pb->mu;
    for (int l = 0; l < pb->n_lines; ++l) {
        const me_line &ln = pb->line[l];
        if (!(ln.lambda0_A > 0.0) || !std::isfinite(ln.lambda0_A) || !std::isfinite(ln.g_eff) ||
            !std::isfinite(ln.eta_ratio))
            return fail(ME_EINVAL, "invalid line parameters");
        k.line[l].lam0 = ln.lambda0_A;
        k.line[l].lam0_c = ln.lambda0_A / kSpeedOfLight;
        k.line[l].dscale = 1e-3 * ln.lambda0_A / pb->lambda_dop_A;
        k.line[l].zfac = kZeeman * ln.g_eff * ln.lambda0_A * ln.lambda0_A;
        k.line[l].half_eta = 0.5 * ln.eta_ratio;
        k.line[l].qs2 = make_float2((float)(k.line[l].half_eta * 0.56418958354775628695),
                                    (float)(k.line[l].half_eta * 0.56418958354775628695));
        {
            const HostTables &ht = host_tables();
            for (int n = 0; n <= 16; ++n) {
                const float c = (float)(2.0 * (double)ht.fad.w32[n] * k.line[l].half_eta);
                k.line[l].wq2[n] = make_float2(c, c);
            }
        }
        k.line[l].zfacL = kZeeman * ln.lambda0_A * ln.lambda0_A;
        if (ln.pattern) {
            int rc = zeeman_pattern(ln.j_lower, ln.g_lower, ln.j_upper, ln.g_upper, k.line[l].ncomp,
                                    k.line[l].cshift, k.line[l].cstr);
            if (rc) return rc;
            for (int g = 0; g < 3; ++g)
                for (int i = 0; i < k.line[l].ncomp[g]; ++i) {
                    k.line[l].cshift32[g][i] = (float)k.line[l].cshift[g][i];
                    k.line[l].cstr32[g][i] = (float)k.line[l].cstr[g][i];
                }
        } else if (ln.pattern != 0) {
            return fail(ME_EINVAL, "pattern must be 0 or 1");
        }
    }
    for (int j = 0; j < pb->n_lambda; ++j) {
        const double v = pb->lambda_A[j];
        if (!std::isfinite(v) || !(v > 0.0)) return fail(ME_EINVAL, "lambda_A must be finite and positive");
        // lambda_j - lambda0_l must be exact in FP64 (Sterbenz): within a factor 2
        for (int l = 0; l < pb->n_lines; ++l)
            if (v > 2.0 * k.line[l].lam0 || 2.0 * v < k.line[l].lam0)
                return fail(ME_EINVAL, "wavelength grid more than a factor 2 from a line");
        k.lam[j] = v;
    }
    return ME_OK;
}

// Zeeman components of lower (J_l, g_l) -> upper (J_u, g_u) in LS coupling
// (Section 5 full pattern), from the closed-form relative line strengths of
// dipole transitions (Condon & Shortley) for Delta J = 0, +-1, normalised per
// group q = M_l - M_u (-1 sigma_blue, 0 pi, +1 sigma_red).  Shift of M_u -> M_l
// in Larmor units toward longer wavelength: g_l M_l - g_u M_u.
int zeeman_pattern(int jl, double gl, int ju, double gu, int n[3], double sh[3][ME_MAX_COMP],
                   double st[3][ME_MAX_COMP])
{
    if (jl < 0 || ju < 0 || jl > 4 || ju > 4 || std::abs(jl - ju) > 1 || (jl == 0 && ju == 0) ||
        !std::isfinite(gl) || !std::isfinite(gu))
        return fail(ME_EINVAL, "invalid Zeeman transition (need |J_l - J_u| <= 1, J <= 4, not 0 -> 0)");
    const int J = ju;
    for (int q = -1; q <= 1; ++q) {
        const int gi = q + 1;
        n[gi] = 0;
        double tot = 0.0;
        for (int mu = -ju; mu <= ju; ++mu) {
            const int ml = mu + q;
            if (ml < -jl || ml > jl) continue;
            double s;
            if (jl == ju) {  // Delta J = 0
                s = q == 0 ? double(mu) * mu
                           : (q < 0 ? double(J + mu) * (J - mu + 1) : double(J - mu) * (J + mu + 1));
            } else if (ju == jl + 1) {  // J_u = J_l + 1
                s = q == 0 ? double(J) * J - double(mu) * mu
                           : (q < 0 ? double(J + mu) * (J + mu - 1) : double(J - mu) * (J - mu - 1));
            } else {  // J_u = J_l - 1
                s = q == 0 ? double(J + 1) * (J + 1) - double(mu) * mu
                           : (q < 0 ? double(J - mu + 1) * (J - mu + 2) : double(J + mu + 1) * (J + mu + 2));
            }
            if (s <= 0.0) continue;
            sh[gi][n[gi]] = gl * ml - gu * mu;
            st[gi][n[gi]] = s;
            tot += s;
            ++n[gi];
        }
        for (int i = 0; i < n[gi]; ++i) st[gi][i] /= tot;
    }
    return ME_OK;
}

int npar_of(const me_problem *pb) { return ME_NPAR + (pb && pb->fill_fraction ? 1 : 0); }

int check_bounds(const me_bounds *b, int npar)
{
    if (!b) return fail(ME_EINVAL, "bounds is NULL");
    for (int d = 0; d < npar; ++d)
        if (!std::isfinite(b->lo[d]) || !std::isfinite(b->hi[d]) || b->lo[d] > b->hi[d])
            return fail(ME_EINVAL, "bounds must be finite with lo <= hi");
    if (b->lo[5] < 0.0) return fail(ME_EINVAL, "damping lower bound must be >= 0");
    if (!(b->lo[4] > 0.0)) return fail(ME_EINVAL, "Doppler-width lower bound must be > 0");
    if (npar > ME_NPAR && (b->lo[ME_NPAR] < 0.0 || b->hi[ME_NPAR] > 1.0))
        return fail(ME_EINVAL, "fill-fraction bounds must lie in [0, 1]");
    return ME_OK;
}

// floor(p 2^32) compared with a uniform u32: p >= 1 -> 2^32, p <= 0 -> 0.
uint64_t prob_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 1ull << 32;
    return (uint64_t)std::floor(p * 4294967296.0);
}

int make_ga(const ga_config *cfg, const me_bounds *b, uint64_t pid0, KGa &g, int npar)
{
    if (!cfg) return fail(ME_EINVAL, "ga_config is NULL");
    if (cfg->npop < ME_MIN_POP || cfg->npop > ME_MAX_POP || cfg->npop % 32)
        return fail(ME_EINVAL, "npop must be a multiple of 32 in [32, 1024]");
    if (cfg->ngen < 0) return fail(ME_EINVAL, "ngen must be >= 0");
    if (!std::isfinite(cfg->pc) || !std::isfinite(cfg->pmut_lsb) || !std::isfinite(cfg->pmut_ratio) ||
        cfg->pmut_ratio < 0.0)
        return fail(ME_EINVAL, "invalid GA probabilities");
    if (cfg->weight_mode != ME_W_INVMAX && cfg->weight_mode != ME_W_USER)
        return fail(ME_EINVAL, "weight_mode must be ME_W_INVMAX or ME_W_USER");
    std::memset(&g, 0, sizeof g);
    g.npop = cfg->npop;
    g.ngen = cfg->ngen;
    g.nsamp = cfg->nsamp;
    g.weight_mode = cfg->weight_mode;
    g.seed = cfg->seed;
    g.pixel_id0 = pid0;
    philox_round_keys(cfg->seed, g.rk);
    g.t_cross = prob_threshold(cfg->pc);
    // bit b (0 = MSB) flips with q_b = pmut_lsb ratio^(15 - b), clamped to [0, 1];
    // t_mut holds the chance of a flip among bits c..b, for the mutation's jumps
    double q[16];
    for (int bit = 0; bit < 16; ++bit) {
        double r = 1.0;
        for (int k = 0; k < 15 - bit; ++k) r *= cfg->pmut_ratio;
        const double p = cfg->pmut_lsb * r;
        q[bit] = p > 0.0 ? (p < 1.0 ? p : 1.0) : 0.0;
    }
    for (int b = 0; b < 16; ++b) {
        double keep = 1.0;  // no flip among bits c..b
        for (int c = b; c >= 0; --c) {
            keep *= 1.0 - q[c];
            g.t_mut[b * (b + 1) / 2 + c] = prob_threshold(1.0 - keep);
        }
    }
    if (b) {
        for (int d = 0; d < npar; ++d) {
            g.lo[d] = b->lo[d];
            g.hi[d] = b->hi[d];
        }
    }
    return ME_OK;
}

cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

int set_error(int code, const std::string &msg) { return fail(code, msg); }

int cuda_error(cudaError_t e, const char *where) { return cuda_fail(e, where); }

const HostTables &host_tables()
{
    static HostTables t = build_tables();
    return t;
}

}  // namespace genesis

using namespace genesis;

extern "C" {

const char *me_last_error(void) { return g_last_error.c_str(); }

int me_version(void) { return 103; }

int me_zeeman_components(const me_line *line, int n[3], double shift[3][ME_MAX_COMP],
                         double strength[3][ME_MAX_COMP])
{
    if (!line || !n || !shift || !strength) return fail(ME_EINVAL, "NULL argument");
    if (line->pattern) return zeeman_pattern(line->j_lower, line->g_lower, line->j_upper, line->g_upper,
                                             n, shift, strength);
    for (int g = 0; g < 3; ++g) {
        n[g] = 1;
        shift[g][0] = (g - 1) * line->g_eff;
        strength[g][0] = 1.0;
    }
    return ME_OK;
}

int me_synth(const me_problem *pb, const double *params, const double *mu_px, int n, void *stokes,
             void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    if (n < 0) return fail(ME_EINVAL, "n must be >= 0");
    if (n == 0) return ME_OK;
    if (!params || !stokes) return fail(ME_EINVAL, "params and stokes must be non-NULL");
    if ((long long)n * pb->n_lambda > (1ll << 31) - 1) return fail(ME_EINVAL, "n * n_lambda too large");
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_synth(k, pb->dtype, params, mu_px, n, stokes, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_synth launch");
}

int me_synth_jac(const me_problem *pb, const double *params, const double *mu_px, int n,
                 void *stokes, void *jac, void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    if (n < 0) return fail(ME_EINVAL, "n must be >= 0");
    if (n == 0) return ME_OK;
    if (!params || !jac) return fail(ME_EINVAL, "params and jac must be non-NULL");
    if ((long long)n * pb->n_lambda > (1ll << 31) - 1) return fail(ME_EINVAL, "n * n_lambda too large");
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_jac(k, pb->dtype, params, mu_px, n, stokes, jac, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_synth_jac launch");
}

int me_synth_vjp(const me_problem *pb, const double *params, const double *mu_px, int n,
                 const void *grad_stokes, double *grad_params, void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    if (n < 0) return fail(ME_EINVAL, "n must be >= 0");
    if (n == 0) return ME_OK;
    if (!params || !grad_stokes || !grad_params)
        return fail(ME_EINVAL, "params, grad_stokes and grad_params must be non-NULL");
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_vjp(k, pb->dtype, params, mu_px, n, grad_stokes, grad_params, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_synth_vjp launch");
}

int me_chi2(const me_problem *pb, const void *obs, const double *w, const double *mu_px, int npix,
            const double *params, double *chi2, void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    if (npix < 0) return fail(ME_EINVAL, "npix must be >= 0");
    if (npix == 0) return ME_OK;
    if (!obs || !params || !chi2) return fail(ME_EINVAL, "obs, params and chi2 must be non-NULL");
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_chi2_f64(k, pb->dtype, obs, w, mu_px, npix, params, chi2, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_chi2 launch");
}

static int ga_invert_impl(const me_problem *pb, const void *obs, const double *w, const double *mu_px,
                          int npix, uint64_t pixel_id0, const me_bounds *bounds, const ga_config *cfg,
                          KSeed sd, KSub sub, double *best, double *chi2, uint16_t *best_genes,
                          void *stream, const char *who)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    const int npar = npar_of(pb);
    if ((rc = check_bounds(bounds, npar))) return rc;
    KGa g;
    if ((rc = make_ga(cfg, bounds, pixel_id0, g, npar))) return rc;
    if (npix < 0) return fail(ME_EINVAL, "npix must be >= 0");
    if (npix == 0) return ME_OK;
    if (!obs || !best || !chi2) return fail(ME_EINVAL, "obs, best and chi2 must be non-NULL");
    if (cfg->weight_mode == ME_W_USER && !w) return fail(ME_EINVAL, "ME_W_USER needs w");
    if (pixel_id0 + (uint64_t)npix < pixel_id0) return fail(ME_EINVAL, "pixel id range overflows");
    if (sd.nseed < 0 || sd.nseed > cfg->npop / 2) return fail(ME_EINVAL, "nseed must be in [0, npop / 2]");
    if (sd.nseed > 0 && !sd.seeds) return fail(ME_EINVAL, "nseed > 0 needs seeds");
    // shared memory: obs + offsets + fitness + genes must fit one block
    const size_t rs = pb->dtype == ME_F32 ? 4 : 8;
    const size_t need = rs * (4 + pb->n_lines) * pb->n_lambda + rs * (cfg->npop + 72) + 128 +
                        (size_t)4 * cfg->npop * npar + 256;
    if (need > 220 * 1024) return fail(ME_EINVAL, "population and grid exceed shared memory");
    if ((rc = ensure_device())) return rc;
    const KGa &gc = g;
    const double *wu = cfg->weight_mode == ME_W_USER ? w : nullptr;
    cudaError_t e = launch_ga_evolve(k, gc, pb->dtype, obs, wu, mu_px, npix, best, best_genes,
                                     as_stream(stream), sd, sub);
    if (e != cudaSuccess) return cuda_fail(e, who);
    e = launch_chi2_f64(k, pb->dtype, obs, wu, mu_px, npix, best, chi2, as_stream(stream), sub);
    return e == cudaSuccess ? ME_OK : cuda_fail(e, who);
}

int ga_invert_batch(const me_problem *pb, const void *obs, const double *w, const double *mu_px,
                    int npix, uint64_t pixel_id0, const me_bounds *bounds, const ga_config *cfg,
                    double *best, double *chi2, uint16_t *best_genes, void *stream)
{
    return ga_invert_impl(pb, obs, w, mu_px, npix, pixel_id0, bounds, cfg, KSeed{}, KSub{}, best, chi2,
                          best_genes, stream, "ga_invert_batch launch");
}

int ga_invert_subset(const me_problem *pb, const void *obs, const double *w, const double *mu_px,
                     int npix, uint64_t pixel_id0, const me_bounds *bounds, const ga_config *cfg,
                     const double *seeds, int nseed, const int *polarity, const double *bounds_px,
                     const int *index, const int *count, double *best, double *chi2, uint16_t *best_genes,
                     void *stream)
{
    return ga_invert_impl(pb, obs, w, mu_px, npix, pixel_id0, bounds, cfg,
                          KSeed{seeds, nseed, polarity, bounds_px},
                          KSub{index, count}, best, chi2, best_genes, stream, "ga_invert_subset launch");
}

int ga_count_evaluations(const me_problem *pb, const void *obs, const double *w,
                         const double *mu_px, int npix, uint64_t pixel_id0,
                         const me_bounds *bounds, const ga_config *cfg, double *best,
                         unsigned long long *counts, void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    const int npar = npar_of(pb);
    if ((rc = check_bounds(bounds, npar))) return rc;
    KGa g;
    if ((rc = make_ga(cfg, bounds, pixel_id0, g, npar))) return rc;
    if (pb->dtype != ME_F32 || cfg->npop > 256)
        return fail(ME_EINVAL, "counting runs support float cubes with npop <= 256");
    if (npix < 0) return fail(ME_EINVAL, "npix must be >= 0");
    if (npix == 0) return ME_OK;
    if (!obs || !best || !counts) return fail(ME_EINVAL, "obs, best and counts must be non-NULL");
    if (cfg->weight_mode == ME_W_USER && !w) return fail(ME_EINVAL, "ME_W_USER needs w");
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_ga_count(k, g, pb->dtype, obs, cfg->weight_mode == ME_W_USER ? w : nullptr,
                                    mu_px, npix, best, counts, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "ga_count_evaluations launch");
}

int ga_fitness(const me_problem *pb, const void *obs, const double *w, const double *mu_px, int npix, int npop,
               int nactive, const double *params, double *fitness, void *resid, void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    if (npix < 0) return fail(ME_EINVAL, "npix must be >= 0");
    if (npop < ME_MIN_POP || npop > ME_MAX_POP || npop % 32)
        return fail(ME_EINVAL, "npop must be a multiple of 32 in [32, 1024]");
    if (nactive < 1 || nactive > npop) return fail(ME_EINVAL, "nactive must be in [1, npop]");
    if (npix == 0) return ME_OK;
    if (!obs || !params || !fitness) return fail(ME_EINVAL, "obs, params and fitness must be non-NULL");
    const size_t rs = pb->dtype == ME_F32 ? 4 : 8;
    const size_t need = rs * (4 + pb->n_lines) * pb->n_lambda + rs * (npop + 72) + 128 +
                        (size_t)4 * npop * npar_of(pb) + 256;
    if (need > 220 * 1024) return fail(ME_EINVAL, "population and grid exceed shared memory");
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_ga_fitness(k, pb->dtype, w ? ME_W_USER : ME_W_INVMAX, obs, w, mu_px, npix, npop, nactive,
                                      params, fitness, resid, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "ga_fitness launch");
}

int me_faddeeva_pairs(const float *x, const float *a, const float *v_b, int n, int mode, float *out, void *stream)
{
    if (n < 0) return fail(ME_EINVAL, "n must be >= 0");
    if (mode < 0 || mode > 2) return fail(ME_EINVAL, "mode must be 0, 1 or 2");
    if (n == 0) return ME_OK;
    if (!x || !a || !out || (mode == 2 && !v_b)) return fail(ME_EINVAL, "NULL argument");
    if (((uintptr_t)x) & 7) return fail(ME_EINVAL, "x must be 8-byte aligned");
    int rc = ensure_device();
    if (rc) return rc;
    cudaError_t e = launch_fad_probe(x, a, v_b, n, mode, out, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_faddeeva_pairs launch");
}

int me_fp32_peak(int packed, int nblocks, int iters, float *out, double *flops, void *stream)
{
    if (nblocks < 1 || iters < 1) return fail(ME_EINVAL, "nblocks and iters must be >= 1");
    if (!out) return fail(ME_EINVAL, "out must be non-NULL");
    int rc = ensure_device();
    if (rc) return rc;
    if (flops) *flops = fma_peak_flops(packed, nblocks, iters);
    cudaError_t e = launch_fma_peak(packed, nblocks, iters, out, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_fp32_peak launch");
}

static int lm_polish_impl(const me_problem *pb, const void *obs, const double *w, const double *mu_px,
                          int npix, const me_bounds *bounds, int iters, double lambda0, unsigned free_mask,
                          KSub sub, double *params_inout, double *chi2_out, void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    const int npar = npar_of(pb);
    if ((rc = check_bounds(bounds, npar))) return rc;
    if (npix < 0 || iters < 0) return fail(ME_EINVAL, "npix and iters must be >= 0");
    if (!(lambda0 > 0.0) || !std::isfinite(lambda0)) return fail(ME_EINVAL, "lambda0 must be positive");
    if (npix == 0) return ME_OK;
    if (!obs || !params_inout) return fail(ME_EINVAL, "obs and params_inout must be non-NULL");
    if ((rc = ensure_device())) return rc;
    KLm lm;
    std::memset(&lm, 0, sizeof lm);
    lm.iters = iters;
    lm.lambda0 = lambda0;
    lm.free_mask = free_mask & ((1u << npar) - 1u);
    for (int d = 0; d < npar; ++d) {
        lm.lo[d] = bounds->lo[d];
        lm.hi[d] = bounds->hi[d];
    }
    cudaError_t e = launch_lm(k, lm, pb->dtype, obs, w, mu_px, npix, params_inout, as_stream(stream), sub);
    if (e != cudaSuccess) return cuda_fail(e, "lm_polish launch");
    if (chi2_out) {
        e = launch_chi2_f64(k, pb->dtype, obs, w, mu_px, npix, params_inout, chi2_out, as_stream(stream), sub);
        if (e != cudaSuccess) return cuda_fail(e, "lm_polish chi2 launch");
    }
    return ME_OK;
}

int lm_polish(const me_problem *pb, const void *obs, const double *w, const double *mu_px, int npix,
              const me_bounds *bounds, int iters, double lambda0, double *params_inout,
              double *chi2_out, void *stream)
{
    return lm_polish_impl(pb, obs, w, mu_px, npix, bounds, iters, lambda0, ~0u, KSub{},
                          params_inout, chi2_out, stream);
}

int lm_fit(const me_problem *pb, const void *obs, const double *w, const double *mu_px, int npix,
           const me_bounds *bounds, int iters, double lambda0, unsigned free_mask, const int *index,
           const int *count, double *params_inout, double *chi2_out, void *stream)
{
    return lm_polish_impl(pb, obs, w, mu_px, npix, bounds, iters, lambda0, free_mask, KSub{index, count},
                          params_inout, chi2_out, stream);
}

int me_prefit_bounds(const double *p_hat, int npix, int npar, const me_bounds *bounds, const double *lower,
                     const double *upper, double *bounds_px, void *stream)
{
    if (npar != ME_NPAR && npar != ME_NPAR_MAX) return fail(ME_EINVAL, "npar must be ME_NPAR or ME_NPAR_MAX");
    int rc = check_bounds(bounds, npar);
    if (rc) return rc;
    if (npix < 0) return fail(ME_EINVAL, "npix must be >= 0");
    if (!lower || !upper) return fail(ME_EINVAL, "lower and upper margins must be non-NULL");
    if (npix == 0) return ME_OK;
    if (!p_hat || !bounds_px) return fail(ME_EINVAL, "p_hat and bounds_px must be non-NULL");
    if ((size_t)npix * npar > (size_t)INT32_MAX) return fail(ME_EINVAL, "npix too large");
    KPrefitBounds r;
    std::memset(&r, 0, sizeof r);
    r.npar = npar;
    for (int k = 0; k < npar; ++k) {
        if (std::isnan(lower[k]) || std::isnan(upper[k])) return fail(ME_EINVAL, "margins must not be NaN");
        r.lo[k] = bounds->lo[k];
        r.hi[k] = bounds->hi[k];
        r.lower[k] = lower[k];
        r.upper[k] = upper[k];
    }
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_prefit_bounds(p_hat, npix, r, bounds_px, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_prefit_bounds launch");
}

int me_classify(const me_problem *pb, const void *obs, int npix, double p_thresh, int q_lo, int q_hi,
                int line, int c_lo, int c_hi, int *flag, int *polarity, double *pol, double *weak,
                double *seeds, double *best, void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    if (npix < 0) return fail(ME_EINVAL, "npix must be >= 0");
    if (!(p_thresh >= 0.0) || !std::isfinite(p_thresh)) return fail(ME_EINVAL, "p_thresh must be finite, >= 0");
    if (q_lo < 0 || q_hi > pb->n_lambda || q_lo >= q_hi) return fail(ME_EINVAL, "quiet window out of range");
    if (c_lo < 0 || c_hi >= pb->n_lambda || c_lo > c_hi) return fail(ME_EINVAL, "line window out of range");
    if (line < 0 || line >= pb->n_lines) return fail(ME_EINVAL, "line out of range");
    if (npix == 0) return ME_OK;
    if (!obs) return fail(ME_EINVAL, "obs must be non-NULL");
    if ((rc = ensure_device())) return rc;
    KClassify c;
    c.p_thresh = p_thresh;
    c.kz = k.line[line].zfac;
    c.q_lo = q_lo;
    c.q_hi = q_hi;
    c.c_lo = c_lo;
    c.c_hi = c_hi;
    c.flag = flag;
    c.polarity = polarity;
    c.pol = pol;
    c.weak = weak;
    c.seeds = seeds;
    c.best = best;
    c.npar = npar_of(pb);
    cudaError_t e = launch_classify(k, pb->dtype, obs, npix, c, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_classify launch");
}

size_t me_select_scratch_bytes(int npix) { return select_scratch_bytes(npix); }

int me_select(const int *flag, int npix, int want, int *index, int *count, void *scratch,
              size_t scratch_bytes, void *stream)
{
    if (npix < 0) return fail(ME_EINVAL, "npix must be >= 0");
    if (!count) return fail(ME_EINVAL, "count must be non-NULL");
    if (npix > 0 && (!flag || !index || !scratch)) return fail(ME_EINVAL, "flag, index and scratch must be non-NULL");
    if (scratch_bytes < select_scratch_bytes(npix)) return fail(ME_EINVAL, "scratch smaller than me_select_scratch_bytes");
    if (((uintptr_t)scratch & 3) != 0) return fail(ME_EINVAL, "scratch must be 4-byte aligned");
    int rc = ensure_device();
    if (rc) return rc;
    cudaError_t e = launch_select(flag, npix, want, index, count, scratch, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_select launch");
}

int me_select_static(const int *flag, int npix, int want, int *index, int *count, void *stream)
{
    if (npix < 0 || npix > ME_SELECT_STATIC_MAX_PIX)
        return fail(ME_EINVAL, "npix must be in [0, ME_SELECT_STATIC_MAX_PIX]");
    if (!count) return fail(ME_EINVAL, "count must be non-NULL");
    if (npix > 0 && (!flag || !index)) return fail(ME_EINVAL, "flag and index must be non-NULL");
    int rc = ensure_device();
    if (rc) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (g_select_static_bytes < select_scratch_bytes(npix)) return fail(ME_EINVAL, "static scratch too small");
    e = launch_select(flag, npix, want, index, count, g_select_static[dev], as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_select_static launch");
}

int lm_uncertainty(const me_problem *pb, const void *obs, const double *w, const double *mu_px,
                   int npix, const double *params, double *sigma, void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    if (npix < 0) return fail(ME_EINVAL, "npix must be >= 0");
    if (npix == 0) return ME_OK;
    if (!obs || !params || !sigma) return fail(ME_EINVAL, "obs, params and sigma must be non-NULL");
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_lm_sigma(k, pb->dtype, obs, w, mu_px, npix, params, sigma, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "lm_uncertainty launch");
}

int me_line_centre(const me_problem *pb, const void *obs, int npix, int half_width, int i_lo,
                   int i_hi, double *lambda_c, int *index, void *stream)
{
    KProblem k;
    int rc = make_problem(pb, k);
    if (rc) return rc;
    if (npix < 0 || half_width < 1) return fail(ME_EINVAL, "need npix >= 0 and half_width >= 1");
    if (npix == 0) return ME_OK;
    if (!obs || !lambda_c) return fail(ME_EINVAL, "obs and lambda_c must be non-NULL");
    const int lo = std::max(i_lo, half_width), hi = std::min(i_hi, pb->n_lambda - 1 - half_width);
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_line_centre(k, pb->dtype, obs, npix, half_width, lo, hi, lambda_c, index,
                                       as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_line_centre launch");
}

int ga_breed(const uint16_t *genes, const double *fitness, int nprob, int npop, int npar, uint64_t pixel_id0,
             int gen, const ga_config *cfg, uint16_t *child, int *elite, void *stream)
{
    KGa g;
    ga_config c = cfg ? *cfg : ga_config{};
    if (!cfg) return fail(ME_EINVAL, "ga_config is NULL");
    if (npar != ME_NPAR && npar != ME_NPAR_MAX) return fail(ME_EINVAL, "npar must be ME_NPAR or ME_NPAR_MAX");
    c.npop = npop;
    int rc = make_ga(&c, nullptr, pixel_id0, g, npar);
    if (rc) return rc;
    if (nprob < 0) return fail(ME_EINVAL, "nprob must be >= 0");
    if (nprob == 0) return ME_OK;
    if (!genes || !fitness || !child) return fail(ME_EINVAL, "genes, fitness and child must be non-NULL");
    if ((rc = ensure_device())) return rc;
    cudaError_t e = launch_ga_breed(g, npar, genes, fitness, nprob, gen, child, elite, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "ga_breed launch");
}

int ga_restart(uint16_t *genes, const double *fitness, int nprob, int npop, int npar, uint64_t sobol_next,
               void *stream)
{
    if (npop < ME_MIN_POP || npop > ME_MAX_POP || npop % 32)
        return fail(ME_EINVAL, "npop must be a multiple of 32 in [32, 1024]");
    if (npar != ME_NPAR && npar != ME_NPAR_MAX) return fail(ME_EINVAL, "npar must be ME_NPAR or ME_NPAR_MAX");
    if (nprob < 0) return fail(ME_EINVAL, "nprob must be >= 0");
    if (nprob == 0) return ME_OK;
    if (!genes || !fitness) return fail(ME_EINVAL, "genes and fitness must be non-NULL");
    if (sobol_next + (uint64_t)npop > (1ull << 32)) return fail(ME_EINVAL, "Sobol index beyond 2^32");
    int rc = ensure_device();
    if (rc) return rc;
    cudaError_t e = launch_ga_restart(npop, npar, genes, fitness, nprob, sobol_next, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "ga_restart launch");
}

int me_philox(const uint32_t *ctr, int n, uint64_t key, uint32_t *out, void *stream)
{
    if (n < 0) return fail(ME_EINVAL, "n must be >= 0");
    if (n == 0) return ME_OK;
    if (!ctr || !out) return fail(ME_EINVAL, "ctr and out must be non-NULL");
    int rc = ensure_device();
    if (rc) return rc;
    cudaError_t e = launch_philox(ctr, n, key, out, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_philox launch");
}

int me_sobol(uint64_t first, int n, int ndim, uint32_t *out, void *stream)
{
    if (n < 0 || ndim < 1 || ndim > 10) return fail(ME_EINVAL, "need n >= 0 and 1 <= ndim <= 10");
    if (n == 0) return ME_OK;
    if (!out) return fail(ME_EINVAL, "out must be non-NULL");
    if (first + (uint64_t)n > (1ull << 32)) return fail(ME_EINVAL, "Sobol index beyond 2^32");
    if ((long long)n * ndim > (1ll << 31) - 1) return fail(ME_EINVAL, "n * ndim too large");
    int rc = ensure_device();
    if (rc) return rc;
    cudaError_t e = launch_sobol(first, n, ndim, out, as_stream(stream));
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_sobol launch");
}

}  // extern "C"
