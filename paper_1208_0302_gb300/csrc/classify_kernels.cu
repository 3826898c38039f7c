// Section 2 pixel selection and weak-field fallback, Section 5.5 seeds and
// polarity, and the order-preserving selection of the pixels to invert.
#include "kernels.h"

namespace genesis {

namespace {

constexpr int kClassifyBlock = 128;  // four pixels (one warp each) per block
constexpr int kSelectTile = 2048;    // flags per selection tile
constexpr int kSelectBlock = 256;    // threads per selection block, 8 flags each
constexpr double kPi = 3.14159265358979323846;

// Tile counts of me_select_static: a file-scope device array sized for
// ME_SELECT_STATIC_MAX_PIX flags (8192 tiles, 32 KiB).  Every slot a call uses
// is written by its count pass before the scan reads it, so nothing has to
// start at zero; concurrent calls share it and therefore race.
static __device__ __align__(256) int g_select_tiles[(ME_SELECT_STATIC_MAX_PIX + kSelectTile - 1) / kSelectTile];

// One pixel's Stokes rows as FP64 values.
template <class RO> struct Rows {
    const RO *o;
    int nl;
    __device__ __forceinline__ double at(int s, int j) const { return (double)o[s * nl + j]; }
};

// Three-point parabola vertex through (x0, y0), (x1, y1), (x2, y2), without
// contraction; x1 when the points are collinear.
__device__ __forceinline__ double vertex3(double x0, double x1, double x2, double y0, double y1, double y2)
{
    const double d0 = __dsub_rn(x1, x0), d2 = __dsub_rn(x1, x2);
    const double e0 = __dsub_rn(y1, y0), e2 = __dsub_rn(y1, y2);
    const double num = __dsub_rn(__dmul_rn(__dmul_rn(d0, d0), e2), __dmul_rn(__dmul_rn(d2, d2), e0));
    const double den = __dsub_rn(__dmul_rn(d0, e2), __dmul_rn(d2, e0));
    return den != 0.0 ? __dsub_rn(x1, __ddiv_rn(__dmul_rn(0.5, num), den)) : x1;
}

// Three-point second difference of Stokes row s at interior point c on the
// (possibly non-uniform) grid.
template <class RO>
__device__ __forceinline__ double second_diff(const double *lam, const Rows<RO> &r, int s, int c)
{
    const double h1 = __dsub_rn(lam[c], lam[c - 1]), h2 = __dsub_rn(lam[c + 1], lam[c]);
    const double y0 = r.at(s, c - 1), y1 = r.at(s, c), y2 = r.at(s, c + 1);
    const double num = __dmul_rn(2.0, __dsub_rn(__dmul_rn(h1, __dsub_rn(y2, y1)), __dmul_rn(h2, __dsub_rn(y1, y0))));
    return __ddiv_rn(num, __dmul_rn(__dmul_rn(h1, h2), __dadd_rn(h1, h2)));
}

// Trapezoid weight of point j in the window [lo, hi].
__device__ __forceinline__ double trap_w(const double *lam, int lo, int hi, int j)
{
    if (lo == hi) return 0.0;
    const double a = j > lo ? __dsub_rn(lam[j], lam[j - 1]) : 0.0;
    const double b = j < hi ? __dsub_rn(lam[j + 1], lam[j]) : 0.0;
    return __dmul_rn(0.5, __dadd_rn(a, b));
}

__device__ __forceinline__ double degrees(double rad) { return __ddiv_rn(__dmul_rn(rad, 180.0), kPi); }

// A seed (B, psi, chi) from B_par and B_perp, psi reflected into the pixel's
// polarity half.
__device__ __forceinline__ void put_seed(double *sd, double bpar, double bperp, double chi, int pol)
{
    double psi = degrees(atan2(bperp, bpar));
    if ((pol > 0 && psi > 90.0) || (pol < 0 && psi < 90.0)) psi = __dsub_rn(180.0, psi);
    sd[0] = __dsqrt_rn(__dadd_rn(__dmul_rn(bpar, bpar), __dmul_rn(bperp, bperp)));
    sd[1] = psi;
    sd[2] = chi;
}

// Warp argmin (want_max = false) or argmax of v with ties to the lowest index.
__device__ __forceinline__ void warp_arg(double &v, int &i, bool want_max)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, off);
        const int oi = __shfl_xor_sync(0xffffffffu, i, off);
        const bool better = want_max ? (ov > v) : (ov < v);
        if (better || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
}

// Section 2 threshold, weak-field estimate, polarity and seeds: one warp per
// pixel, FP64 throughout.  Extrema are lane-parallel (exact); each running
// sum is taken by one lane in increasing index, so every result except the
// angles (atan2) repeats the plain sequential evaluation bit for bit.
template <class RO>
__global__ void __launch_bounds__(kClassifyBlock)
k_classify(const __grid_constant__ KProblem pb, const RO *__restrict__ obs, int npix, const KClassify c)
{
    const int lane = threadIdx.x & 31;
    const int pix = blockIdx.x * (kClassifyBlock / 32) + (threadIdx.x >> 5);
    if (pix >= npix) return;
    const int nl = pb.n_lambda;
    const double *lam = pb.lam;
    const Rows<RO> r{obs + (size_t)pix * 4 * nl, nl};
    const int lo = c.c_lo, hi = c.c_hi;

    // extrema: |Q|, |U|, |V| over the grid; the I+V, I-V cores and the V
    // lobes over the line window
    double qx = 0.0, ux = 0.0, vx = 0.0;
    for (int j = lane; j < nl; j += 32) {
        qx = fmax(qx, fabs(r.at(1, j)));
        ux = fmax(ux, fabs(r.at(2, j)));
        vx = fmax(vx, fabs(r.at(3, j)));
    }
    double vp = INFINITY, vm = INFINITY, vhi = -INFINITY, vlo = INFINITY;
    int ip = hi + 1, im = hi + 1, jhi = hi + 1, jlo = hi + 1;
    for (int j = lo + lane; j <= hi; j += 32) {
        const double I = r.at(0, j), V = r.at(3, j);
        const double a = __dadd_rn(I, V), b = __dsub_rn(I, V);
        if (a < vp) { vp = a; ip = j; }
        if (b < vm) { vm = b; im = j; }
        if (V > vhi) { vhi = V; jhi = j; }
        if (V < vlo) { vlo = V; jlo = j; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        qx = fmax(qx, __shfl_xor_sync(0xffffffffu, qx, off));
        ux = fmax(ux, __shfl_xor_sync(0xffffffffu, ux, off));
        vx = fmax(vx, __shfl_xor_sync(0xffffffffu, vx, off));
    }
    warp_arg(vp, ip, false);
    warp_arg(vm, im, false);
    warp_arg(vhi, jhi, true);
    warp_arg(vlo, jlo, false);

    // sequential sums, one per lane
    const int nq = c.q_hi - c.q_lo;
    double acc = 0.0, acc2 = 0.0;
    if (lane < 4) {  // quiet-window mean (and, for Q, U, V, variance)
        for (int j = c.q_lo; j < c.q_hi; ++j) acc = __dadd_rn(acc, r.at(lane, j));
        acc = __ddiv_rn(acc, (double)nq);
        if (lane > 0) {
            for (int j = c.q_lo; j < c.q_hi; ++j) {
                const double d = __dsub_rn(r.at(lane, j), acc);
                acc2 = __dadd_rn(acc2, __dmul_rn(d, d));
            }
            acc2 = __ddiv_rn(acc2, (double)nq);
        }
    } else if (lane < 7) {  // least-squares sums of Q I'', U I'', I''^2
        for (int j = lo > 1 ? lo : 1; j <= hi && j + 1 < nl; ++j) {
            const double d2 = second_diff(lam, r, 0, j);
            const double y = lane == 6 ? d2 : r.at(lane - 3, j);
            acc = __dadd_rn(acc, __dmul_rn(y, d2));
        }
    } else if (lane < 9) {  // trapezoid integrals of |V| and L
        for (int j = lo; j <= hi; ++j) {
            const double wj = trap_w(lam, lo, hi, j);
            double y;
            if (lane == 7) {
                y = fabs(r.at(3, j));
            } else {
                const double q = r.at(1, j), u = r.at(2, j);
                y = __dsqrt_rn(__dadd_rn(__dmul_rn(q, q), __dmul_rn(u, u)));
            }
            acc = __dadd_rn(acc, __dmul_rn(wj, y));
        }
    } else if (lane == 9) {  // total variation of I
        for (int j = lo; j < hi; ++j) acc = __dadd_rn(acc, fabs(__dsub_rn(r.at(0, j + 1), r.at(0, j))));
    } else if (lane == 10) {  // total variation of I'
        for (int j = lo + 1; j < hi; ++j) {
            const double sl = __ddiv_rn(__dsub_rn(r.at(0, j + 1), r.at(0, j)), __dsub_rn(lam[j + 1], lam[j]));
            const double sr = __ddiv_rn(__dsub_rn(r.at(0, j), r.at(0, j - 1)), __dsub_rn(lam[j], lam[j - 1]));
            acc = __dadd_rn(acc, fabs(__dsub_rn(sl, sr)));
        }
    }
    const double ic = __shfl_sync(0xffffffffu, acc, 0);
    if (lane >= 11 && lane < 15) {  // centre-of-gravity moments of I_c - (I +- V)
        const bool plus = lane < 13, moment = (lane & 1) != 0;
        for (int j = lo; j <= hi; ++j) {
            const double wj = trap_w(lam, lo, hi, j);
            const double I = r.at(0, j), V = r.at(3, j);
            const double a = __dmul_rn(wj, __dsub_rn(ic, plus ? __dadd_rn(I, V) : __dsub_rn(I, V)));
            acc = __dadd_rn(acc, moment ? __dmul_rn(a, lam[j]) : a);
        }
    }
    double v[16], v2[4];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __shfl_sync(0xffffffffu, acc, q);
#pragma unroll
    for (int q = 0; q < 4; ++q) v2[q] = __shfl_sync(0xffffffffu, acc2, q);
    if (lane != 0) return;

    // threshold
    const double p = __ddiv_rn(
        __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(ux, ux)), __dmul_rn(vx, vx))), ic);
    const double sp = __ddiv_rn(__dmul_rn(c.p_thresh, __dsqrt_rn(__dadd_rn(__dadd_rn(v2[1], v2[2]), v2[3]))), ic);
    const int flag = p > sp ? 1 : 0;
    const int pol = jhi < jlo ? 1 : (jhi > jlo ? -1 : 0);

    // weak field
    auto core = [&](int bi, bool plus) {
        if (bi - 1 < 0 || bi + 1 >= nl) return lam[bi];
        double y[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const double I = r.at(0, bi - 1 + t), V = r.at(3, bi - 1 + t);
            y[t] = plus ? __dadd_rn(I, V) : __dsub_rn(I, V);
        }
        return vertex3(lam[bi - 1], lam[bi], lam[bi + 1], y[0], y[1], y[2]);
    };
    const double two_kz = __dmul_rn(2.0, c.kz);
    const double bpar = __ddiv_rn(__dsub_rn(core(ip, true), core(im, false)), two_kz);
    const double qa = v[4], ub = v[5], dd = v[6];
    double chi = degrees(__dmul_rn(0.5, atan2(-ub, -qa)));
    if (chi < 0.0) chi = __dadd_rn(chi, 180.0);
    const double amp = __dsqrt_rn(__dadd_rn(__dmul_rn(qa, qa), __dmul_rn(ub, ub)));
    const double bperp = dd > 0.0 ? __ddiv_rn(__dsqrt_rn(__ddiv_rn(__dmul_rn(4.0, amp), dd)), c.kz) : 0.0;
    const double bmag = __dsqrt_rn(__dadd_rn(__dmul_rn(bpar, bpar), __dmul_rn(bperp, bperp)));
    const double theta = degrees(atan2(bperp, bpar));

    if (c.flag) c.flag[pix] = flag;
    if (c.polarity) c.polarity[pix] = pol;
    if (c.pol) {
        c.pol[(size_t)pix * 2] = p;
        c.pol[(size_t)pix * 2 + 1] = sp;
    }
    if (c.weak) {
        double *wo = c.weak + (size_t)pix * 5;
        wo[0] = bmag;
        wo[1] = theta;
        wo[2] = chi;
        wo[3] = bpar;
        wo[4] = bperp;
    }
    if (c.seeds) {
        double *sd = c.seeds + (size_t)pix * 12;
        put_seed(sd, bpar, bperp, chi, pol);
        const double av = v[7], al = v[8], tvi = v[9], tvd = v[10];
        const double bpi = tvi > 0.0 ? __ddiv_rn(__dmul_rn(pol < 0 ? -1.0 : 1.0, av), __dmul_rn(c.kz, tvi)) : 0.0;
        const double bti = tvd > 0.0 ? __ddiv_rn(__dsqrt_rn(__ddiv_rn(__dmul_rn(4.0, al), tvd)), c.kz) : 0.0;
        put_seed(sd + 3, bpi, bti, chi, pol);
        const double np = v[11], dp = v[12], nm = v[13], dm = v[14];
        const double bcog =
            (dp != 0.0 && dm != 0.0) ? __ddiv_rn(__dsub_rn(__ddiv_rn(np, dp), __ddiv_rn(nm, dm)), two_kz) : 0.0;
        put_seed(sd + 6, bcog, bperp, chi, pol);
        put_seed(sd + 9, bpar, bperp, chi, pol);
        sd[9] = 0.0;
    }
    if (c.best && !flag) {  // weak-field answer for the pixels below the threshold
        double *bo = c.best + (size_t)pix * c.npar;
        bo[0] = bmag;
        bo[1] = theta;
        bo[2] = chi;
        for (int d = 3; d < c.npar; ++d) bo[d] = __longlong_as_double(0x7ff8000000000000ll);
    }
}

// ------------------------------------------------------------- selection
// Three passes over tiles of kSelectTile flags: count per tile, exclusive
// scan of the tile counts (one block), and a scatter that re-counts inside
// each tile.  Each thread owns 8 consecutive flags, so indices come out in
// increasing order.

__device__ __forceinline__ int block_exclusive_scan(int x, int *s_warp, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < nw) s_warp[lane] = w;  // inclusive prefix over warps
    }
    __syncthreads();
    total = s_warp[nw - 1];
    const int base = warp > 0 ? s_warp[warp - 1] : 0;
    __syncthreads();  // s_warp may be reused by the caller
    return base + inc - x;
}

__device__ __forceinline__ int tile_flags(const int *flag, int npix, int want, int first, unsigned &bits)
{
    int n = 0;
    bits = 0;
#pragma unroll
    for (int e = 0; e < kSelectTile / kSelectBlock; ++e) {
        const int i = first + e;
        if (i < npix && flag[i] == want) {
            bits |= 1u << e;
            ++n;
        }
    }
    return n;
}

__global__ void __launch_bounds__(kSelectBlock)
k_select_count(const int *__restrict__ flag, int npix, int want, int *__restrict__ tile_count)
{
    __shared__ int s_warp[32];
    unsigned bits;
    const int first = blockIdx.x * kSelectTile + threadIdx.x * (kSelectTile / kSelectBlock);
    int total;
    block_exclusive_scan(tile_flags(flag, npix, want, first, bits), s_warp, total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_select_scan(int *__restrict__ tile, int ntiles, int *__restrict__ count)
{
    __shared__ int s_warp[32];
    const int per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int t0 = threadIdx.x * per, t1 = min(t0 + per, ntiles);
    int sum = 0;
    for (int t = t0; t < t1; ++t) sum += tile[t];
    int total;
    int off = block_exclusive_scan(sum, s_warp, total);
    for (int t = t0; t < t1; ++t) {
        const int n = tile[t];
        tile[t] = off;
        off += n;
    }
    if (threadIdx.x == 0) *count = total;
}

__global__ void __launch_bounds__(kSelectBlock)
k_select_scatter(const int *__restrict__ flag, int npix, int want, const int *__restrict__ tile_off,
                 int *__restrict__ index)
{
    __shared__ int s_warp[32];
    unsigned bits;
    const int first = blockIdx.x * kSelectTile + threadIdx.x * (kSelectTile / kSelectBlock);
    int total;
    int pos = tile_off[blockIdx.x] + block_exclusive_scan(tile_flags(flag, npix, want, first, bits), s_warp, total);
#pragma unroll
    for (int e = 0; e < kSelectTile / kSelectBlock; ++e)
        if (bits & (1u << e)) index[pos++] = first + e;
}

// Section 5.3 bound rule, one thread per (pixel, parameter): [max(lo,
// p - lower), min(hi, p + upper)], the global interval where that is empty
// or the prefit is NaN.
__global__ void k_prefit_bounds(const double *__restrict__ p_hat, int npix, const KPrefitBounds r,
                                double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int M = r.npar;
    if (i >= npix * M) return;
    const int pix = i / M, k = i - pix * M;
    const double p = p_hat[i];
    double a = __dsub_rn(p, r.lower[k]), b = __dadd_rn(p, r.upper[k]);
    if (!(a > r.lo[k])) a = r.lo[k];
    if (!(b < r.hi[k])) b = r.hi[k];
    if (!(a < b)) {
        a = r.lo[k];
        b = r.hi[k];
    }
    out[(size_t)pix * 2 * M + k] = a;
    out[(size_t)pix * 2 * M + M + k] = b;
}

}  // namespace

cudaError_t launch_prefit_bounds(const double *p_hat, int npix, const KPrefitBounds &r, double *out,
                                 cudaStream_t st)
{
    if (npix <= 0) return cudaSuccess;
    const int n = npix * r.npar;
    k_prefit_bounds<<<(n + 255) / 256, 256, 0, st>>>(p_hat, npix, r, out);
    return cudaGetLastError();
}

cudaError_t launch_classify(const KProblem &pb, int dtype, const void *obs, int npix, const KClassify &c,
                            cudaStream_t st)
{
    if (npix <= 0) return cudaSuccess;
    const int per = kClassifyBlock / 32;
    const int grid = (npix + per - 1) / per;
    if (dtype == ME_F32)
        k_classify<float><<<grid, kClassifyBlock, 0, st>>>(pb, (const float *)obs, npix, c);
    else
        k_classify<double><<<grid, kClassifyBlock, 0, st>>>(pb, (const double *)obs, npix, c);
    return cudaGetLastError();
}

cudaError_t select_static_scratch(void **ptr, size_t *bytes)
{
    *bytes = sizeof(g_select_tiles);
    return cudaGetSymbolAddress(ptr, g_select_tiles);
}

size_t select_scratch_bytes(int npix)
{
    const size_t ntiles = npix > 0 ? ((size_t)npix + kSelectTile - 1) / kSelectTile : 0;
    return ntiles * sizeof(int);
}

cudaError_t launch_select(const int *flag, int npix, int want, int *index, int *count, void *scratch,
                          cudaStream_t st)
{
    if (npix <= 0) return cudaMemsetAsync(count, 0, sizeof(int), st);
    const int ntiles = (npix + kSelectTile - 1) / kSelectTile;
    int *tile = (int *)scratch;
    k_select_count<<<ntiles, kSelectBlock, 0, st>>>(flag, npix, want, tile);
    k_select_scan<<<1, 1024, 0, st>>>(tile, ntiles, count);
    k_select_scatter<<<ntiles, kSelectBlock, 0, st>>>(flag, npix, want, tile, index);
    return cudaGetLastError();
}

}  // namespace genesis
