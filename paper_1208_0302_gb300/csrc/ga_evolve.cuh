// Fused genetic-algorithm inversion kernel template for sm_103a (Section 3,
// Algorithm 1; Section 5.6), shared by the translation units that instantiate
// it (9 parameters; 10 with the fill fraction of Section 5.2).
//
//
// One thread block per pixel, one thread per individual.  The pixel's
// observed Stokes profiles, its wavelength offsets, the population's uint16
// genotypes (double-buffered) and fitness stay in shared memory for all
// generations; no host round trip happens between generations.  Each thread
// walks the wavelength grid for its own individual, so every lane of a warp
// reads the same shared-memory word (broadcast) and the chi2 sum needs no
// cross-thread reduction.
#pragma once

#include <type_traits>

#include "kernels.h"
#include "me_pair.cuh"
#include "rng_device.cuh"

namespace genesis {
namespace {


// Per-thread work counts of the counting instantiation: the fitness
// evaluations' Faddeeva evaluations by region of their own point.
struct WorkCount {
    unsigned long long interior, mid, even2, far;
};

template <class R> __device__ __forceinline__ R clean_fit(R f)
{
    return f == f ? f : R(INFINITY);  // NaN ranks as +infinity
}

// Kahan-compensated accumulation of r^2.
template <class R> __device__ __forceinline__ void kahan_sq(R &s, R &c, R r)
{
    const R y = r * r - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
}

// Four consecutive R values of a 16-byte aligned shared-memory row.
__device__ __forceinline__ void load4(const float *p, float v[4])
{
    const float4 q = *(const float4 *)p;
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double *p, double v[4])
{
    const double2 a = *(const double2 *)p, b = *(const double2 *)(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Shared-memory layouts.  FP32: wavelength pairs (2p, 2p+1) interleaved for
// packed FP32x2 use, 8 values per pair: (I, I', Q, Q', U, U', V, V') and
// (d0, d0', d1, d1', d2, d2', d3, d3') for the per-line offsets; an odd grid
// repeats its last point as the partner of the last pair.  FP64: rows of 4
// per wavelength.
template <class R> __device__ __forceinline__ int obs_idx(int s, int j)
{
    return sizeof(R) == 4 ? (j >> 1) * 8 + s * 2 + (j & 1) : j * 4 + s;
}
template <class R> __device__ __forceinline__ int padded_lambda(int nl)
{
    return sizeof(R) == 4 ? (nl + 1) & ~1 : nl;
}

template <class R> struct GaDecode;
// The pixel's decode domain in shared memory (per-pixel bounds of Section
// 5.3 and the polarity restriction of Section 5.5 already applied):
// double lo[M], hi[M], then float lo[M], scale[M] = (hi - lo) / 65535.
struct DecodeDomain {
    double lo[ME_NPAR_MAX], hi[ME_NPAR_MAX];
    float lo32[ME_NPAR_MAX], sc32[ME_NPAR_MAX];
};
template <> struct GaDecode<float> {
    static __device__ __forceinline__ float get(const DecodeDomain &D, int d, uint16_t g)
    {
        return fmaf((float)g, D.sc32[d], D.lo32[d]);
    }
};
template <> struct GaDecode<double> {
    static __device__ __forceinline__ double get(const DecodeDomain &D, int d, uint16_t g)
    {
        return decode64(g, D.lo[d], D.hi[d]);
    }
};

// Eq. chisq for one individual, FP32 (or FP64) synthesis over the whole grid.
// s_obs rows are (I, Q, U, V) of one wavelength; s_doff rows hold
// lambda_j - lambda0_l for l = 0..3: one vector load each per wavelength.
// STORE (verification kernel only): res, when not NULL, receives the
// residuals O - S as [4][nl].
template <class R, int NL, bool COUNT, bool PAT, bool FILL, bool STORE = false>
__device__ __forceinline__ R fitness_rows(const KProblem &pb, int nlines, int nl, const R *p, R mu,
                                          const R *s_obs, const R *s_doff, const R *he,
                                          const R *s_w2, R inv_nu, WorkCount &wc,
                                          R *res = nullptr)
{
    const Geo<R> geo = make_geo<R, NL, FILL>(pb, nlines, p, mu);
    R sI = 0, sQ = 0, sU = 0, sV = 0, cI = 0, cQ = 0, cU = 0, cV = 0;
    for (int j = 0; j < nl; ++j) {
        R doff[4], ob[4];
        load4(s_doff + 4 * j, doff);
        load4(s_obs + 4 * j, ob);
        const Stokes4<R> s = me_point<R, NL, PAT, FILL>(geo, doff, he, nlines, pb.line);
        if (COUNT) wc.interior += count_interior<R, NL, PAT>(geo, doff, nlines, pb.line);
        if (STORE && res) {
            res[j] = ob[0] - s.I;
            res[nl + j] = ob[1] - s.Q;
            res[2 * nl + j] = ob[2] - s.U;
            res[3 * nl + j] = ob[3] - s.V;
        }
        kahan_sq(sI, cI, ob[0] - s.I);
        kahan_sq(sQ, cQ, ob[1] - s.Q);
        kahan_sq(sU, cU, ob[2] - s.U);
        kahan_sq(sV, cV, ob[3] - s.V);
    }
    return (s_w2[0] * sI + s_w2[1] * sQ + s_w2[2] * sU + s_w2[3] * sV) * inv_nu;
}


// Eq. chisq for one individual with the FP32 pair path (two wavelengths per
// step, packed FP32x2 arithmetic), as a Kahan-compensated sum.  The residuals
// come out weighted: the staged Q, U, V rows carry the pixel's weights
// (weight_obs_rows) and so do the individual's Q, U, V output constants, and
// the I residual takes w_I with one multiply.  Each pair's eight squared
// weighted residuals are summed by packed FMAs, its two lanes added, and the
// result taken into one scalar running total with Kahan's compensation, so
// the sum's relative error stays at a few units of 2^-24 whatever the number
// of wavelengths.  The fitness only ranks
// individuals; the best individual's chi2 is re-evaluated in FP64.
// s_kc: the calling thread's shared-memory slots, three float4 at s_kc[k],
// s_kc[k + blockDim], s_kc[k + 2 blockDim] (k = threadIdx.x), which hold the
// individual's closed-form constants and w_I for the length of the call:
// they are read once per pair instead of holding registers through the
// profile evaluations.
template <int NL, bool COUNT, bool PAT, bool FILL, bool STORE = false>
__device__ __forceinline__ float fitness_pairs(const KProblem &pb, int nlines, int nl, const float *p,
                                               float mu, const float *s_obs, const float *s_doff,
                                               const float *he, const float *s_w2, float inv_nu,
                                               WorkCount &wc, float4 *s_kc, float *res = nullptr)
{
    Geo<float> geo = make_geo<float, NL, FILL>(pb, nlines, p, mu);
    pair_thresholds(geo, nlines);
    geo.vmask = __activemask();
    const float *sw = s_w2 + 4;  // the weights themselves
    geo.kQ *= sw[1];
    geo.kUV *= sw[1];
    geo.kU *= sw[2];
    geo.kQV *= sw[2];
    geo.kV *= sw[3];
    const int kt = threadIdx.x, nt = blockDim.x;
    s_kc[kt] = make_float4(geo.kIs, geo.kIp, geo.kIp2, geo.kV2);
    s_kc[nt + kt] = make_float4(geo.muS1, geo.S0, geo.kQ, geo.kUV);
    s_kc[2 * nt + kt] = make_float4(geo.kU, geo.kQV, geo.kV, sw[0]);
    const float4 *kc = s_kc + kt;
    float sum = 0.f, comp = 0.f;
    const int npair = (nl + 1) >> 1;
    EvalCount cnt{0u, 0u, 0u, 0u};
    for (int q = 0; q < npair; ++q) {
        const float4 d0 = *(const float4 *)(s_doff + 8 * q);
        float2 doff2[ME_MAX_LINES];
        doff2[0] = make_float2(d0.x, d0.y);
        doff2[1] = make_float2(d0.z, d0.w);
        if (NL == 0 || NL > 2) {
            const float4 d1 = *(const float4 *)(s_doff + 8 * q + 4);
            doff2[2] = make_float2(d1.x, d1.y);
            doff2[3] = make_float2(d1.z, d1.w);
        }
        const bool y_real = 2 * q + 1 < nl;
        float wIs;
        const Stokes4x2 rr = resid_x2<NL, COUNT, PAT, FILL>(geo, doff2, s_obs + 8 * q, he, nlines, y_real, cnt, pb.line, kc, nt,
                                                            wIs);
        float2 rI = mul2(rr.I, f2(wIs)), rQ = rr.Q, rU = rr.U, rV = rr.V;
        if (!y_real) rI.y = rQ.y = rU.y = rV.y = 0.f;  // padded partner
        if (STORE && res) {
            const int j = 2 * q;
            res[j] = rI.x;
            res[nl + j] = rQ.x;
            res[2 * nl + j] = rU.x;
            res[3 * nl + j] = rV.x;
            if (y_real) {
                res[j + 1] = rI.y;
                res[nl + j + 1] = rQ.y;
                res[2 * nl + j + 1] = rU.y;
                res[3 * nl + j + 1] = rV.y;
            }
        }
        float2 t2 = fma2(rQ, rQ, mul2(rI, rI));
        t2 = fma2(rU, rU, t2);
        t2 = fma2(rV, rV, t2);
        const float y = (t2.x + t2.y) - comp;  // Kahan: comp holds the lost low part, negated
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    if (COUNT) {
        wc.interior += cnt.interior;
        wc.mid += cnt.mid;
        wc.even2 += cnt.even2;
        wc.far += cnt.far;
    }
    return (sum - comp) * inv_nu;
}

template <class R, int NL, bool COUNT, bool PAT, bool FILL, bool STORE = false>
__device__ __forceinline__ R fitness(const KProblem &pb, int nlines, int nl, const R *p, R mu,
                                     const R *s_obs, const R *s_doff, const R *he,
                                     const R *s_w2, R inv_nu, WorkCount &wc, float4 *s_kc, R *res = nullptr)
{
    if constexpr (std::is_same<R, float>::value)
        return fitness_pairs<NL, COUNT, PAT, FILL, STORE>(pb, nlines, nl, p, mu, s_obs, s_doff, he, s_w2,
                                                          inv_nu, wc, s_kc, res);
    else
        return fitness_rows<R, NL, COUNT, PAT, FILL, STORE>(pb, nlines, nl, p, mu, s_obs, s_doff, he, s_w2,
                                                            inv_nu, wc, res);
}

// argmin over the block's fitness, ties to the lowest index.  Every thread
// gets the result.  Uses one __syncthreads().
template <class R>
__device__ __forceinline__ int block_argmin(const R *s_fit, R *s_wmin, int *s_widx)
{
    const int k = threadIdx.x, lane = k & 31, warp = k >> 5, nw = blockDim.x >> 5;
    R v = s_fit[k];
    int idx = k;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const R ov = __shfl_down_sync(0xffffffffu, v, off);
        const int oi = __shfl_down_sync(0xffffffffu, idx, off);
        if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (lane == 0) { s_wmin[warp] = v; s_widx[warp] = idx; }
    __syncthreads();
    R bv = s_wmin[0];
    int bi = s_widx[0];
    for (int w = 1; w < nw; ++w) {
        const R ov = s_wmin[w];
        const int oi = s_widx[w];
        if (ov < bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    return bi;
}

// Stable rank of individual k in (fitness, index) order.
template <class R> __device__ __forceinline__ int stable_rank(const R *s_fit, int npop, int k)
{
    const R fk = s_fit[k];
    int r = 0;
    for (int j = 0; j < npop; ++j) {
        const R fj = s_fit[j];
        r += (fj < fk || (fj == fk && j < k)) ? 1 : 0;
    }
    return r;
}

// Select (binary tournament), recombine (one-point crossover with lane k^1),
// mutate (per-bit, LSB-biased) and elitism for child slot k.  Must be called
// by all lanes of full warps (npop is a multiple of 32).
template <class R, int M>
__device__ __forceinline__ void breed_one(const KGa &ga, uint64_t pid, int t, int k, int npop,
                                          const R *s_fit, const uint16_t *s_cur, int elite,
                                          uint16_t *s_row, uint16_t g[M])
{
    const U4 u = ga_random_rk(ga.rk, pid, t, (uint32_t)k, kPurposeSelect);
    const int i = (int)(((uint64_t)u.x * (uint64_t)npop) >> 32);
    int j = i + 1 + (int)(((uint64_t)u.y * (uint64_t)(npop - 1)) >> 32);  // at most 2 npop - 2
    if (j >= npop) j -= npop;
    const R fi = s_fit[i], fj = s_fit[j];
    const int win = (fj < fi || (fj == fi && j < i)) ? j : i;
#pragma unroll
    for (int d = 0; d < M; ++d) g[d] = s_cur[win * M + d];

    // the pair's crossover draws: words z, w of the even slot's block
    const uint32_t cz = __shfl_sync(0xffffffffu, u.z, (k & 31) & ~1);
    const uint32_t cw = __shfl_sync(0xffffffffu, u.w, (k & 31) & ~1);
    const bool cross = (uint64_t)cz < ga.t_cross;
    const int c = 1 + (int)(((uint64_t)cw * (uint64_t)(16 * M - 1)) >> 32);
#pragma unroll
    for (int d = 0; d < M; ++d) {
        const uint32_t pg = __shfl_xor_sync(0xffffffffu, (uint32_t)g[d], 1);
        if (cross) {
            const int b0 = 16 * d;  // MSB-first string bits [b0, b0 + 16)
            if (b0 >= c) {
                g[d] = (uint16_t)pg;
            } else if (b0 + 16 > c) {
                const uint32_t mask = (1u << (16 - (c - b0))) - 1u;  // bits at or after the cut
                g[d] = (uint16_t)(((uint32_t)g[d] & ~mask) | (pg & mask));
            }
        }
    }

    // Mutation (every bit b flips on its own with probability q_b), word by
    // word through this slot's shared-memory row (a rolled loop keeps the code
    // small).  The slot's draws u_0, u_1, ... (four per Philox block, purposes
    // 2, 3, ...) jump from flip to flip, from the word's LSB toward its MSB:
    // with bits 0..b still open, u >= t(b, 0) leaves them all unflipped;
    // otherwise the next flip is bit c, the largest c <= b with u < t(b, c),
    // and bits 0..c-1 stay open.  A word without flips takes one draw.
#pragma unroll
    for (int d = 0; d < M; ++d) s_row[d] = g[d];
    U4 blk = {0u, 0u, 0u, 0u};
    uint32_t nblk = 0, left = 0;
#pragma unroll 1
    for (int d = 0; d < M; ++d) {
        uint32_t word = s_row[d];
        int b = 15;
        while (b >= 0) {
            if (left == 0) {
                blk = ga_random_rk(ga.rk, pid, t, (uint32_t)k, kPurposeMutate + nblk);
                ++nblk;
                left = 4;
            }
            const uint64_t uv = blk.x;
            blk.x = blk.y;
            blk.y = blk.z;
            blk.z = blk.w;
            --left;
            const uint64_t *row = ga.t_mut + b * (b + 1) / 2;
            if (uv >= row[0]) break;
            int lo = 0, hi = b;  // the largest c with uv < row[c]; row[0] qualifies
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (uv < row[mid]) lo = mid;
                else hi = mid - 1;
            }
            word ^= 1u << (15 - lo);
            b = lo - 1;
        }
        s_row[d] = (uint16_t)word;
    }
#pragma unroll
    for (int d = 0; d < M; ++d) g[d] = s_row[d];
    if (k == 0) {
#pragma unroll
        for (int d = 0; d < M; ++d) g[d] = s_cur[elite * M + d];
    }
}

struct GaSmem {
    // byte offsets into dynamic shared memory
    int obs, doff, fit, wmin, widx, w2, he, dom, genes, kc, total;
};

template <class R>
__host__ __device__ __forceinline__ GaSmem ga_smem_layout(int nl, int nlines, int npop, int npar)
{
    GaSmem L;
    int o = 0;
    auto take = [&](int bytes, int align) {
        o = (o + align - 1) / align * align;
        const int at = o;
        o += bytes;
        return at;
    };
    const int nlp = sizeof(R) == 4 ? (nl + 1) & ~1 : nl;  // padded to whole pairs in FP32
    L.obs = take(4 * nlp * (int)sizeof(R), 16);
    L.doff = take(4 * nlp * (int)sizeof(R), 16);
    L.fit = take(npop * (int)sizeof(R), 16);
    L.wmin = take(32 * (int)sizeof(R), 16);
    L.widx = take(32 * 4, 16);
    L.w2 = take(8 * (int)sizeof(R), 16);  // w^2 of I, Q, U, V, then w
    L.he = take(4 * (int)sizeof(R), 16);
    L.dom = take((int)sizeof(DecodeDomain), 16);  // the pixel's decode domain
    L.genes = take(2 * npop * npar * 2, 16);
    L.kc = take(sizeof(R) == 4 ? 3 * npop * 16 : 0, 16);  // FP32: 3 float4 of closed-form constants per thread
    L.total = (o + 15) / 16 * 16;
    return L;
}

// Section 5.4 inverse-max weights of the staged pixel (warp 0), written as
// w^2 (s_w2[0..3]) and w (s_w2[4..7]).
template <class R>
__device__ __forceinline__ void weights_invmax_w2(const R *s_obs, int nl, R *s_w2)
{
    const int lane = threadIdx.x & 31;
    R imax = -R(INFINITY), imin = R(INFINITY), mq = 0, mu = 0, mv = 0;
    for (int j = lane; j < nl; j += 32) {
        const R I = s_obs[obs_idx<R>(0, j)];
        imax = I > imax ? I : imax;
        imin = I < imin ? I : imin;
        const R aq = fabs(s_obs[obs_idx<R>(1, j)]), au = fabs(s_obs[obs_idx<R>(2, j)]);
        const R av = fabs(s_obs[obs_idx<R>(3, j)]);
        mq = aq > mq ? aq : mq;
        mu = au > mu ? au : mu;
        mv = av > mv ? av : mv;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        R o = __shfl_xor_sync(0xffffffffu, imax, off); imax = o > imax ? o : imax;
        o = __shfl_xor_sync(0xffffffffu, imin, off); imin = o < imin ? o : imin;
        o = __shfl_xor_sync(0xffffffffu, mq, off); mq = o > mq ? o : mq;
        o = __shfl_xor_sync(0xffffffffu, mu, off); mu = o > mu ? o : mu;
        o = __shfl_xor_sync(0xffffffffu, mv, off); mv = o > mv ? o : mv;
    }
    if (lane == 0) {
        const R d[4] = {imax - imin, mq, mu, mv};
        const R fl = R(1e-6) * fabs(imax);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const R dd = d[s] > fl ? d[s] : fl;
            const R w = dd > R(0) ? R(1) / dd : R(0);
            s_w2[s] = w * w;
            s_w2[4 + s] = w;
        }
    }
}

// Per-launch constants of a GA block: s_doff in the layout of obs_idx with
// lambda_j - lambda0_l (exact in FP64, then rounded; a padded partner repeats
// the last point) and s_he[l] = eta_ratio_l / 2.
template <class R>
__device__ __forceinline__ void stage_offsets_ga(const KProblem &pb, int nlines, int nl, int k, R *s_doff,
                                                 R *s_he)
{
    if (k < 4) s_he[k] = k < nlines ? R(pb.line[k].half_eta) : R(0);
    for (int i = k; i < 4 * padded_lambda<R>(nl); i += blockDim.x) {
        const int j = i >> 2, l = i & 3;
        const int jj = j < nl ? j : nl - 1;
        s_doff[obs_idx<R>(l, j)] = l < nlines ? R(pb.lam[jj] - pb.line[l].lam0) : R(0);
    }
}

// a1: one pixel's Stokes profiles from [4][nl] in HBM into the shared-memory
// layout of obs_idx (16-byte vector loads when a vector stays in one row).
template <class R>
__device__ __forceinline__ void stage_obs(const R *o, int nl, int k, R *s_obs)
{
    constexpr int VW = 16 / (int)sizeof(R);  // elements per 16-byte vector
    if (nl % VW == 0 && (((uintptr_t)o) & 15) == 0) {
        for (int i = k; i < 4 * nl / VW; i += blockDim.x) {
            const int e = i * VW, st = e / nl, j = e - st * nl;
            if (VW == 4) {
                const float4 q = __ldg((const float4 *)o + i);
                s_obs[obs_idx<R>(st, j)] = R(q.x);
                s_obs[obs_idx<R>(st, j + 1)] = R(q.y);
                s_obs[obs_idx<R>(st, j + 2)] = R(q.z);
                s_obs[obs_idx<R>(st, j + 3)] = R(q.w);
            } else {
                const double2 q = __ldg((const double2 *)o + i);
                s_obs[obs_idx<R>(st, j)] = R(q.x);
                s_obs[obs_idx<R>(st, j + 1)] = R(q.y);
            }
        }
    } else {
        for (int i = k; i < 4 * nl; i += blockDim.x) {
            const int st = i / nl, j = i - st * nl;
            s_obs[obs_idx<R>(st, j)] = o[i];
        }
    }
    if (padded_lambda<R>(nl) > nl && k < 4) s_obs[obs_idx<R>(k, nl)] = o[k * nl + nl - 1];
}

// a2: the pixel's squared weights, the caller's (ME_W_USER) or Section 5.4's
// inverse-max weights of the staged profiles (warp 0).
template <class R>
__device__ __forceinline__ void stage_weights(int weight_mode, const double *w_user, int pix, const R *s_obs,
                                              int nl, int k, R *s_w2)
{
    if (weight_mode == ME_W_USER) {
        if (k < 4) {
            const double wv = w_user[(size_t)pix * 4 + k];
            s_w2[k] = R(wv * wv);
            s_w2[4 + k] = R(fabs(wv));
        }
    } else if (k < 32) {
        weights_invmax_w2<R>(s_obs, nl, s_w2);
    }
}

// FP32 pair path: the pixel's weights w_Q, w_U, w_V folded into its staged
// Q, U, V rows (after the weights are known), so that the fitness forms
// weighted residuals directly (see fitness_pairs).  FP64 rows stay as staged.
template <class R>
__device__ __forceinline__ void weight_obs_rows(R *s_obs, int nl, int k, const R *s_w2)
{
    if constexpr (sizeof(R) == 4) {
        const int nlp = padded_lambda<R>(nl);
        for (int i = k; i < 3 * nlp; i += blockDim.x) {
            const int st = 1 + i / nlp, j = i - (st - 1) * nlp;
            s_obs[obs_idx<R>(st, j)] *= s_w2[4 + st];
        }
    }
}

// Register budget per thread.  FP32 instantiations for npop <= 256 with one
// or two effective-triplet lines: GENESIS_GA_NREG32 = 72, so that seven
// 128-thread blocks fit an SM's 64K registers (more resident warps hide the
// FP32 pipe's latency; a few bytes spill in the two-line form, whose launch
// is still 0.5 % faster than six blocks at 80 registers).  The other FP32
// ones for npop <= 256 (any line count, full patterns) keep 80, where they
// spill less.  1024-thread instantiations: 64, so that a whole block fits.
// FP64 ones are bound by the FP64 units and may use up to 255.
#ifndef GENESIS_GA_NREG32
#define GENESIS_GA_NREG32 72
#endif
// Build option: GENESIS_GA_MAXNREG=N caps every instantiation at N registers
// per thread instead (for tuning the cap).
#ifdef GENESIS_GA_MAXNREG
#define GENESIS_GA_BOUNDS(MAXT, R, NL, PAT) __maxnreg__(GENESIS_GA_MAXNREG)
#else
#define GENESIS_GA_BOUNDS(MAXT, R, NL, PAT)                                                         \
    __maxnreg__((MAXT) > 256 ? 65536 / (MAXT)                                                     \
                             : (sizeof(R) == 4 ? ((NL) > 0 && !(PAT) ? GENESIS_GA_NREG32 : 80) : 255))
#endif

template <class R, int NL, int MAXT, bool COUNT, bool PAT, int M>
__global__ void GENESIS_GA_BOUNDS(MAXT, R, NL, PAT)
k_ga_evolve(const __grid_constant__ KProblem pb, const __grid_constant__ KGa ga,
            const R *__restrict__ obs, const double *__restrict__ w_user,
            const double *__restrict__ mu_px, int npix, double *__restrict__ best,
            uint16_t *__restrict__ best_genes, unsigned long long *__restrict__ counts,
            const KSeed sd, const KSub sub)
{
    constexpr bool FILL = M > ME_NPAR;  // parameter 9: the fill fraction (Section 5.2)
    unsigned long long nfit = 0;
    WorkCount wc{};
    extern __shared__ __align__(16) unsigned char smem[];
    const int nl = pb.n_lambda;
    const int nlines = NL > 0 ? NL : pb.n_lines;
    const int npop = ga.npop;
    const int k = threadIdx.x;
    const GaSmem L = ga_smem_layout<R>(nl, nlines, npop, M);
    R *s_obs = (R *)(smem + L.obs);
    R *s_doff = (R *)(smem + L.doff);
    R *s_fit = (R *)(smem + L.fit);
    R *s_wmin = (R *)(smem + L.wmin);
    int *s_widx = (int *)(smem + L.widx);
    R *s_w2 = (R *)(smem + L.w2);
    R *s_he = (R *)(smem + L.he);
    DecodeDomain &D = *(DecodeDomain *)(smem + L.dom);
    uint16_t *s_genes = (uint16_t *)(smem + L.genes);
    float4 *s_kc = (float4 *)(smem + L.kc);

    // per-launch constants
    const R inv_nu = R(1) / R(4 * nl - M);
    stage_offsets_ga<R>(pb, nlines, nl, k, s_doff, s_he);

    const int nrun = sub.count ? min(*sub.count, npix) : npix;
    for (int blk = blockIdx.x; blk < nrun; blk += gridDim.x) {
        const int pix = sub.index ? sub.index[blk] : blk;
        if (pix < 0 || pix >= npix) continue;  // a bad index skips the block, uniformly
        if (k < M) {  // the pixel's decode domain of parameter k
            double a = sd.bounds_px ? sd.bounds_px[(size_t)pix * 2 * M + k] : ga.lo[k];
            double b = sd.bounds_px ? sd.bounds_px[(size_t)pix * 2 * M + M + k] : ga.hi[k];
            if (k == 1 && sd.polarity) polarity_bounds(sd.polarity[pix], a, b, a, b);
            D.lo[k] = a;
            D.hi[k] = b;
            D.lo32[k] = (float)a;
            D.sc32[k] = (float)((b - a) / 65535.0);
        }
        // a1: stage the pixel's Stokes profiles
        stage_obs<R>(obs + (size_t)pix * 4 * nl, nl, k, s_obs);
        __syncthreads();
        // a2: weights
        stage_weights<R>(ga.weight_mode, w_user, pix, s_obs, nl, k, s_w2);
        __syncthreads();
        if (sizeof(R) == 4) {
            weight_obs_rows<R>(s_obs, nl, k, s_w2);
            __syncthreads();
        }
        R he[ME_MAX_LINES];
#pragma unroll
        for (int l = 0; l < ME_MAX_LINES; ++l) he[l] = s_he[l];
        const R mu = mu_px ? R(mu_px[pix]) : R(pb.mu);
        const uint64_t pid = ga.pixel_id0 + (uint64_t)pix;

        // a3 + a4: Sobol points 1..npop, the last nseed taking the seeds'
        // (B, psi, chi) genes, decode, evaluate
        uint16_t g[M];
        R p[M];
#pragma unroll
        for (int d = 0; d < M; ++d) g[d] = (uint16_t)(sobol_point((uint64_t)(k + 1), d) >> 16);
        if (k >= npop - sd.nseed) {
            const double *sv = sd.seeds + ((size_t)pix * sd.nseed + (k - (npop - sd.nseed))) * 3;
            const double x0 = sv[0], x1 = sv[1], x2 = sv[2];
            if (x0 == x0) g[0] = encode64(x0, D.lo[0], D.hi[0]);
            if (x1 == x1) g[1] = encode64(x1, D.lo[1], D.hi[1]);
            if (x2 == x2) g[2] = encode64(x2, D.lo[2], D.hi[2]);
        }
#pragma unroll
        for (int d = 0; d < M; ++d) p[d] = GaDecode<R>::get(D, d, g[d]);
        int cur = 0;
#pragma unroll
        for (int d = 0; d < M; ++d) s_genes[k * M + d] = g[d];
        s_fit[k] = clean_fit(fitness<R, NL, COUNT, PAT, FILL>(pb, nlines, nl, p, mu, s_obs, s_doff, he, s_w2, inv_nu, wc, s_kc));
        if (COUNT) ++nfit;
        uint64_t sobol_next = (uint64_t)npop + 1;

        for (int t = 1; t <= ga.ngen; ++t) {
            __syncthreads();  // fitness and genes of generation t-1 complete
            const int elite = block_argmin<R>(s_fit, s_wmin, s_widx);  // a9
            const uint16_t *s_cur = s_genes + cur * npop * M;
            uint16_t *s_nxt = s_genes + (cur ^ 1) * npop * M;
            breed_one<R, M>(ga, pid, t, k, npop, s_fit, s_cur, elite, s_nxt + k * M, g);  // a10-a12
            __syncthreads();  // every tournament has read s_fit
#pragma unroll
            for (int d = 0; d < M; ++d) {
                s_nxt[k * M + d] = g[d];
                p[d] = GaDecode<R>::get(D, d, g[d]);
            }
            cur ^= 1;
            s_fit[k] = clean_fit(fitness<R, NL, COUNT, PAT, FILL>(pb, nlines, nl, p, mu, s_obs, s_doff, he, s_w2, inv_nu, wc, s_kc));
            if (COUNT) ++nfit;
            // a13: worst-half Sobol restart.  The individual of rank npop/2 + i
            // takes Sobol point sobol_next + i; thread i evaluates it, so the
            // new half fills whole warps (the idle half of the gene double
            // buffer carries the individuals' indices).
            if (ga.nsamp > 0 && t % ga.nsamp == 0 && t < ga.ngen) {
                __syncthreads();
                const int rank = stable_rank<R>(s_fit, npop, k);
                int *s_ridx = (int *)(s_genes + (cur ^ 1) * npop * M);
                if (rank >= npop / 2) s_ridx[rank - npop / 2] = k;
                __syncthreads();
                if (k < npop / 2) {
                    const int kr = s_ridx[k];
                    const uint64_t n = sobol_next + (uint64_t)k;
                    uint16_t *s_c = s_genes + cur * npop * M;
#pragma unroll
                    for (int d = 0; d < M; ++d) {
                        g[d] = (uint16_t)(sobol_point(n, d) >> 16);
                        s_c[kr * M + d] = g[d];
                        p[d] = GaDecode<R>::get(D, d, g[d]);
                    }
                    s_fit[kr] = clean_fit(
                        fitness<R, NL, COUNT, PAT, FILL>(pb, nlines, nl, p, mu, s_obs, s_doff, he, s_w2, inv_nu, wc, s_kc));
                    if (COUNT) ++nfit;
                }
                sobol_next += (uint64_t)(npop / 2);
            }
        }
        __syncthreads();
        const int b = block_argmin<R>(s_fit, s_wmin, s_widx);
        // a14: decoded best individual (its FP64 chi2 is a separate pass)
        if (k < M) {
            const uint16_t gb = s_genes[cur * npop * M + b * M + k];
            best[(size_t)pix * M + k] =
                decode64(gb, D.lo[k], D.hi[k]);
            if (best_genes) best_genes[(size_t)pix * M + k] = gb;
        }
        __syncthreads();  // shared memory is reused by the next pixel
    }
    if (COUNT) {
        // evaluations per synthesis: every real wavelength point runs each
        // line's components (three for an effective triplet)
        unsigned long long per_point = 0;
        for (int l = 0; l < nlines; ++l) {
            const int nc = pb.line[l].ncomp[0] + pb.line[l].ncomp[1] + pb.line[l].ncomp[2];
            per_point += nc ? nc : 3;
        }
        atomicAdd(counts + 0, nfit);
        atomicAdd(counts + 1, wc.interior);
        atomicAdd(counts + 2, nfit * (unsigned long long)nl * per_point);
        atomicAdd(counts + 3, wc.far);
        atomicAdd(counts + 4, wc.mid);
        atomicAdd(counts + 5, wc.even2);
    }
}

template <class R, int NL, int MAXT, bool COUNT = false, bool PAT = false, int M = ME_NPAR>
cudaError_t launch_evolve_t(const KProblem &pb, const KGa &ga, const void *obs, const double *w,
                            const double *mu_px, int npix, double *best, uint16_t *best_genes,
                            cudaStream_t st, unsigned long long *counts = nullptr, KSeed sd = {},
                            KSub sub = {})
{
    const int nlines = NL > 0 ? NL : pb.n_lines;
    const GaSmem L = ga_smem_layout<R>(pb.n_lambda, nlines, ga.npop, M);
    auto kern = k_ga_evolve<R, NL, MAXT, COUNT, PAT, M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    kern<<<npix, ga.npop, L.total, st>>>(pb, ga, (const R *)obs, w, mu_px, npix, best, best_genes, counts,
                                          sd, sub);
    return cudaGetLastError();
}

}  // namespace
}  // namespace genesis
