// FP32 FMA-pipe throughput probe (sm_103a).  Not part of the method: it
// measures the peak that the GA kernel's achieved FP32 rate is reported
// against, on the GPU and at the clock the benchmark runs at.
//
// Every thread runs kChains independent FMA chains x <- x * m + b, unrolled,
// so that the pipe never waits on a dependency; the scalar form issues FFMA,
// the packed form FFMA2 (two FP32 FMAs per lane per instruction, the form the
// GA's fitness loop uses).  The chains converge to b / (1 - m) and never
// reach a denormal or an overflow.
#include <cuda_runtime.h>

namespace genesis {

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kPeakThreads = 256;

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, float m, float b, float *__restrict__ out)
{
    const float s = 1.0f + 1e-3f * (float)(threadIdx.x & 31);
    if (PACKED) {
        float2 x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = make_float2(s + c, s - c);
        const float2 mm = make_float2(m, m), bb = make_float2(b, b);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], mm, bb);
        }
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += x[c].x + x[c].y;
        out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    } else {
        float x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = s + c;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], m, b);
        }
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += x[c];
        out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    }
}

}  // namespace

// FP32 flops one launch performs (FMA = 2).
double fma_peak_flops(int packed, int nblocks, int iters)
{
    return 2.0 * (packed ? 2.0 : 1.0) * kChains * kUnroll * (double)iters * kPeakThreads * (double)nblocks;
}

int fma_peak_threads() { return kPeakThreads; }

cudaError_t launch_fma_peak(int packed, int nblocks, int iters, float *out, cudaStream_t st)
{
    if (packed)
        k_fma_peak<true><<<nblocks, kPeakThreads, 0, st>>>(iters, 0.999f, 1e-3f, out);
    else
        k_fma_peak<false><<<nblocks, kPeakThreads, 0, st>>>(iters, 0.999f, 1e-3f, out);
    return cudaGetLastError();
}

}  // namespace genesis
