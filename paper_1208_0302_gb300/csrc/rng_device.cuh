// Counter-based random numbers for the GA operators (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace genesis {

struct U4 { uint32_t x, y, z, w; };

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the
// multiply-xor bijection with multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key
// increments 0x9E3779B9, 0xBB67AE85 after every round.
__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t m0 = (uint64_t)0xD2511F53u * c.x, m1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(m0 >> 32), lo0 = (uint32_t)m0;
        const uint32_t hi1 = (uint32_t)(m1 >> 32), lo1 = (uint32_t)m1;
#endif
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same generator with its key schedule precomputed: round r XORs in
// rk[r] = (k0 + r W0, k1 + r W1) mod 2^32, which the host forms once per
// launch (the schedule depends on the seed alone).
__host__ __device__ __forceinline__ U4 philox4x32_10_rk(U4 c, const uint32_t (*rk)[2])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t m0 = (uint64_t)0xD2511F53u * c.x, m1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(m0 >> 32), lo0 = (uint32_t)m0;
        const uint32_t hi1 = (uint32_t)(m1 >> 32), lo1 = (uint32_t)m1;
#endif
        U4 n;
        n.x = hi1 ^ c.y ^ rk[r][0];
        n.y = lo1;
        n.z = hi0 ^ c.w ^ rk[r][1];
        n.w = lo0;
        c = n;
    }
    return c;
}

// GA random-number streams.  Counter = (pixel id lo, pixel id hi, generation,
// index << 8 | purpose): purpose 0 = the tournament of child slot `index`
// (words x, y) and, for an even slot, the crossover of its pair (words z, w);
// 2 + i = the mutation draws 4i..4i+3 of slot `index`.
enum : uint32_t { kPurposeSelect = 0, kPurposeMutate = 2 };

__device__ __forceinline__ U4 ga_random(uint64_t seed, uint64_t pid, int gen, uint32_t idx,
                                        uint32_t purpose)
{
    U4 c;
    c.x = (uint32_t)pid;
    c.y = (uint32_t)(pid >> 32);
    c.z = (uint32_t)gen;
    c.w = (idx << 8) | purpose;
    return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}
// The same stream with the launch's precomputed round keys.
__device__ __forceinline__ U4 ga_random_rk(const uint32_t (*rk)[2], uint64_t pid, int gen, uint32_t idx,
                                           uint32_t purpose)
{
    U4 c;
    c.x = (uint32_t)pid;
    c.y = (uint32_t)(pid >> 32);
    c.z = (uint32_t)gen;
    c.w = (idx << 8) | purpose;
    return philox4x32_10_rk(c, rk);
}

// Sobol direction numbers, [dimension][bit], filled at initialisation.
constexpr int kSobolDims = 10;
static __constant__ uint32_t c_sobol[kSobolDims][32];

// Point n (< 2^32) of dimension d in Gray-code order (point 0 is the origin):
// XOR of the direction numbers selected by the bits of n ^ (n >> 1).  The
// table index is the same in every lane, so constant-cache reads broadcast.
__device__ __forceinline__ uint32_t sobol_point(uint64_t n, int d)
{
    const uint32_t g = (uint32_t)(n ^ (n >> 1));
    uint32_t x = 0;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) x ^= ((g >> i) & 1u) ? c_sobol[d][i] : 0u;
    return x;
}

}  // namespace genesis
