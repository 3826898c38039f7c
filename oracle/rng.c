/*
 * Oracle: counter-based Philox4x32-10 and the Sobol sequence.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <pthread.h>
#include <stdint.h>

#include "oracle.h"

/*
 * Philox4x32-10 as defined by Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of
 *   (x0,x1,x2,x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0))
 * with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the key bumped by the Weyl
 * constants (0x9E3779B9, 0xBB67AE85) after every round.
 */
void or_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        const uint32_t y1 = (uint32_t)p1;
        const uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        const uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/*
 * Sobol sequence (Section 5.6; Bratley & Fox 1988 construction).
 * The Bratley-Fox table of polynomials and initial numbers is not part of the
 * paper, so the direction numbers are generated here:
 *   - dimension 0 is the van der Corput sequence (m_k = 1 for all k);
 *   - dimension d >= 1 uses the d-th primitive polynomial over GF(2), in order
 *     of increasing degree and, within a degree, increasing integer encoding;
 *     primitivity is tested by checking that x has multiplicative order
 *     2^s - 1 modulo the polynomial;
 *   - the s initial numbers are m_k = 2^k - 1 (the largest odd value below
 *     2^k), and later ones follow the Sobol recurrence
 *     m_k = 2 a_1 m_{k-1} ^ 4 a_2 m_{k-2} ^ ... ^ 2^s m_{k-s} ^ m_{k-s}.
 * Direction number k (1-based) is V_k = m_k * 2^(32-k).  Points are taken in
 * Gray-code order: x_n = XOR of V_{i+1} over the set bits i of n ^ (n >> 1).
 */
static int poly_degree(uint32_t p)
{
    int d = -1;
    while (p) { ++d; p >>= 1; }
    return d;
}

static int is_primitive(uint32_t poly)
{
    const int s = poly_degree(poly);
    if (s < 1 || !(poly & 1u)) return 0;
    const uint32_t order = (1u << s) - 1u;
    uint32_t r = 1u; /* x^0 mod poly */
    for (uint32_t k = 1; k <= order; ++k) {
        r <<= 1; /* multiply by x */
        if (r & (1u << s)) r ^= poly;
        if (r == 1u) return k == order;
    }
    return 0;
}

/* The n-th (0-based) primitive polynomial in the enumeration order above. */
static uint32_t nth_primitive(int n)
{
    int found = -1;
    for (uint32_t p = 2u; p < (1u << 20); ++p) {
        if (is_primitive(p)) {
            if (++found == n) return p;
        }
    }
    return 0u;
}

void or_sobol_directions(int dim, uint32_t v[32])
{
    uint64_t m[33];
    if (dim == 0) {
        for (int k = 1; k <= 32; ++k) m[k] = 1;
    } else {
        const uint32_t poly = nth_primitive(dim - 1);
        const int s = poly_degree(poly);
        for (int k = 1; k <= s && k <= 32; ++k) m[k] = (1ull << k) - 1ull;
        for (int k = s + 1; k <= 32; ++k) {
            uint64_t mk = m[k - s] ^ (m[k - s] << s);
            for (int i = 1; i < s; ++i) {
                /* coefficient a_i of x^(s-i) */
                const uint64_t ai = (poly >> (s - i)) & 1u;
                if (ai) mk ^= m[k - i] << i;
            }
            m[k] = mk;
        }
    }
    for (int k = 1; k <= 32; ++k) v[k - 1] = (uint32_t)(m[k] << (32 - k));
}

#define OR_SOBOL_CACHE 16
static uint32_t sobol_cache[OR_SOBOL_CACHE][32];
static pthread_once_t sobol_once = PTHREAD_ONCE_INIT;

static void sobol_cache_init(void)
{
    for (int d = 0; d < OR_SOBOL_CACHE; ++d) or_sobol_directions(d, sobol_cache[d]);
}

uint32_t or_sobol_u32(uint64_t n, int dim)
{
    uint32_t tmp[32];
    const uint32_t *v;
    if (dim < OR_SOBOL_CACHE) {
        pthread_once(&sobol_once, sobol_cache_init);
        v = sobol_cache[dim];
    } else {
        or_sobol_directions(dim, tmp);
        v = tmp;
    }
    const uint64_t g = n ^ (n >> 1);
    uint32_t x = 0;
    for (int i = 0; i < 32; ++i)
        if ((g >> i) & 1u) x ^= v[i];
    return x;
}
