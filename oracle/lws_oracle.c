/*
 * CPU ORACLE for the 1D problem (least weight subsequence) - test
 * infrastructure only.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code, header or table with the CUDA library and
 * must never be linked into it.
 *
 * What it computes: Eq. (1D) of Tang & Gao, "Balanced Partitioning of
 * Several Cache-Oblivious Algorithms" (Sec. "PACO 1D"): given D[0] and a
 * weight w(i, j) computable in O(1) without memory accesses,
 *
 *   D[j] = min_{0 <= i < j} ( D[i] + w(i, j) )      for 1 <= j <= n.
 *
 * The paper leaves w abstract.  Weight families (`kind`):
 *
 *   0  the benchmark's weight: d = j - i - T,
 *        q = d*d if |d| < 4096, else 2^24,
 *        w = q + (fmix32((i * 0x9E3779B1) ^ j ^ seed) & 255)
 *      where fmix32 is the 32-bit finaliser of MurmurHash3 (Appleby):
 *        h ^= h >> 16; h *= 0x85EBCA6B; h ^= h >> 13; h *= 0xC2B2AE35; h ^= h >> 16
 *      with all products modulo 2^32.  A paragraph-like cost (lines near T
 *      long are cheap) with a small pseudo-random term so that no structure
 *      (monotone minima, Monge) holds exactly.
 *   1  w = (j - i)^2            (test family)
 *   2  w = T                    (test family)
 *   3  w = q only (kind 0 without the hashed term)   (test family)
 *
 * Arithmetic in int64; results fit int32 for the benchmark's weight because
 * D[j] <= D[0] + w(0, j) < D[0] + 2^24 + 256.
 *
 * Algorithm: the textbook double loop in order of j, O(n^2) time, no
 * blocking, no threads.
 */
#include <stdint.h>
#include <stdlib.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)

static uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

static int64_t weight(int kind, int64_t i, int64_t j, int64_t T, uint32_t seed)
{
    switch (kind) {
    case 0:
    case 3: {
        const int64_t d = j - i - T;
        int64_t w = (d > -4096 && d < 4096) ? d * d : ((int64_t)1 << 24);
        if (kind == 0) w += fmix32(((uint32_t)i * 0x9E3779B1u) ^ (uint32_t)j ^ seed) & 255u;
        return w;
    }
    case 1:
        return (j - i) * (j - i);
    default:
        return T;
    }
}

/* D[0] = d0; writes D[0..n] (n + 1 values).  `argmin`, when not NULL,
 * receives the smallest minimising i of each j (argmin[0] = -1). */
int oracle_lws(int64_t n, int64_t d0, int kind, int64_t T, uint32_t seed, int64_t *D, int64_t *argmin)
{
    if (n < 0 || !D || kind < 0 || kind > 3) return ORACLE_EINVAL;
    D[0] = d0;
    if (argmin) argmin[0] = -1;
    for (int64_t j = 1; j <= n; ++j) {
        int64_t best = D[0] + weight(kind, 0, j, T, seed);
        int64_t arg = 0;
        for (int64_t i = 1; i < j; ++i) {
            const int64_t v = D[i] + weight(kind, i, j, T, seed);
            if (v < best) {
                best = v;
                arg = i;
            }
        }
        D[j] = best;
        if (argmin) argmin[j] = arg;
    }
    return ORACLE_OK;
}

/* The weight itself, for tests that enumerate paths. */
int64_t oracle_lws_weight(int kind, int64_t i, int64_t j, int64_t T, uint32_t seed)
{
    return weight(kind, i, j, T, seed);
}
