/*
 * paco_lws.h - C ABI of the 1D-problem kernel (least weight subsequence).
 *
 * Eq. (1D) of Tang & Gao, "Balanced Partitioning of Several Cache-Oblivious
 * Algorithms" (Sec. "PACO 1D"): given D[0] and a weight w(i, j) computed in
 * O(1) without memory accesses,
 *
 *   D[j] = min_{0 <= i < j} ( D[i] + w(i, j) )      for 1 <= j <= n.
 *
 * The paper leaves w abstract; this library evaluates the weight
 *
 *   d = j - i - T
 *   w(i, j) = (|d| < 4096 ? d*d : 2^24) + (noise ? fmix32((i * 0x9E3779B1) ^ j ^ seed) & 255 : 0)
 *
 * (products modulo 2^32 inside the hash; fmix32 is the 32-bit finaliser of
 * MurmurHash3: h ^= h >> 16; h *= 0x85EBCA6B; h ^= h >> 13; h *= 0xC2B2AE35;
 * h ^= h >> 16): a paragraph-like cost, cheap for jumps near T, with a small
 * hashed term.  All arithmetic is integer; D fits int32 because every D[j]
 * is at most D[0] + w(0, j) < D[0] + 2^24 + 256.
 *
 * Conventions are those of paco_lcs.h (contexts, streams, ownership, error
 * words read by paco_ctx_sync).
 */
#ifndef PACO_LWS_H
#define PACO_LWS_H

#include <stdint.h>

#include "paco_lcs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct paco_lws_weight {
    int32_t T;        /* preferred jump length, in [-2^20, 2^20]          */
    uint32_t seed;    /* seed of the hashed term                           */
    int32_t noise;    /* 1: add the hashed byte, 0: the squared term only  */
} paco_lws_weight;

/* Writes d_D[0..n] (n + 1 int32 values, device memory) with D[0] = d0.
 * n in [0, 2^30], d0 in [0, 2^30).  Stream ordered.  Errors at enqueue:
 * PACO_EINVAL (NULL context / weight / output, out-of-range arguments),
 * PACO_ENOMEM, PACO_EDEVICE; a bounded wait between blocks that timed out
 * is returned by the next paco_ctx_sync as PACO_ETIMEOUT. */
int paco_lws(paco_ctx *ctx, int64_t n, int32_t d0, const paco_lws_weight *w, int32_t *d_D, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PACO_LWS_H */
