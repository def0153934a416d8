/*
 * paco_affine.h - C ABI of the affine-gap alignment kernels.
 *
 * The footnote to Eq. (1) of Tang & Gao, "Balanced Partitioning of Several
 * Cache-Oblivious Algorithms" (Sec. "PACO LCS"), names pairwise sequence
 * alignment with affine gap cost (Gotoh 1982) as the problem whose
 * recurrence is like the LCS one.  This library fills that table on the GPU
 * with the same row-band dataflow as the LCS path: for byte strings a (n
 * rows) and b (m columns) and the scores below,
 *
 *   E[i][j] = max(E[i][j-1], H[i][j-1] - gap_open) - gap_extend
 *   F[i][j] = max(F[i-1][j], H[i-1][j] - gap_open) - gap_extend
 *   H[i][j] = max(H[i-1][j-1] + s(a[i-1], b[j-1]), E[i][j], F[i][j])
 *   s(x, y) = +match if x == y, else -mismatch
 *
 * with H[0][0] = 0, H[i][0] = -(gap_open + i*gap_extend), H[0][j] =
 * -(gap_open + j*gap_extend), E[i][0] = F[0][j] = -infinity.  H[n][m] is the
 * best score of a global alignment in which every aligned column scores s
 * and every maximal run of k gap columns in one sequence costs
 * gap_open + k*gap_extend.
 *
 * Conventions are those of paco_lcs.h (contexts, streams, ownership, error
 * words read by paco_ctx_sync).  Additionally:
 * - The four scores are in [0, 65535].
 * - Every reachable value must fit well inside int32: a call is rejected
 *   with PACO_EINVAL unless match * min(n, m) <= 2^29 and
 *   2 * gap_open + gap_extend * (n + m) <= 2^29 (per pair for batches).
 * - Outputs are int32.  A device-side failure (a bounded wait between row
 *   bands that timed out) is returned by the next paco_ctx_sync as
 *   PACO_ETIMEOUT.
 */
#ifndef PACO_AFFINE_H
#define PACO_AFFINE_H

#include <stdint.h>

#include "paco_lcs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct paco_affine_scores {
    int32_t match;       /* added for an aligned column of equal symbols     */
    int32_t mismatch;    /* subtracted for an aligned column of unequal ones */
    int32_t gap_open;    /* subtracted once per maximal gap run              */
    int32_t gap_extend;  /* subtracted per gap column                        */
} paco_affine_scores;

/* One pair, device pointers.  a: n bytes, b: m bytes.  Writes the score
 * H[n][m] to *d_score (one int32, required) and, when not NULL,
 * d_bottom_row[j] = H[n][j] (m+1 values) and d_right_col[i] = H[i][m] (n+1
 * values).  Stream ordered.  Errors at enqueue: PACO_EINVAL (NULL context
 * or score, bad length, scores out of range), PACO_ENOMEM, PACO_EDEVICE. */
int paco_affine_align(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                      const paco_affine_scores *scores, int32_t *d_score, int32_t *d_bottom_row,
                      int32_t *d_right_col, void *stream);

/* The same with HOST buffers: copies a and b to the device, aligns, copies
 * the outputs back and synchronises `stream` (NULL = the context's own
 * stream) before returning.  Device errors are returned directly. */
int paco_affine_align_host(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                           const paco_affine_scores *scores, int32_t *score, int32_t *bottom_row,
                           int32_t *right_col, void *stream);

/* Independent pairs in one launch.  a_cat / b_cat: concatenated device
 * strings; a_off / b_off: HOST int64 offsets (npairs + 1 each, starting at
 * 0, non-decreasing); pair k is a_cat[a_off[k] .. a_off[k+1]) against
 * b_cat[b_off[k] .. b_off[k+1]).  Writes d_score[k] (device, npairs int32).
 * Stream ordered.  Errors: PACO_EINVAL, PACO_ENOMEM, PACO_EDEVICE. */
int paco_affine_batch(paco_ctx *ctx, const uint8_t *a_cat, const int64_t *a_off, const uint8_t *b_cat,
                      const int64_t *b_off, int32_t npairs, const paco_affine_scores *scores,
                      int32_t *d_score, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PACO_AFFINE_H */
