/*
 * CPU ORACLE for global alignment with affine gap costs (test infrastructure
 * only).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code, header or table with the CUDA library and
 * must never be linked into it.
 *
 * What it computes: the footnote to Eq. (1) of Tang & Gao, "Balanced
 * Partitioning of Several Cache-Oblivious Algorithms" (Sec. "PACO LCS"),
 * names pairwise sequence alignment with affine gap cost (Gotoh 1982) as the
 * problem whose recurrence is like Eq. (1).  The paper fixes no scoring, so
 * the scores are caller parameters (all >= 0):
 *
 *   s(x, y) = +match if x == y, else -mismatch
 *   a run of k consecutive gap columns in one sequence costs open + k*extend
 *
 * and the score of a global alignment is the sum of s over its aligned
 * columns minus the cost of each gap run; an insertion run directly followed
 * by a deletion run is two runs.  Gotoh's three-value recurrence gives the
 * best score of a[0..i) against b[0..j):
 *
 *   E[i][j] = max(E[i][j-1], H[i][j-1] - open) - extend     (b[j-1] against a gap)
 *   F[i][j] = max(F[i-1][j], H[i-1][j] - open) - extend     (a[i-1] against a gap)
 *   H[i][j] = max(H[i-1][j-1] + s(a[i-1], b[j-1]), E[i][j], F[i][j])
 *
 * with H[0][0] = 0, H[i][0] = -(open + i*extend) and H[0][j] =
 * -(open + j*extend) for i, j > 0, and E[i][0] = F[0][j] = -infinity.
 *
 * Outputs: score = H[n][m], bottom_row[j] = H[n][j] (j = 0..m),
 * right_col[i] = H[i][m] (i = 0..n).  Arithmetic in int64 with -infinity
 * far below any reachable value.
 *
 * Algorithm: the textbook row sweep (row i from row i-1), O(nm) time, O(m)
 * space.  No blocking, no SIMD, no threads inside one pair.
 */
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

static const int64_t NEG_INF = INT64_MIN / 4;

static int64_t max_i64(int64_t x, int64_t y) { return x > y ? x : y; }

int oracle_affine(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                  int64_t match, int64_t mismatch, int64_t open, int64_t extend,
                  int64_t *score, int64_t *bottom_row, int64_t *right_col)
{
    if (n < 0 || m < 0 || match < 0 || mismatch < 0 || open < 0 || extend < 0) return ORACLE_EINVAL;
    if ((n > 0 && !a) || (m > 0 && !b)) return ORACLE_EINVAL;

    int64_t *Hp = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));   /* H[i-1][.] */
    int64_t *Fp = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));   /* F[i-1][.] */
    int64_t *Hc = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));   /* H[i][.]   */
    if (!Hp || !Fp || !Hc) { free(Hp); free(Fp); free(Hc); return ORACLE_ENOMEM; }

    /* row 0 */
    Hp[0] = 0;
    Fp[0] = NEG_INF;
    for (int64_t j = 1; j <= m; ++j) {
        Hp[j] = -(open + j * extend);
        Fp[j] = NEG_INF;
    }
    if (right_col) right_col[0] = Hp[m];

    for (int64_t i = 1; i <= n; ++i) {
        const uint8_t ai = a[i - 1];
        /* column 0 */
        Hc[0] = -(open + i * extend);
        int64_t E = NEG_INF;                               /* E[i][0] */
        for (int64_t j = 1; j <= m; ++j) {
            E = max_i64(E, Hc[j - 1] - open) - extend;                 /* E[i][j] */
            const int64_t F = max_i64(Fp[j], Hp[j] - open) - extend;   /* F[i][j] */
            const int64_t s = (ai == b[j - 1]) ? match : -mismatch;
            int64_t H = Hp[j - 1] + s;
            H = max_i64(H, E);
            H = max_i64(H, F);
            Hc[j] = H;
            Fp[j] = F;             /* F[i-1][j] is not needed any more */
        }
        if (right_col) right_col[i] = Hc[m];
        int64_t *t = Hp; Hp = Hc; Hc = t;
    }
    if (bottom_row)
        for (int64_t j = 0; j <= m; ++j) bottom_row[j] = Hp[j];
    *score = Hp[m];
    free(Hp); free(Fp); free(Hc);
    return ORACLE_OK;
}

/* ---------------------------------------------------------------- batch */

typedef struct {
    const uint8_t *a_cat, *b_cat;
    const int64_t *a_off, *b_off;
    int64_t npairs;
    int64_t match, mismatch, open, extend;
    int64_t *score;
    int64_t next;
    int rc;
    pthread_mutex_t mu;
} AffineBatch;

static void *affine_worker(void *arg)
{
    AffineBatch *J = (AffineBatch *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        const int64_t k = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (k >= J->npairs) return NULL;
        const int64_t n = J->a_off[k + 1] - J->a_off[k];
        const int64_t m = J->b_off[k + 1] - J->b_off[k];
        const int rc = oracle_affine(J->a_cat + J->a_off[k], n, J->b_cat + J->b_off[k], m, J->match, J->mismatch,
                                     J->open, J->extend, &J->score[k], NULL, NULL);
        if (rc != ORACLE_OK) {
            pthread_mutex_lock(&J->mu);
            J->rc = rc;
            pthread_mutex_unlock(&J->mu);
        }
    }
}

/* Scores of independent pairs, spread over `threads` host threads. */
int oracle_affine_batch(const uint8_t *a_cat, const int64_t *a_off, const uint8_t *b_cat, const int64_t *b_off,
                        int64_t npairs, int64_t match, int64_t mismatch, int64_t open, int64_t extend,
                        int64_t *score, int threads)
{
    if (npairs < 0 || threads < 1) return ORACLE_EINVAL;
    AffineBatch J = {a_cat, b_cat, a_off, b_off, npairs, match, mismatch, open, extend, score, 0, ORACLE_OK};
    pthread_mutex_init(&J.mu, NULL);
    pthread_t tid[256];
    if (threads > 256) threads = 256;
    int started = 0;
    for (int t = 0; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, affine_worker, &J) != 0) break;
        ++started;
    }
    if (started == 0) affine_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    pthread_mutex_destroy(&J.mu);
    return J.rc;
}
