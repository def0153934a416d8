/*
 * CPU ORACLE for the LCS table (test infrastructure only).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code, header or table with the CUDA library and
 * must never be linked into it.
 *
 * What it computes: the LCS recurrence of Eq. (1) of Tang & Gao, "Balanced
 * Partitioning of Several Cache-Oblivious Algorithms" (Sec. "PACO LCS"),
 * written literally in its select form, with the table's first row and
 * first column taken from caller boundaries instead of zeros (all zeros when
 * the caller passes NULL, which is Eq. (1) exactly):
 *
 *   H[0][j] = top[j]            (j = 0..m)
 *   H[i][0] = left[i]           (i = 0..n),   top[0] == left[0]
 *   H[i][j] = H[i-1][j-1] + 1              if a[i-1] == b[j-1]
 *           = max(H[i-1][j], H[i][j-1])    otherwise      (1<=i<=n, 1<=j<=m)
 *
 * Outputs: L = H[n][m], bottom_row[j] = H[n][j] (j = 0..m),
 * right_col[i] = H[i][m] (i = 0..n).
 *
 * Algorithm: the textbook two-row sweep (row i from row i-1), O(nm) time,
 * O(m) space.  No blocking, no SIMD, no threads inside one pair.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

static int32_t max_i32(int32_t x, int32_t y) { return x > y ? x : y; }

/* Returns ORACLE_OK and writes *len, or a negative error code. */
int oracle_lcs(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
               const int32_t *top, const int32_t *left,
               int32_t *bottom_row, int32_t *right_col, int32_t *len)
{
    if (n < 0 || m < 0) return ORACLE_EINVAL;
    if ((n > 0 && !a) || (m > 0 && !b)) return ORACLE_EINVAL;
    if (top && left && top[0] != left[0]) return ORACLE_EINVAL;

    int32_t *prev = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    if (!prev || !cur) { free(prev); free(cur); return ORACLE_ENOMEM; }

    /* row 0 */
    for (int64_t j = 0; j <= m; ++j) prev[j] = top ? top[j] : 0;
    if (right_col) right_col[0] = prev[m];

    for (int64_t i = 1; i <= n; ++i) {
        cur[0] = left ? left[i] : 0;
        const uint8_t ai = a[i - 1];
        for (int64_t j = 1; j <= m; ++j) {
            if (ai == b[j - 1])
                cur[j] = prev[j - 1] + 1;
            else
                cur[j] = max_i32(prev[j], cur[j - 1]);
        }
        if (right_col) right_col[i] = cur[m];
        int32_t *t = prev; prev = cur; cur = t;
    }
    /* prev now holds row n */
    if (bottom_row) memcpy(bottom_row, prev, (size_t)(m + 1) * sizeof(int32_t));
    if (len) *len = prev[m];
    free(prev);
    free(cur);
    return ORACLE_OK;
}

/* Full (n+1) x (m+1) table, row-major, for small cases only. */
int oracle_lcs_table(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                     const int32_t *top, const int32_t *left, int32_t *H)
{
    if (n < 0 || m < 0 || !H) return ORACLE_EINVAL;
    if (top && left && top[0] != left[0]) return ORACLE_EINVAL;
    const int64_t w = m + 1;
    for (int64_t j = 0; j <= m; ++j) H[j] = top ? top[j] : 0;
    for (int64_t i = 1; i <= n; ++i) {
        H[i * w] = left ? left[i] : 0;
        for (int64_t j = 1; j <= m; ++j) {
            if (a[i - 1] == b[j - 1])
                H[i * w + j] = H[(i - 1) * w + (j - 1)] + 1;
            else
                H[i * w + j] = max_i32(H[(i - 1) * w + j], H[i * w + (j - 1)]);
        }
    }
    return ORACLE_OK;
}

/* ---- many independent pairs, spread over host threads (pairs are
 *      independent, so this is only a loop over oracle_lcs) ---- */
struct batch_job {
    const uint8_t *a_cat; const int64_t *a_off;
    const uint8_t *b_cat; const int64_t *b_off;
    int32_t *len; int32_t *rows_cat; const int64_t *row_off;
    int32_t *cols_cat; const int64_t *col_off;
    int64_t npairs;
    int64_t next;              /* shared work counter */
    pthread_mutex_t mu;
    int status;
};

static void *batch_worker(void *arg)
{
    struct batch_job *J = (struct batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t k = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (k >= J->npairs) break;
        const int64_t n = J->a_off[k + 1] - J->a_off[k];
        const int64_t m = J->b_off[k + 1] - J->b_off[k];
        int32_t *row = J->rows_cat ? J->rows_cat + J->row_off[k] : NULL;
        int32_t *col = J->cols_cat ? J->cols_cat + J->col_off[k] : NULL;
        int rc = oracle_lcs(J->a_cat + J->a_off[k], n, J->b_cat + J->b_off[k], m,
                            NULL, NULL, row, col, J->len + k);
        if (rc != ORACLE_OK) {
            pthread_mutex_lock(&J->mu);
            J->status = rc;
            pthread_mutex_unlock(&J->mu);
        }
    }
    return NULL;
}

int oracle_lcs_batch(const uint8_t *a_cat, const int64_t *a_off,
                     const uint8_t *b_cat, const int64_t *b_off, int64_t npairs,
                     int32_t *len, int32_t *rows_cat, const int64_t *row_off,
                     int32_t *cols_cat, const int64_t *col_off, int threads)
{
    if (npairs < 0 || !len) return ORACLE_EINVAL;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    struct batch_job J;
    J.a_cat = a_cat; J.a_off = a_off; J.b_cat = b_cat; J.b_off = b_off;
    J.len = len; J.rows_cat = rows_cat; J.row_off = row_off;
    J.cols_cat = cols_cat; J.col_off = col_off;
    J.npairs = npairs; J.next = 0; J.status = ORACLE_OK;
    pthread_mutex_init(&J.mu, NULL);
    pthread_t tid[256];
    int started = 0;
    for (int t = 0; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, batch_worker, &J) != 0) break;
        ++started;
    }
    if (started == 0) batch_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    pthread_mutex_destroy(&J.mu);
    return J.status;
}
