/*
 * CPU CROSS-CHECK for the LCS oracle (test infrastructure only).
 *
 * Only the tests use this file.  It shares no code with the CUDA library
 * (nor with lcs_oracle.c) and must never be linked into the library.
 *
 * A second, independent way to the same numbers as the two-row DP of
 * lcs_oracle.c: the bit-vector LCS of Allison & Dix (IPL 23, 1986) in the
 * form of Crochemore et al. (IPL 80, 2001) / Hyyro (2004), written here
 * from those papers with multi-word vectors of 64-bit words.  For the rows of
 * a (bit i = row i) and column j of b with match vector
 * M = {i : a[i] == b[j]}, one column is
 *
 *     V' = (V + (V & M)) | (V & ~M)           (addition carries across words)
 *
 * starting from V = all ones.  Bit i of V is 0 exactly when the table has a
 * vertical step between rows i and i+1 at that column, so
 *   H[n][j] = number of zero bits of V after column j   (the bottom row)
 *   H[i][m] = zero bits among the first i bits of the final V (the column).
 * Zero first row and column only (the form those papers state).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int popc64(uint64_t x) {
    int c = 0;
    while (x) {
        x &= x - 1;
        ++c;
    }
    return c;
}

/* bottom_row[m+1], right_col[n+1] may be NULL.  Returns 0, or -1 on
 * allocation failure / bad arguments. */
int oracle_lcs_bitpar(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, int32_t *L,
                      int32_t *bottom_row, int32_t *right_col) {
    if (n < 0 || m < 0) return -1;
    const int64_t nw = (n + 63) / 64;
    uint64_t *V = (uint64_t *)malloc((size_t)(nw ? nw : 1) * 8);
    uint64_t *peq = (uint64_t *)calloc((size_t)256 * (size_t)(nw ? nw : 1), 8);
    if (!V || !peq) {
        free(V);
        free(peq);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) peq[(size_t)a[i] * (size_t)nw + (size_t)(i / 64)] |= (uint64_t)1 << (i % 64);
    for (int64_t w = 0; w < nw; ++w) V[w] = ~(uint64_t)0;
    const uint64_t tail = (n % 64) ? (((uint64_t)1 << (n % 64)) - 1) : ~(uint64_t)0;
    if (bottom_row) bottom_row[0] = 0;
    for (int64_t j = 0; j < m; ++j) {
        const uint64_t *M = peq + (size_t)b[j] * (size_t)nw;
        uint64_t carry = 0;
        int64_t zeros = 0;
        for (int64_t w = 0; w < nw; ++w) {
            const uint64_t v = V[w], x = v & M[w];
            const uint64_t s1 = v + x;
            const uint64_t c1 = s1 < v;
            const uint64_t s = s1 + carry;
            const uint64_t c2 = s < s1;
            carry = c1 | c2;
            V[w] = s | (v & ~M[w]);
            const uint64_t live = (w == nw - 1) ? tail : ~(uint64_t)0;
            zeros += popc64(~V[w] & live);
        }
        if (bottom_row) bottom_row[j + 1] = (int32_t)zeros;
        if (j == m - 1 && L) *L = (int32_t)zeros;
    }
    if (m == 0 && L) *L = 0;
    if (right_col) {
        int32_t acc = 0;
        right_col[0] = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (m > 0 && !((V[i / 64] >> (i % 64)) & 1)) ++acc;
            right_col[i + 1] = acc;
        }
    }
    free(V);
    free(peq);
    return 0;
}
