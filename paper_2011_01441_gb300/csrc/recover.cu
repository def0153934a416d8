// paco_lcs_subsequence: one longest common subsequence, not only its length.
//
// The paper computes the length and notes that returning the subsequence is
// the harder variant (Sec. "PACO LCS", footnote to Eq. (1)).  Recovery here
// follows Hirschberg's linear-space divide and conquer (Hirschberg, CACM
// 18(6), 1975) on top of the boundary engine: a subproblem (rows [i0, i1) of
// a, columns [j0, j1) of b) with at least two rows is cut at the middle row
// h; the bottom row F of (a[i0, h), b[j0, j1)) and the bottom row R of the
// reversed lower half (a[h, i1) reversed against b[j0, j1) reversed) give
// F[j] + R[w - j] = the best LCS through column j0 + j of the cut, and the
// column k with the largest sum (the smallest such column on ties) splits
// the subproblem into (a[i0, h), b[j0, j0 + k)) and (a[h, i1), b[j0 + k, j1)).
// All subproblems of one level go through the batch engine as one launch
// (two pairs each).  A subproblem of at most 31 rows is solved directly by
// one warp: a ballot over the rows gives each column's match word, one
// bit-vector word per column (Allison & Dix / Hyyro, V' = (V + (V & M)) |
// (V & ~M)) is stored, and one lane walks back from the corner.  Every row of
// a ends in exactly one such subproblem, so the matched rows, read in order,
// are the subsequence.
#include "../../include/paco_lcs.h"
#include "ctx.hpp"
#include "paco_internal.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

namespace paco {

namespace {

struct Seg {         // one string piece of a level's batch
    int64_t src;     // first position in the source string
    int64_t dst;     // position in the level's concatenation
    int64_t len;
    int32_t reverse; // 1: copied back to front
    int32_t pad;
};

struct Split {       // one subproblem cut at its middle row
    int64_t row_f;   // offset of F (forward bottom row) in the level's rows
    int64_t row_r;   // offset of R (reversed bottom row)
    int64_t w;       // columns of the subproblem
};

struct Base {        // a subproblem of at most 31 rows, solved by one warp
    int64_t i0, i1, j0, j1;
};

__global__ void k_gather(const uint8_t *src, const Seg *segs, uint8_t *dst) {
    const Seg s = segs[blockIdx.x];
    for (int64_t t = threadIdx.x; t < s.len; t += blockDim.x)
        dst[s.dst + t] = src[s.reverse ? s.src + s.len - 1 - t : s.src + t];
}

// k = argmax_j F[j] + R[w - j], the smallest j on ties.
__global__ void k_split_column(const int32_t *rows, const Split *sp, int64_t *k_out) {
    const Split s = sp[blockIdx.x];
    long long best = -1;  // (value << 32) | (0xffffffff - j): max picks the largest value, then the smallest j
    for (int64_t j = threadIdx.x; j <= s.w; j += blockDim.x) {
        const long long v = (long long)rows[s.row_f + j] + (long long)rows[s.row_r + s.w - j];
        const long long key = (v << 32) | (long long)(0xffffffffLL - j);
        best = key > best ? key : best;
    }
    __shared__ long long red[32];
    for (int o = 16; o > 0; o >>= 1) {
        const long long y = __shfl_down_sync(0xffffffffu, best, o);
        best = y > best ? y : best;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        best = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -1;
        for (int o = 16; o > 0; o >>= 1) {
            const long long y = __shfl_down_sync(0xffffffffu, best, o);
            best = y > best ? y : best;
        }
        if (threadIdx.x == 0) k_out[blockIdx.x] = 0xffffffffLL - (best & 0xffffffffLL);
    }
}

// One warp per base subproblem (h <= 31 rows, w columns, zero boundaries):
// lane r holds a[i0 + r]; column j's match word is the ballot of the lanes
// whose symbol equals b[j]; the warp keeps V (bit r clear = vertical step
// below row r) and lane 0 stores V after each column in vs[j].  Then lane 0
// walks back from (h, w): H(i, j) = zero bits of column j's V below row i.
__global__ void k_base_lcs(const uint8_t *a, const uint8_t *b, const Base *bs, uint32_t *vs, int32_t *match) {
    const Base B = bs[blockIdx.x];
    const int lane = threadIdx.x;
    const int h = (int)(B.i1 - B.i0);
    const int64_t w = B.j1 - B.j0;
    const int ar = lane < h ? (int)a[B.i0 + lane] : 1000;  // rows past h never match
    uint32_t V = 0xffffffffu;
    for (int64_t jb = 0; jb < w; jb += 32) {  // 32 column symbols per coalesced load
        const int bl = jb + lane < w ? (int)b[B.j0 + jb + lane] : -1;
        const int cnt = (int)min((int64_t)32, w - jb);
        for (int jj = 0; jj < cnt; ++jj) {
            const uint32_t M = __ballot_sync(0xffffffffu, ar == __shfl_sync(0xffffffffu, bl, jj));
            V = (V + (V & M)) | (V & ~M);
            if (lane == 0) vs[B.j0 + jb + jj] = V;
        }
    }
    __syncwarp();
    if (lane != 0) return;
    auto H = [&](int i, int64_t j) -> int {  // H[i][j] of the subproblem
        if (i == 0 || j == 0) return 0;
        const uint32_t v = vs[B.j0 + j - 1];
        return __popc(~v & ((1u << i) - 1u));
    };
    int i = h;
    int64_t j = w;
    while (i > 0 && j > 0) {
        if (a[B.i0 + i - 1] == b[B.j0 + j - 1]) {  // Eq. (1): a diagonal step
            match[B.i0 + i - 1] = (int32_t)(B.j0 + j - 1);
            --i;
            --j;
        } else if (H(i - 1, j) == H(i, j)) {
            --i;
        } else {
            --j;
        }
    }
}

constexpr int kCB = 1024;  // rows per compaction block

// Compaction of match[0, n) (>= 0 kept) into (ai, bj) pairs in row order:
// pass 1 counts per block, pass 2 scans the counts, pass 3 writes.
__global__ void k_count(const int32_t *match, int64_t n, int64_t *cnt) {
    const int64_t i = blockIdx.x * (int64_t)kCB + threadIdx.x;
    const int v = (i < n && match[i] >= 0) ? 1 : 0;
    const int c = __syncthreads_count(v);
    if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

__global__ void k_scan_counts(int64_t *cnt, int64_t nb, int32_t *len) {
    if (threadIdx.x != 0) return;
    int64_t acc = 0;
    for (int64_t k = 0; k < nb; ++k) {
        const int64_t c = cnt[k];
        cnt[k] = acc;
        acc += c;
    }
    *len = (int32_t)acc;
}

__global__ void k_write_pairs(const int32_t *match, int64_t n, const int64_t *base, int32_t *ai, int32_t *bj) {
    __shared__ int warp_tot[kCB / 32];
    const int64_t i = blockIdx.x * (int64_t)kCB + threadIdx.x;
    const int v = (i < n && match[i] >= 0) ? 1 : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_tot[w] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int k = 0; k < w; ++k) before += warp_tot[k];
    before += __popc(bal & ((1u << lane) - 1u));
    if (v) {
        const int64_t o = base[blockIdx.x] + before;
        ai[o] = (int32_t)i;
        bj[o] = match[i];
    }
}

struct Sub {
    int64_t i0, i1, j0, j1;
};

template <class T>
int upload(DevBuf &d, const std::vector<T> &v, cudaStream_t st) {
    const size_t bytes = v.size() * sizeof(T);
    if (d.bytes < bytes) {
        if (d.ptr) cudaFreeAsync(d.ptr, st);
        d.ptr = nullptr;
        d.bytes = 0;
        const size_t want = std::max(bytes * 2, (size_t)4096);
        if (cudaMallocAsync(&d.ptr, want, st) != cudaSuccess) return PACO_ENOMEM;
        d.bytes = want;
    }
    if (bytes && cudaMemcpyAsync(d.ptr, v.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return PACO_EDEVICE;
    return PACO_OK;
}

int grow(DevBuf &d, size_t bytes, cudaStream_t st) {
    if (d.bytes >= bytes) return PACO_OK;
    if (d.ptr) cudaFreeAsync(d.ptr, st);
    d.ptr = nullptr;
    d.bytes = 0;
    const size_t want = std::max(bytes * 2, (size_t)4096);
    if (cudaMallocAsync(&d.ptr, want, st) != cudaSuccess) return PACO_ENOMEM;
    d.bytes = want;
    return PACO_OK;
}

}  // namespace

int run_subsequence(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, int32_t *d_ai,
                    int32_t *d_bj, int32_t *d_len, cudaStream_t st) {
    if (!ctx->recover) ctx->recover = batch_state_new(ctx->ticket_ptr(), ctx->err_ptr());
    if (!ctx->recover) return PACO_ENOMEM;
    DevBuf match, seg_a, seg_b, acat, bcat, rows, lens, splits, kbuf, bases, vstore, cnt;
    auto release = [&]() {
        for (DevBuf *d : {&match, &seg_a, &seg_b, &acat, &bcat, &rows, &lens, &splits, &kbuf, &bases, &vstore, &cnt})
            if (d->ptr) cudaFreeAsync(d->ptr, st);
    };
    auto fail = [&](int rc) {
        release();
        return rc;
    };
    int rc;
    if ((rc = grow(match, (size_t)std::max<int64_t>(n, 1) * 4, st)) != PACO_OK) return fail(rc);
    if (cudaMemsetAsync(match.ptr, 0xff, (size_t)std::max<int64_t>(n, 1) * 4, st) != cudaSuccess)
        return fail(PACO_EDEVICE);

    std::vector<Sub> cur;
    if (n > 0 && m > 0) cur.push_back({0, n, 0, m});
    std::vector<Seg> sa, sb;
    std::vector<Split> sp;
    std::vector<Base> base;  // every subproblem of at most 31 rows, solved at the end
    std::vector<int64_t> a_off, b_off, row_off, kh;
    std::vector<Sub> cut;
    while (!cur.empty()) {
        sa.clear();
        sb.clear();
        sp.clear();
        cut.clear();
        a_off.assign(1, 0);
        b_off.assign(1, 0);
        row_off.clear();
        int64_t rows_tot = 0;
        for (const Sub &s : cur) {
            const int64_t h = s.i1 - s.i0, w = s.j1 - s.j0;
            if (h <= 0 || w <= 0) continue;
            if (h <= 31) {
                base.push_back({s.i0, s.i1, s.j0, s.j1});
                continue;
            }
            const int64_t mid = s.i0 + h / 2;
            cut.push_back(s);
            // forward: a[i0, mid) against b[j0, j1)
            sa.push_back({s.i0, a_off.back(), mid - s.i0, 0, 0});
            a_off.push_back(a_off.back() + (mid - s.i0));
            sb.push_back({s.j0, b_off.back(), w, 0, 0});
            b_off.push_back(b_off.back() + w);
            row_off.push_back(rows_tot);
            rows_tot += w + 1;
            // reversed lower half: a[mid, i1) and b[j0, j1), both back to front
            sa.push_back({mid, a_off.back(), s.i1 - mid, 1, 0});
            a_off.push_back(a_off.back() + (s.i1 - mid));
            sb.push_back({s.j0, b_off.back(), w, 1, 0});
            b_off.push_back(b_off.back() + w);
            row_off.push_back(rows_tot);
            rows_tot += w + 1;
            sp.push_back({row_off[row_off.size() - 2], row_off.back(), w});
        }
        if (cut.empty()) break;
        const int32_t np = (int32_t)(2 * cut.size());
        if ((rc = upload(seg_a, sa, st)) != PACO_OK || (rc = upload(seg_b, sb, st)) != PACO_OK ||
            (rc = upload(splits, sp, st)) != PACO_OK)
            return fail(rc);
        if ((rc = grow(acat, (size_t)a_off.back() + 16, st)) != PACO_OK ||
            (rc = grow(bcat, (size_t)b_off.back() + 16, st)) != PACO_OK ||
            (rc = grow(rows, (size_t)rows_tot * 4 + 16, st)) != PACO_OK ||
            (rc = grow(lens, (size_t)np * 4 + 16, st)) != PACO_OK ||
            (rc = grow(kbuf, cut.size() * 8 + 16, st)) != PACO_OK)
            return fail(rc);
        k_gather<<<(unsigned)sa.size(), 256, 0, st>>>(a, (const Seg *)seg_a.ptr, (uint8_t *)acat.ptr);
        k_gather<<<(unsigned)sb.size(), 256, 0, st>>>(b, (const Seg *)seg_b.ptr, (uint8_t *)bcat.ptr);
        if (cudaGetLastError() != cudaSuccess) return fail(PACO_EDEVICE);
        rc = run_batch(ctx, ctx->recover, (const uint8_t *)acat.ptr, a_off.data(), (const uint8_t *)bcat.ptr,
                       b_off.data(), np, (int32_t *)lens.ptr, (int32_t *)rows.ptr, row_off.data(), nullptr, nullptr,
                       st, false, 0, kMaxSigma);
        if (rc != PACO_OK) return fail(rc);
        k_split_column<<<(unsigned)cut.size(), 256, 0, st>>>((const int32_t *)rows.ptr, (const Split *)splits.ptr,
                                                            (int64_t *)kbuf.ptr);
        kh.resize(cut.size());
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(kh.data(), kbuf.ptr, cut.size() * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(set_cuda_error(ctx, e, "subsequence level"));
        int dev_err = 0;
        if (cudaMemcpy(&dev_err, ctx->err_ptr(), sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
            dev_err != 0)
            return fail(dev_err);
        std::vector<Sub> next;
        next.reserve(2 * cut.size());
        for (size_t k = 0; k < cut.size(); ++k) {
            const Sub &s = cut[k];
            const int64_t mid = s.i0 + (s.i1 - s.i0) / 2, col = s.j0 + kh[k];
            next.push_back({s.i0, mid, s.j0, col});
            next.push_back({mid, s.i1, col, s.j1});
        }
        cur.swap(next);
    }
    // the base subproblems (disjoint column ranges: one word per column of b)
    if (!base.empty()) {
        if ((rc = upload(bases, base, st)) != PACO_OK) return fail(rc);
        if ((rc = grow(vstore, (size_t)std::max<int64_t>(m, 1) * 4, st)) != PACO_OK) return fail(rc);
        k_base_lcs<<<(unsigned)base.size(), 32, 0, st>>>(a, b, (const Base *)bases.ptr, (uint32_t *)vstore.ptr,
                                                        (int32_t *)match.ptr);
        if (cudaGetLastError() != cudaSuccess) return fail(PACO_EDEVICE);
    }
    // compaction in row order
    const int64_t nb = (std::max<int64_t>(n, 1) + kCB - 1) / kCB;
    if ((rc = grow(cnt, (size_t)nb * 8 + 16, st)) != PACO_OK) return fail(rc);
    k_count<<<(unsigned)nb, kCB, 0, st>>>((const int32_t *)match.ptr, n, (int64_t *)cnt.ptr);
    k_scan_counts<<<1, 32, 0, st>>>((int64_t *)cnt.ptr, nb, d_len);
    k_write_pairs<<<(unsigned)nb, kCB, 0, st>>>((const int32_t *)match.ptr, n, (const int64_t *)cnt.ptr, d_ai, d_bj);
    cudaError_t e = cudaGetLastError();
    release();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PACO_OK : set_cuda_error(ctx, e, "subsequence compaction");
}

}  // namespace paco

extern "C" int paco_lcs_subsequence(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                                    int32_t *d_ai, int32_t *d_bj, int32_t *d_len, void *stream) {
    if (!ctx || n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL || !d_len) return PACO_EINVAL;
    if ((n > 0 && !a) || (m > 0 && !b)) return PACO_EINVAL;
    if (n > 0 && m > 0 && (!d_ai || !d_bj)) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    return paco::run_subsequence(ctx, a, n, b, m, d_ai, d_bj, d_len, (cudaStream_t)stream);
}
