// Global alignment with affine gap costs (Gotoh's recurrence, the variant
// the footnote to Eq. (1) of the paper names): row-band kernel, host plan and
// the C ABI of include/paco_affine.h.
//
// Layout.  A pair's rows are cut into bands of 32 lanes x R rows; one warp
// owns one band and sweeps every column.  Inside a band the rows run skewed
// along anti-diagonals: at step t, band row i (lane i / R, slot i % R)
// computes column t - i.  The R cells a lane computes in one step are then
// independent of each other; each takes (H, F, symbol) of the row above from
// the previous step: from its own registers, from the lane above by one
// shuffle, or, for the band's first row, from a 32-column staging buffer in
// shared memory.  The band's last row is parked in shared memory by its
// lane, one predicated store per step, and published once per 32 steps as
// one 64-bit word per column in global memory: H, H - F and the launch's
// tag, written and read as single 64-bit accesses, so the band below can
// tell a published word from a stale one without fences or flags.  The band below loads the words of the next
// 32 columns one chunk ahead and checks their tags when it stages them.
// Bands are jobs taken from an atomic ticket in an order in which every band
// comes after the band above it, so a band only ever waits for a running one.
#include "../../include/paco_affine.h"
#include "bp_device.cuh"
#include "ctx.hpp"
#include "paco_internal.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

namespace paco {
namespace {

// -infinity of the kernel: below every reachable score (they lie within
// +-2^29 by the argument checks) with room to subtract scores for the few
// hundred steps a row runs before its first column.
constexpr int kNeg = -(1 << 30);
constexpr int kAffChunk = 32;           // columns per staging chunk of a band's first row (one per lane)
constexpr int kAffWarps = 4;            // warps per CTA (independent job takers)
constexpr int kNoSym = -1;              // column symbol outside [1, m]: never equal
constexpr int kDeadRow = 256;           // row symbol of a row past the band: never equal

struct AffJob {
    int64_t a_off;     // first row symbol of the band
    int64_t b_off;     // first column symbol of the pair
    int64_t in_off;    // hbuf word of the band above's column 0, or -1 (first band)
    int64_t out_off;   // hbuf word of this band's column 0, or -1 (last band)
    int32_t r0;        // DP rows above the band (its rows are r0+1 .. r0+nr)
    int32_t nr;        // rows in the band, 1 .. 32 R
    int32_t m;         // columns of the pair
    int32_t pair;
    int32_t in_job;    // job index of the band above, or -1 (first band)
    int32_t last;      // 1: last band of the pair
    int32_t pad[2];
};
static_assert(sizeof(AffJob) == 64, "job descriptor is one 64-byte line");

struct AffArgs {
    const uint8_t *a_cat;
    const uint8_t *b_cat;
    const AffJob *jobs;
    int njobs;
    uint64_t *hbuf;           // tagged words of each band's last row, per column
    int *ticket;              // job ticket (zeroed before launch)
    int *err;
    int32_t *score;           // per pair
    int32_t *bottom_row;      // optional: H[n][j], pair k at row_off[k]
    const int64_t *row_off;
    int32_t *right_col;       // optional: H[i][m], pair k at col_off[k]
    const int64_t *col_off;
    int gm, gx, go, ge;
    uint32_t tag;             // tag of this launch, 1 .. kTagMask
    long long wait_limit_ns;
    int stall_job;            // tests: job whose input words never carry the tag (-1: none)
};

// Word of a band's last row at one column: bits 0..31 H, bits 32..50
// H - F (0 <= H - F <= match + 2 (open + extend) < 2^19 because H >= F and
// H[i][j] - H[i-1][j] <= match + open + extend), bits 51..63 the tag.
constexpr int kTagShift = 51;
constexpr uint32_t kTagMask = 0x1fff;
static __device__ __forceinline__ uint64_t pack_hf(int h, int f, uint32_t tag) {
    return (uint64_t)(uint32_t)h | ((uint64_t)(uint32_t)(h - f) << 32) | ((uint64_t)tag << kTagShift);
}
static __device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Raw inputs of the band's first row at column `col` (lanes 0..15 of a
// chunk): the word of the band above (0 for the first band or past column
// m) and the column symbol.
struct ChunkIn {
    uint64_t w;
    int sym;
};
static __device__ __forceinline__ ChunkIn load_chunk(const AffArgs &P, const AffJob &J, int col) {
    ChunkIn c{0, kNoSym};
    if ((threadIdx.x & 31) < kAffChunk && col <= J.m) {
        if (J.in_job >= 0) c.w = dev::ld_relaxed_u64(P.hbuf + J.in_off + col);
        if (col >= 1) c.sym = (int)P.b_cat[J.b_off + col - 1];
    }
    return c;
}

// Slow path of settle_chunk: reload the stale words until every lane's word
// carries `tag` (bounded wait).  Scalar arguments only, so the band's state
// stays in registers.  Returns the word; *ok = 0 on timeout or a raised error.
struct Settled {
    uint64_t w;
    int ok;
};
static __device__ __noinline__ Settled settle_slow(const uint64_t *src, bool need, uint64_t w, uint32_t tag, int *err,
                                                   long long limit) {
    bool ready = !need || (uint32_t)(w >> kTagShift) == tag;
    const uint64_t t0 = dev::global_ns();
    for (int spin = 0;; ++spin) {
        if (spin > 8) __nanosleep(32);
        if (!ready) {
            w = dev::ld_relaxed_u64(src);
            ready = (uint32_t)(w >> kTagShift) == tag;
        }
        if (__all_sync(dev::kFull, ready)) return Settled{w, 1};
        int bad = 0;
        if ((threadIdx.x & 31) == 0) {
            if (dev::ld_relaxed_i32(err) != 0) {
                bad = 1;
            } else if ((long long)(dev::global_ns() - t0) > limit) {
                dev::raise_error(err, kEtimeout);
                bad = 1;
            }
        }
        if (__shfl_sync(dev::kFull, bad, 0)) return Settled{w, 0};
    }
}

// Makes sure every word of a chunk loaded earlier carries this launch's tag;
// false on timeout or a raised error.  Warp-uniform.
static __device__ __forceinline__ bool settle_chunk(const AffArgs &P, const AffJob &J, int col, ChunkIn &c,
                                                    uint32_t want) {
    const bool need = J.in_job >= 0 && (threadIdx.x & 31) < kAffChunk && col <= J.m;
    const bool ready = !need || (uint32_t)(c.w >> kTagShift) == want;
    if (__all_sync(dev::kFull, ready)) return true;
    const Settled r = settle_slow(P.hbuf + J.in_off + col, need, c.w, want, P.err, P.wait_limit_ns);
    c.w = r.w;
    return r.ok != 0;
}

// (H, F, symbol) entering the band's first row at column `col`.
static __device__ __forceinline__ int4 band_input(const AffArgs &P, const AffJob &J, int col, const ChunkIn &c) {
    if (col > J.m) return make_int4(kNeg, kNeg, kNoSym, 0);
    int4 v;
    if (J.in_job < 0) {
        v.x = col == 0 ? 0 : -(P.go + P.ge * col);  // H[0][col]
        v.y = kNeg;                                   // F[0][col]
    } else {
        v.x = (int)(uint32_t)c.w;
        v.y = v.x - (int)((c.w >> 32) & 0x7ffff);
    }
    v.z = c.sym;
    v.w = 0;
    return v;
}

template <int R>
struct BandState {
    int as[R];                     // row symbols
    int H[R];                      // H of the slot's last cell
    int G[R];                      // that H - (open + extend): opens a gap right or down
    int F[R], E[R], D[R], B[R];
    int rc[R];                     // H[row][m]
};

// One step of the band: every slot's cell on its anti-diagonal.  No
// branches and no memory operations besides the shuffles, so the unrolled
// steps of a chunk form one block the compiler can interleave.  CAPTURE
// records H at column m.
template <int R, bool CAPTURE>
static __device__ __forceinline__ void band_step(BandState<R> &S, const int4 in, int t, int lane, int m, int gm,
                                                 int gx, int ge, int goe) {
    int hu0 = __shfl_up_sync(dev::kFull, S.H[R - 1], 1);
    int fu0 = __shfl_up_sync(dev::kFull, S.F[R - 1], 1);
    int bu0 = __shfl_up_sync(dev::kFull, S.B[R - 1], 1);
    if (lane == 0) {
        hu0 = in.x;
        fu0 = in.y;
        bu0 = in.z;
    }
    const int gu0 = hu0 - goe;
#pragma unroll
    for (int k = R - 1; k >= 0; --k) {
        const int hu = k ? S.H[k - 1] : hu0;   // H[i-1][j]
        const int gu = k ? S.G[k - 1] : gu0;   // H[i-1][j] - open - extend
        const int fu = k ? S.F[k - 1] : fu0;   // F[i-1][j]
        const int bu = k ? S.B[k - 1] : bu0;   // symbol of column j
        const int s = S.as[k] == bu ? gm : -gx;
        const int e = max(S.E[k] - ge, S.G[k]);
        const int f = max(fu - ge, gu);
        const int h = max(max(S.D[k] + s, e), f);
        S.D[k] = hu;
        S.E[k] = e;
        S.F[k] = f;
        S.H[k] = h;
        S.G[k] = h - goe;
        S.B[k] = bu;
        if (CAPTURE && t == m + lane * R + k) S.rc[k] = h;
    }
}

// The band's last row over a chunk of steps: lane u holds (H, F) of step
// base + u, i.e. column base + u - (nr - 1).
struct OutChunk {
    int h, f;
};

// Publish the gathered chunk whose first step is `base` (steps below T).
static __device__ __forceinline__ void flush_out(const AffArgs &P, const AffJob &J, const OutChunk &o, int lane,
                                                 int base, int T, uint64_t *out) {
    const int j = base + lane - (J.nr - 1);
    if (lane < kAffChunk && base + lane < T && j >= 0 && j <= J.m) {
        if (!J.last) {
            st_relaxed_u64(out + j, pack_hf(o.h, o.f, P.tag));
        } else {
            if (P.bottom_row) P.bottom_row[P.row_off[J.pair] + j] = o.h;
            if (j == J.m) P.score[J.pair] = o.h;
        }
    }
}

template <int R, int KL, bool PAIR>
static __device__ __forceinline__ void affine_band(const AffArgs &P, const AffJob &J, int jid, int4 (*stage)[kAffChunk],
                                                   int2 *sout) {
    const int lane = threadIdx.x & 31;
    const int m = J.m, nr = J.nr;
    const int gm = P.gm, gx = P.gx, ge = P.ge, goe = P.go + P.ge;
    const int last_lane = (nr - 1) / R;
    BandState<R> S;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r = lane * R + k;
        S.as[k] = r < nr ? (int)P.a_cat[J.a_off + r] : kDeadRow;
        S.H[k] = S.F[k] = S.E[k] = S.D[k] = S.G[k] = kNeg;
        S.B[k] = kNoSym;
        S.rc[k] = kNeg;
    }
    uint64_t *out = J.last ? nullptr : P.hbuf + J.out_off;
    OutChunk o{kNeg, kNeg};
    // the last row's lane parks (H, F) of step u in the warp's shared slot
    // u (one predicated store per step); lanes 0..15 take them at the
    // chunk's end
    const bool is_last = lane == last_lane;
#define COLLECT(u) do { if (is_last) sout[u] = make_int2(S.H[KL], S.F[KL]); } while (0)
#define GATHER() do { __syncwarp(); if (lane < kAffChunk) { const int2 v = sout[lane]; o.h = v.x; o.f = v.y; } __syncwarp(); } while (0)
    // the tag the band's input words must carry (a value no word carries
    // for the test-only stalled job)
    const uint32_t want = jid == P.stall_job ? kTagMask + 1 : P.tag;

    // chunk 0 settled into the stage, chunk 1 loading into registers
    ChunkIn cur = load_chunk(P, J, lane);
    if (!settle_chunk(P, J, lane, cur, want)) return;
    if (lane < kAffChunk) stage[0][lane] = band_input(P, J, lane, cur);
    cur = load_chunk(P, J, kAffChunk + lane);
    __syncwarp();

    const int T = m + nr;              // steps: the last row reaches column m at T - 1
    const int hot = (m / kAffChunk) * kAffChunk;   // steps before `hot` never reach column m
    // Every chunk runs as one block of 32 steps (unrolled), the chunks from
    // `hot` on with the capture of column m (the right column).  The steps
    // of the last chunk past T - 1 touch only cells beyond the table, which
    // nothing reads.  The band below waits for this band's last chunk, so a
    // slow tail here would delay every band after it.  A single pair's chain
    // runs one band per warp scheduler and takes the fully unrolled block; a
    // batch, with many warps per SM running different bands, takes blocks
    // half as long (less code for the instruction cache to hold).
    const int nchunks = (T + kAffChunk - 1) / kAffChunk;
    for (int c = 0; c < nchunks; ++c) {
        if (c > 0) {
            GATHER();
            flush_out(P, J, o, lane, (c - 1) * kAffChunk, T, out);
            const int col = c * kAffChunk + lane;
            if (!settle_chunk(P, J, col, cur, want)) return;
            __syncwarp();
            if (lane < kAffChunk) stage[c & 1][lane] = band_input(P, J, col, cur);
            cur = load_chunk(P, J, col + kAffChunk);
            __syncwarp();
        }
        const int4 *st = stage[c & 1];
        const int t0 = c * kAffChunk;
        if (t0 < hot) {
#pragma unroll(PAIR ? kAffChunk : kAffChunk / 2)
            for (int u = 0; u < kAffChunk; ++u) {
                band_step<R, false>(S, st[u], t0 + u, lane, m, gm, gx, ge, goe);
                COLLECT(u);
            }
        } else {
#pragma unroll 4
            for (int u = 0; u < kAffChunk; ++u) {
                band_step<R, true>(S, st[u], t0 + u, lane, m, gm, gx, ge, goe);
                COLLECT(u);
            }
        }
    }
    GATHER();
    flush_out(P, J, o, lane, (nchunks - 1) * kAffChunk, T, out);
#undef COLLECT
#undef GATHER
    if (P.right_col) {
        const int64_t base = P.col_off[J.pair] + J.r0 + 1;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int r = lane * R + k;
            if (r < nr) P.right_col[base + r] = S.rc[k];
        }
        if (J.in_job < 0 && lane == 0) P.right_col[P.col_off[J.pair]] = -(P.go + P.ge * m);  // H[0][m]
    }
}

template <int R, bool PAIR>
__global__ void __launch_bounds__(32 * kAffWarps) k_affine(AffArgs P) {
    __shared__ int4 stage[kAffWarps][2][kAffChunk];
    __shared__ int2 sout[kAffWarps][kAffChunk];
    const int w = threadIdx.x >> 5;
    for (;;) {
        int jid = 0;
        if ((threadIdx.x & 31) == 0) jid = atomicAdd(P.ticket, 1);
        jid = __shfl_sync(dev::kFull, jid, 0);
        if (jid >= P.njobs) return;
        const AffJob J = P.jobs[jid];
        switch ((J.nr - 1) % R) {
            case 0: affine_band<R, 0, PAIR>(P, J, jid, stage[w], sout[w]); break;
            case 1: affine_band<R, 1, PAIR>(P, J, jid, stage[w], sout[w]); break;
            case 2: if (R > 2) affine_band<R, (R > 2 ? 2 : 0), PAIR>(P, J, jid, stage[w], sout[w]); break;
            case 3: if (R > 3) affine_band<R, (R > 3 ? 3 : 0), PAIR>(P, J, jid, stage[w], sout[w]); break;
            case 4: if (R > 4) affine_band<R, (R > 4 ? 4 : 0), PAIR>(P, J, jid, stage[w], sout[w]); break;
            case 5: if (R > 5) affine_band<R, (R > 5 ? 5 : 0), PAIR>(P, J, jid, stage[w], sout[w]); break;
            case 6: if (R > 6) affine_band<R, (R > 6 ? 6 : 0), PAIR>(P, J, jid, stage[w], sout[w]); break;
            case 7: if (R > 7) affine_band<R, (R > 7 ? 7 : 0), PAIR>(P, J, jid, stage[w], sout[w]); break;
        }
    }
}

// Pairs with n == 0 or m == 0: the closed forms of the boundary rows.
__global__ void k_affine_degenerate(const int32_t *pairs, int count, const int64_t *a_off, const int64_t *b_off,
                                    int go, int ge, int32_t *score, int32_t *bottom_row, const int64_t *row_off,
                                    int32_t *right_col, const int64_t *col_off) {
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const int k = pairs[q];
        const int64_t n = a_off[k + 1] - a_off[k], m = b_off[k + 1] - b_off[k];
        auto gap = [&](int64_t len) { return len == 0 ? 0 : -(int)(go + ge * len); };
        if (threadIdx.x == 0) score[k] = gap(n + m);
        if (bottom_row)
            for (int64_t j = threadIdx.x; j <= m; j += blockDim.x) bottom_row[row_off[k] + j] = gap(n + j);
        if (right_col)
            for (int64_t i = threadIdx.x; i <= n; i += blockDim.x) right_col[col_off[k] + i] = gap(i + m);
    }
}

int aff_occupancy(int R) {
    int blocks = 0;
    cudaError_t e = R == 8   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_affine<8, false>, 32 * kAffWarps, 0)
                    : R == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_affine<2, false>, 32 * kAffWarps, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_affine<4, false>, 32 * kAffWarps, 0);
    return e == cudaSuccess ? std::max(blocks, 1) : 1;
}

}  // namespace

// Scratch of the affine path, owned by the context.
struct AffineState {
    DevBuf jobs, hbuf, flags, offs, degen;
    uint32_t tag = 0;             // tag of the last launch (0: none yet)
    std::vector<int64_t> key;     // a_off and b_off of the planned layout
    int plan_rows = 0, njobs = 0, ndegen = 0;
    std::vector<AffJob> h_jobs;
    std::vector<int64_t> h_offs;
};

void affine_state_free(AffineState *A) {
    if (!A) return;
    for (DevBuf *b : {&A->jobs, &A->hbuf, &A->flags, &A->offs, &A->degen})
        if (b->ptr) cudaFree(b->ptr);
    delete A;
}

static bool scores_ok(const paco_affine_scores *s) {
    auto in = [](int32_t v) { return v >= 0 && v <= 65535; };
    return s && in(s->match) && in(s->mismatch) && in(s->gap_open) && in(s->gap_extend);
}

static bool pair_fits(const paco_affine_scores &s, int64_t n, int64_t m) {
    const int64_t lim = (int64_t)1 << 29;
    return (int64_t)s.match * std::min(n, m) <= lim && 2 * (int64_t)s.gap_open + (int64_t)s.gap_extend * (n + m) <= lim;
}

// Plan and launch: pairs (host offsets), rows of pair k = a side.
static int run_affine(paco_ctx *ctx, const uint8_t *a_cat, const int64_t *h_a_off, const uint8_t *b_cat,
                      const int64_t *h_b_off, int npairs, const paco_affine_scores &sc, int32_t *d_score,
                      int32_t *bottom_row, int32_t *right_col, cudaStream_t st) {
    if (!ctx->affine) ctx->affine = new (std::nothrow) AffineState();
    AffineState *A = ctx->affine;
    if (!A) return PACO_ENOMEM;
    int R = ctx->opt_affine_rows ? ctx->opt_affine_rows : 4;
    const int band = 32 * R;

    // The plan depends only on the pair lengths and R: a call with the same
    // layout as the last one reuses the uploaded jobs and offsets.
    const size_t np1 = (size_t)npairs + 1;
    bool same = A->plan_rows == R && A->key.size() == 2 * np1;
    for (size_t k = 0; same && k < np1; ++k) same = A->key[k] == h_a_off[k] && A->key[np1 + k] == h_b_off[k];
    cudaError_t e = cudaSuccess;
    if (!same) {
        // offsets: a_off, b_off, row_off, col_off (npairs + 1 each)
        A->h_offs.assign(4 * np1, 0);
        int64_t *ao = A->h_offs.data(), *bo = ao + np1, *ro = bo + np1, *co = ro + np1;
        for (size_t k = 0; k < np1; ++k) {
            ao[k] = h_a_off[k];
            bo[k] = h_b_off[k];
        }
        std::vector<int32_t> degen;
        std::vector<int> order;
        int max_bands = 0;
        for (int k = 0; k < npairs; ++k) {
            const int64_t n = ao[k + 1] - ao[k], m = bo[k + 1] - bo[k];
            ro[k + 1] = ro[k] + m + 1;
            co[k + 1] = co[k] + n + 1;
            if (n == 0 || m == 0) {
                degen.push_back(k);
            } else {
                order.push_back(k);
                max_bands = std::max(max_bands, (int)((n + band - 1) / band));
            }
        }
        // bands level by level, larger pairs first within a level: every band
        // after the band above it
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return (ao[x + 1] - ao[x]) * (bo[x + 1] - bo[x]) > (ao[y + 1] - ao[y]) * (bo[y + 1] - bo[y]);
        });
        A->h_jobs.clear();
        std::vector<int> prev_job(npairs, -1);
        std::vector<int64_t> prev_out(npairs, -1);
        int64_t hcols = 0;
        for (int lvl = 0; lvl < max_bands; ++lvl) {
            for (int k : order) {
                const int64_t n = ao[k + 1] - ao[k], m = bo[k + 1] - bo[k];
                const int64_t r0 = (int64_t)lvl * band;
                if (r0 >= n) continue;
                AffJob J{};
                J.r0 = (int32_t)r0;
                J.nr = (int32_t)std::min<int64_t>(band, n - r0);
                J.m = (int32_t)m;
                J.pair = k;
                J.a_off = ao[k] + r0;
                J.b_off = bo[k];
                J.in_job = prev_job[k];
                J.in_off = prev_out[k];
                J.last = r0 + J.nr == n;
                J.out_off = -1;
                if (!J.last) {
                    J.out_off = hcols;
                    hcols += m + 1;
                }
                prev_job[k] = (int)A->h_jobs.size();
                prev_out[k] = J.out_off;
                A->h_jobs.push_back(J);
            }
        }
        const int njobs = (int)A->h_jobs.size();
        int rc;
        if ((rc = ensure_bytes(ctx, A->offs, A->h_offs.size() * 8)) != PACO_OK) return rc;
        if ((rc = ensure_bytes(ctx, A->jobs, std::max<size_t>(1, njobs) * sizeof(AffJob))) != PACO_OK) return rc;
        if ((rc = ensure_bytes(ctx, A->flags, 16)) != PACO_OK) return rc;
        if ((rc = ensure_bytes(ctx, A->hbuf, std::max<int64_t>(1, hcols) * 8)) != PACO_OK) return rc;
        if ((rc = ensure_bytes(ctx, A->degen, std::max<size_t>(1, degen.size()) * 4)) != PACO_OK) return rc;
        e = cudaMemcpyAsync(A->offs.ptr, A->h_offs.data(), A->h_offs.size() * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && njobs)
            e = cudaMemcpyAsync(A->jobs.ptr, A->h_jobs.data(), (size_t)njobs * sizeof(AffJob), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !degen.empty())
            e = cudaMemcpyAsync(A->degen.ptr, degen.data(), degen.size() * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // pageable staging must be read before reuse
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "affine plan upload");
        A->key.assign(h_a_off, h_a_off + np1);
        A->key.insert(A->key.end(), h_b_off, h_b_off + np1);
        A->plan_rows = R;
        A->njobs = njobs;
        A->ndegen = (int)degen.size();
    }
    const int njobs = A->njobs, ndegen = A->ndegen;
    if (e == cudaSuccess) e = cudaMemsetAsync(A->flags.ptr, 0, 4, st);
    // a new tag per launch; after the 13-bit tag wraps, words of the launch
    // that used the same tag are cleared first
    A->tag = A->tag % kTagMask + 1;
    if (e == cudaSuccess && A->tag == 1) e = cudaMemsetAsync(A->hbuf.ptr, 0, A->hbuf.bytes, st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "affine launch set-up");
    const int64_t *d_off = (const int64_t *)A->offs.ptr;
    if (ndegen) {
        k_affine_degenerate<<<std::min(ndegen, 4096), 128, 0, st>>>(
            (const int32_t *)A->degen.ptr, ndegen, d_off, d_off + np1, sc.gap_open, sc.gap_extend,
            d_score, bottom_row, d_off + 2 * np1, right_col, d_off + 3 * np1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "k_affine_degenerate");
    }
    if (njobs) {
        AffArgs P{};
        P.a_cat = a_cat;
        P.b_cat = b_cat;
        P.jobs = (const AffJob *)A->jobs.ptr;
        P.njobs = njobs;
        P.hbuf = (uint64_t *)A->hbuf.ptr;
        P.tag = A->tag;
        P.ticket = (int *)A->flags.ptr;
        P.err = ctx->err_ptr();
        P.score = d_score;
        P.bottom_row = bottom_row;
        P.row_off = d_off + 2 * np1;
        P.right_col = right_col;
        P.col_off = d_off + 3 * np1;
        P.gm = sc.match;
        P.gx = sc.mismatch;
        P.go = sc.gap_open;
        P.ge = sc.gap_extend;
        P.wait_limit_ns = ctx->wait_limit_ns;
        P.stall_job = ctx->test_stall;
        // The bands of one pair form one chain whose pace is its slowest
        // band's, so a single pair gets one CTA per SM (one band per warp
        // scheduler); independent pairs fill every resident slot.
        const int per_sm = npairs == 1 ? 1 : aff_occupancy(R);
        const int grid = std::min(ctx->sms * per_sm, (njobs + kAffWarps - 1) / kAffWarps);
        cudaEventRecord(ctx->ev0, st);
        const bool pair = npairs == 1;
        if (R == 8) pair ? k_affine<8, true><<<grid, 32 * kAffWarps, 0, st>>>(P) : k_affine<8, false><<<grid, 32 * kAffWarps, 0, st>>>(P);
        else if (R == 2) pair ? k_affine<2, true><<<grid, 32 * kAffWarps, 0, st>>>(P) : k_affine<2, false><<<grid, 32 * kAffWarps, 0, st>>>(P);
        else pair ? k_affine<4, true><<<grid, 32 * kAffWarps, 0, st>>>(P) : k_affine<4, false><<<grid, 32 * kAffWarps, 0, st>>>(P);
        e = cudaGetLastError();
        cudaEventRecord(ctx->ev1, st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "k_affine");
        ctx->timed = true;
        ctx->timed_name = "k_affine";
    }
    return PACO_OK;
}

}  // namespace paco

using namespace paco;

extern "C" {

int paco_affine_align(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                      const paco_affine_scores *scores, int32_t *d_score, int32_t *d_bottom_row,
                      int32_t *d_right_col, void *stream) {
    if (!ctx || !d_score || !scores_ok(scores)) return PACO_EINVAL;
    if (n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL) return PACO_EINVAL;
    if ((n > 0 && !a) || (m > 0 && !b) || !pair_fits(*scores, n, m)) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    // more bands than columns keeps more warps busy: rows = the longer side
    // (the table of (b, a) is the transpose, with the same score)
    const bool tr = m > n;
    int64_t ao[2] = {0, tr ? m : n}, bo[2] = {0, tr ? n : m};
    return run_affine(ctx, tr ? b : a, ao, tr ? a : b, bo, 1, *scores, d_score, tr ? d_right_col : d_bottom_row,
                      tr ? d_bottom_row : d_right_col, (cudaStream_t)stream);
}

int paco_affine_batch(paco_ctx *ctx, const uint8_t *a_cat, const int64_t *a_off, const uint8_t *b_cat,
                      const int64_t *b_off, int32_t npairs, const paco_affine_scores *scores, int32_t *d_score,
                      void *stream) {
    if (!ctx || npairs < 0 || !scores_ok(scores) || (npairs > 0 && (!a_off || !b_off || !d_score))) return PACO_EINVAL;
    if (npairs == 0) return PACO_OK;
    if (a_off[0] != 0 || b_off[0] != 0) return PACO_EINVAL;
    for (int k = 0; k < npairs; ++k) {
        const int64_t n = a_off[k + 1] - a_off[k], m = b_off[k + 1] - b_off[k];
        if (n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL || !pair_fits(*scores, n, m)) return PACO_EINVAL;
    }
    if ((a_off[npairs] > 0 && !a_cat) || (b_off[npairs] > 0 && !b_cat)) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    return run_affine(ctx, a_cat, a_off, b_cat, b_off, npairs, *scores, d_score, nullptr, nullptr,
                      (cudaStream_t)stream);
}

int paco_affine_align_host(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                           const paco_affine_scores *scores, int32_t *score, int32_t *bottom_row,
                           int32_t *right_col, void *stream) {
    if (!ctx || !score || !scores_ok(scores)) return PACO_EINVAL;
    if (n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL) return PACO_EINVAL;
    if ((n > 0 && !a) || (m > 0 && !b) || !pair_fits(*scores, n, m)) return PACO_EINVAL;
    cudaStream_t st;
    int rc;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        st = stream ? (cudaStream_t)stream : ctx->own_stream;
        if ((rc = ensure_bytes(ctx, ctx->h_a, (size_t)n + 16)) != PACO_OK) return rc;
        if ((rc = ensure_bytes(ctx, ctx->h_b, (size_t)m + 16)) != PACO_OK) return rc;
        if ((rc = ensure_bytes(ctx, ctx->h_row, ((size_t)m + 1) * 4)) != PACO_OK) return rc;
        if ((rc = ensure_bytes(ctx, ctx->h_col, ((size_t)n + 1) * 4)) != PACO_OK) return rc;
        if ((rc = ensure_bytes(ctx, ctx->h_len, 16)) != PACO_OK) return rc;
        cudaError_t e = cudaSuccess;
        if (n) e = cudaMemcpyAsync(ctx->h_a.ptr, a, (size_t)n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && m) e = cudaMemcpyAsync(ctx->h_b.ptr, b, (size_t)m, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "host inputs to device");
    }
    rc = paco_affine_align(ctx, (const uint8_t *)ctx->h_a.ptr, n, (const uint8_t *)ctx->h_b.ptr, m, scores,
                           (int32_t *)ctx->h_len.ptr, bottom_row ? (int32_t *)ctx->h_row.ptr : nullptr,
                           right_col ? (int32_t *)ctx->h_col.ptr : nullptr, st);
    if (rc != PACO_OK) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaError_t e = cudaSuccess;
    if (bottom_row) e = cudaMemcpyAsync(bottom_row, ctx->h_row.ptr, ((size_t)m + 1) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && right_col)
        e = cudaMemcpyAsync(right_col, ctx->h_col.ptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost, st);
    int32_t hs = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, ctx->h_len.ptr, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "device outputs to host");
    *score = hs;
    int err = 0;
    e = cudaMemcpy(&err, ctx->err_ptr(), sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "read error word");
    if (err != 0) {
        cudaMemset(ctx->err_ptr(), 0, sizeof(int));
        return err;
    }
    return PACO_OK;
}

}  // extern "C"
