// Batch of independent pairs in one persistent launch (CUDA-graph captured).
//
// Every pair is a table of Eq. (1) (Tang & Gao, Sec. "PACO LCS") with zero
// first row/column.  Its rows run along the bits of the longer string; the
// rows are cut into segments of at most 32 lanes x 31 rows, each segment is
// one warp job that streams all columns of the pair; a pair taller than one
// warp chains its segments through epoch-tagged carry words in global memory
// (the same hand-off the single-pair strips use).  Jobs are ordered by the
// length of the segment chain they start (critical path first, then the
// largest pair), so the persistent warps, which take jobs from one atomic
// ticket, end together: this is the balanced share of cells per SM the PACO
// partition asks for, here over independent pairs instead of one table.
#include "../../include/paco_lcs.h"
#include "bp_device.cuh"
#include "ctx.hpp"
#include "paco_internal.hpp"

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

namespace paco {

namespace {

using namespace dev;

static __device__ __forceinline__ void st_u32_if(bool p, uint32_t *ptr, uint32_t v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.global.u32 [%1], %2;\n\t}"
                 ::"r"((uint32_t)p), "l"(ptr), "r"(v));
}

enum : uint32_t {
    kTransposed = 1u,
    kInGlobal = 2u,   // top carries from tagged words of an earlier job
    kOutGlobal = 4u,  // bottom carries to tagged words for a later job
    kFinal = 8u,      // the pair's last segment: writes its length
    kLeftIn = 16u,    // tiles: the first column's vertical steps from tagged lane words
    kRightOut = 32u   // tiles: the last column's vertical steps to tagged lane words
};
// Size classes of the streamed side S (bits 8..9 of SegJob::flags); each
// class runs with its own autotuned chunk width.
constexpr int kClassShift = 8;
constexpr int kClasses = 4;
inline int size_class(int64_t S) { return S < 256 ? 0 : (S < 1024 ? 1 : (S < 4096 ? 2 : 3)); }

struct SegJob {
    int64_t rows_off;  // first row of the segment in the rows string (cat offset)
    int64_t cols_off;  // first column of the pair in the column string (cat offset)
    int32_t nrows;     // rows of this segment (1 .. 992)
    int32_t S;         // columns of the pair
    int32_t pair;
    uint32_t flags;
    int64_t hin;       // tagged input carry row (kInGlobal)
    int64_t hout;      // tagged output carry row (kOutGlobal)
    int64_t rword;     // first right-column lane word of the segment, or -1
    int64_t bword;     // first bottom-row step word of the pair (kFinal), or -1
    int64_t vin;       // tiles: first tagged lane word of the left column (kLeftIn)
    int64_t vout;      // tiles: first tagged lane word of the right column (kRightOut)
    int32_t join0;     // tiles: jobs whose completion must be seen first (-1: none),
    int32_t join1;     //   the fork-join order of a divide-and-conquer schedule
    int32_t done;      // tiles: index of this job's completion flag, or -1
    int32_t pad;
};
// (cols_off indexes the column-offset array, not the concatenation)

// One pair's streamed string -> its column-table offsets at a 16-byte
// aligned position of the batch's offset array.
struct ColJob {
    int64_t src;      // offset of the streamed string in its concatenation
    int64_t dst;      // offset in the column-offset array (multiple of 4)
    int64_t len;
    int32_t from_a;   // 1: the streamed string is in a_cat
    int32_t pad;
};

// Symbol c uses match-table row c + 1; row 0 is all zero.  Symbols outside
// the declared alphabet (>= sigma) point at row 0 and raise PACO_EINVAL.
__global__ void k_pair_column_offsets(const uint8_t *a_cat, const uint8_t *b_cat, const ColJob *cj,
                                      uint32_t *coffs, int sigma, int *err) {
    const ColJob J = cj[blockIdx.x];
    const uint8_t *src = (J.from_a ? a_cat : b_cat) + J.src;
    bool bad = false;
    for (int64_t j = threadIdx.x; j < J.len; j += blockDim.x) {
        uint32_t c = src[j];
        if ((int)c >= sigma) {
            bad = true;
            c = 0u;
        } else {
            c += 1u;
        }
        coffs[J.dst + j] = c * 128u;
    }
    if (bad) atomicCAS(err, 0, kEinval);
}

struct BatchArgs {
    const uint8_t *a_cat, *b_cat;
    const uint32_t *coffs;  // column-table offsets, pair by pair (16-byte aligned starts)
    const SegJob *jobs;
    int64_t njobs;
    uint64_t *hbuf;
    uint32_t *rbits;
    uint32_t *bbits;
    int32_t *len;
    int *ticket;
    int *err;
    const uint32_t *epoch_dev;
    long long wait_limit_ns;
    int sigma;       // declared alphabet: symbols are < sigma
    int table_rows;  // rows of the per-warp match table: the zero row, then one per symbol
    int cls_chunk[4];  // chunk width of each size class
    uint64_t *vbuf;    // tiles: tagged lane words of column cuts (kLeftIn / kRightOut)
    uint32_t *done;    // tiles: completion flags (the epoch when done)
};

// One lane waits until a tagged word carries `want`; bounded like every
// wait (on a timeout the error is raised and the stale value returned).
static __device__ __noinline__ uint64_t poll_tagged(const uint64_t *p, uint32_t want, int *err, long long limit) {
    uint64_t v = ld_relaxed_u64(p);
    if ((uint32_t)(v >> 32) == want) return v;
    const uint64_t t0 = global_ns();
    for (;;) {
        v = ld_relaxed_u64(p);
        if ((uint32_t)(v >> 32) == want) return v;
        if (ld_relaxed_i32(err) != 0) return v;
        if ((long long)(global_ns() - t0) > limit) {
            raise_error(err, kEtimeout);
            return v;
        }
    }
}

static __device__ __noinline__ void wait_done(const uint32_t *flag, uint32_t want, int *err, long long limit) {
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v == want || ld_relaxed_i32(err) != 0) return;
        if ((long long)(global_ns() - t0) > limit) {
            raise_error(err, kEtimeout);
            return;
        }
        __nanosleep(64);
    }
}

// Column offsets reach the warp through a shared ring of 32-column words,
// copied kColAhead words ahead (lane 31 trails lane 0 by at most 31*8/32 + 1
// = 9 words); two mirror slots after the ring repeat slots 0 and 1, so a
// lane's window of the next 32 + 2C columns never wraps.
constexpr int kColRing = 32;
constexpr int kColAhead = 8;

// One warp job (a segment of up to 32 lanes x 31 rows of one pair, all its
// columns) with chunk width C.  Lane 31 hands the bottom row on.
template <int C, bool TILES>
static __device__ __forceinline__ void batch_job(const BatchArgs &P, const SegJob &J, const int lane, uint32_t *pm,
                                                 const uint32_t pm_lane, uint32_t *cols_ptr, const uint32_t col_ring,
                                                 const uint32_t epoch) {
    constexpr int K = 32 / C;
    {
        const bool tr = (J.flags & kTransposed) != 0;
        const uint8_t *rows = tr ? P.b_cat : P.a_cat;
        const uint32_t *boff = P.coffs + J.cols_off;
        const int64_t S = J.S;
        const int64_t rbase = J.rows_off + (int64_t)lane * kLaneRows;
        const int left_rows = J.nrows - lane * kLaneRows;
        const int nreal = left_rows <= 0 ? 0 : (left_rows >= kLaneRows ? kLaneRows : left_rows);
        const uint32_t realmask = (1u << nreal) - 1u;
        uint32_t aw[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) aw[k] = 0;
#pragma unroll
        for (int r = 0; r < kLaneRows; ++r)
            if (r < nreal) aw[r >> 2] |= (uint32_t)__ldg(rows + rbase + r) << ((r & 3) * 8);
        bool badsym = false;
#pragma unroll
        for (int r = 0; r < kLaneRows; ++r) {
            if (r < nreal) {
                const uint32_t ch = (aw[r >> 2] >> ((r & 3) * 8)) & 0xffu;
                if ((int)ch < P.sigma) pm[(ch + 1) * 32 + lane] |= 1u << r;
                else badsym = true;
            }
        }
        if (badsym) atomicCAS(P.err, 0, kEinval);
        uint32_t V = 0xffffffffu;  // zero first column: no vertical steps; bit 31 held at 1
        if (TILES && (J.join0 >= 0 || J.join1 >= 0)) {  // tiles: the fork-join order
            if (lane == 0) {
                if (J.join0 >= 0) wait_done(P.done + J.join0, epoch, P.err, P.wait_limit_ns);
                if (J.join1 >= 0) wait_done(P.done + J.join1, epoch, P.err, P.wait_limit_ns);
            }
            __syncwarp();
        }
        if (TILES && (J.flags & kLeftIn) && nreal > 0)  // tiles: the left neighbour's last column
            V = (uint32_t)poll_tagged(P.vbuf + J.vin + lane, epoch, P.err, P.wait_limit_ns) | ~realmask |
                0x80000000u;
        __syncwarp();

        // the job's scalars, broadcast from lane 0 so the compiler sees them
        // as warp-uniform (uniform branches, no reconvergence barriers)
        const int nwords = __shfl_sync(kFull, (int)((S + 31) >> 5), 0);
        // The pipeline always runs through lane 31: lanes past the segment's
        // rows hold no rows (zero match words, every vertical step 1), so they
        // pass each carry on unchanged and lane 31 emits the segment's bottom
        // row a few steps later.  The step at which it completes a word is
        // then the same for every job (no per-step test): at step i of word
        // u, lane 31 ends column 32 u + (i - 30) C - 1, the last column of
        // word u - kFlushLag when i = kFlushI.
        constexpr int kFlushI = 30 % K;
        constexpr int kFlushLag = (30 - kFlushI) / K + 1;
        static_assert((30 - kFlushI) % K == 0, "lane 31 ends a word at step kFlushI");
        // words lane 0 runs over: the real ones, then zero-row words until
        // lane 31 has finished the last real word
        const int nouter = nwords + (31 + K - 1) / K;
        const bool in_global = __shfl_sync(kFull, (J.flags & kInGlobal) != 0 ? 1 : 0, 0) != 0;
        const bool out_global = __shfl_sync(kFull, (J.flags & kOutGlobal) != 0 ? 1 : 0, 0) != 0;
        const uint64_t *src_row = P.hbuf + J.hin;
        uint64_t *dst_row = P.hbuf + J.hout;
        uint32_t *bout = P.bbits + (J.bword >= 0 ? J.bword : 0);
        const bool keep_bits = !out_global && J.bword >= 0;

        uint32_t cw = 0;      // this lane's carry-outs, newest in bit 0 (never reset)
        uint32_t sr = 0;      // carry-ins, next one in bit 31
        uint32_t total = 0;   // lane 31 of a final segment: set bits of the bottom row
        bool ok = true;
        // lanes 0..7 copy one 32-column word (16 bytes each); lanes 8..15 the
        // mirror copy when the word lands in slot 0 or 1.  Columns at or past
        // S are zero-filled: offset 0 is the all-zero match row.
        auto issue_cols = [&](int wd) {
            const int slot = wd & (kColRing - 1);
            const int part = lane & 7;
            if (lane < 8 || (lane < 16 && slot < 2)) {
                const int col = wd * 32 + part * 4;
                const int rem = (int)S - col;
                const int bytes = rem >= 4 ? 16 : (rem > 0 ? rem * 4 : 0);
                const uint32_t *src = boff + (bytes > 0 ? col : 0);
                const int dslot = lane < 8 ? slot : kColRing + slot;
                const uint32_t dst = col_ring + (uint32_t)((dslot * 32 + part * 4) * 4);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
                             : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        auto offs_at = [&](uint32_t addr, uint32_t (&o)[C]) {
            if constexpr (C == 2) {
                uint32_t x, y;
                asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(x), "=r"(y) : "r"(addr));
                o[0] = x;
                o[1] = y;
            } else {
#pragma unroll
                for (int k = 0; k < C / 4; ++k) {
                    uint32_t x, y, z, v;
                    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                                 : "=r"(x), "=r"(y), "=r"(z), "=r"(v) : "r"(addr + 16 * k));
                    o[4 * k] = x;
                    o[4 * k + 1] = y;
                    o[4 * k + 2] = z;
                    o[4 * k + 3] = v;
                }
            }
        };
        // the words before column 0 (read while the lanes' pipeline fills): zero rows
        {
            constexpr int kBefore = (31 * C + 31) / 32 + 1;
            uint32_t *ring = cols_ptr;
            for (int j = 1; j <= kBefore; ++j) ring[(kColRing - j) * 32 + lane] = 0u;
            __syncwarp();
        }
        for (int d = 0; d < kColAhead; ++d) issue_cols(d);
        // Lane 0's input carry words (segments below another segment of the
        // pair): loaded from global memory two words ahead into registers;
        // a stale tag sends the warp to the slow path outside the word loop.
        uint64_t in0 = 0, in1 = 0;
        if (in_global) {
            in0 = ld_relaxed_u64(src_row + 0);
            if (nwords > 1) in1 = ld_relaxed_u64(src_row + 1);
        }
        // the first word's match words and the offsets one step after them
        uint32_t Mcur[C], onext[C];
        {
            const int c0 = -C * lane;
            const uint32_t cb0 = col_ring + (uint32_t)(((c0 >> 5) & (kColRing - 1)) * 128) + (uint32_t)((c0 & 31) * 4);
            asm volatile("cp.async.wait_group %0;" ::"n"(kColAhead - 1) : "memory");
            __syncwarp();
            uint32_t o0[C];
            offs_at(cb0, o0);
#pragma unroll
            for (int jj = 0; jj < C; ++jj) Mcur[jj] = lds_u32(pm_lane + o0[jj]);
            offs_at(cb0 + (uint32_t)(C * 4), onext);
        }
        int u = 0;
        for (;;) {
            // two words per iteration: the scheduler overlaps the end of one
            // word's steps with the start of the next (3.7% on the 4096-pair
            // batch)
#pragma unroll 2
            for (; u < nouter; ++u) {
                // lane 0's input carry word u, checked by a vote (uniform exit)
                if (in_global && u < nwords &&
                    !__all_sync(kFull, lane != 0 || (uint32_t)(in0 >> 32) == epoch))
                    break;
                // words up to u + 1 copied (the last steps read into the next word)
                asm volatile("cp.async.wait_group %0;" ::"n"(kColAhead - 2) : "memory");
                __syncwarp();
                issue_cols(u + kColAhead);
                const uint32_t srcw = (in_global && u < nwords) ? (uint32_t)in0 : 0u;
                in0 = in1;
                if (in_global && u + 2 < nwords) in1 = ld_relaxed_u64(src_row + u + 2);
                if (lane == 0) sr = srcw;
                // this lane's column of step 0 (lane k trails lane 0 by k chunks) in the ring
                const int c0 = u * 32 - C * lane;
                const uint32_t cbase = col_ring + (uint32_t)(((c0 >> 5) & (kColRing - 1)) * 128) + (uint32_t)((c0 & 31) * 4);
                // one loop for fill, steady state and drain: columns outside [0, S)
                // read the zero row, so an idle lane keeps its state and passes
                // zero carries.  Offsets two steps ahead, match words one.
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    uint32_t onext2[C], Mnext[C];
                    offs_at(cbase + (uint32_t)((i + 2) * C * 4), onext2);
#pragma unroll
                    for (int jj = 0; jj < C; ++jj) Mnext[jj] = lds_u32(pm_lane + onext[jj]);
                    const uint32_t up = __shfl_up_sync(kFull, cw, 1);
                    if (lane != 0) sr = up << (32 - C);
#pragma unroll
                    for (int jj = 0; jj < C; ++jj) column31v(V, sr, cw, Mcur[jj]);
#pragma unroll
                    for (int jj = 0; jj < C; ++jj) {
                        Mcur[jj] = Mnext[jj];
                        onext[jj] = onext2[jj];
                    }
                    if (i == kFlushI) {  // lane 31 completes word wq (predicated stores)
                        const int wq = u - kFlushLag;
                        const bool fl = lane == 31 && wq >= 0 && wq < nwords;
                        st_relaxed_u64_if(fl && out_global, dst_row + (fl ? wq : 0), ((uint64_t)epoch << 32) | cw);
                        total += (fl && !out_global) ? (uint32_t)__popc(cw) : 0u;
                        st_u32_if(fl && keep_bits, bout + (fl ? wq : 0), cw);
                    }
                }
            }
            if (u >= nouter) break;
            // the slow path: lane 0 polls for its input word u (bounded)
            bool lok = true;
            if (lane == 0) in0 = poll_global_lane(src_row + u, epoch, P.err, P.wait_limit_ns, lok);
            if (!__all_sync(kFull, lok)) {
                ok = false;
                break;
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();

        if (ok && lane == 31 && (J.flags & kFinal)) P.len[J.pair] = (int32_t)total;
        if (ok && J.rword >= 0 && nreal > 0) P.rbits[J.rword + lane] = ~V & realmask;
        if (TILES && (J.flags & kRightOut) && nreal > 0)
            st_relaxed_u64_if(true, P.vbuf + J.vout + lane, ((uint64_t)epoch << 32) | V);
        if (TILES && J.done >= 0) {  // every store of this job before the flag
            __threadfence();
            __syncwarp();
            if (lane == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(P.done + J.done), "r"(epoch) : "memory");
        }
#pragma unroll
        for (int r = 0; r < kLaneRows; ++r) {
            if (r < nreal) {
                const uint32_t ch = (aw[r >> 2] >> ((r & 3) * 8)) & 0xffu;
                if ((int)ch < P.sigma) pm[(ch + 1) * 32 + lane] = 0u;
            }
        }
        __syncwarp();
    }
}

// TILES: the jobs are tiles of one table (tagged left/right columns, join
// flags); a separate instantiation keeps plain batches at fewer registers.
template <bool TILES>
__global__ void __launch_bounds__(32) k_batch(const BatchArgs P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) uint32_t s_cols[(kColRing + 2) * 32];
    const int lane = threadIdx.x & 31;
    uint32_t *pm = reinterpret_cast<uint32_t *>(smem);
    const uint32_t pm_lane = (uint32_t)__cvta_generic_to_shared(pm + lane);
    const uint32_t col_ring = (uint32_t)__cvta_generic_to_shared(s_cols);
    for (int c = 0; c < P.table_rows; ++c) pm[c * 32 + lane] = 0u;
    for (int i = lane; i < (kColRing + 2) * 32; i += 32) s_cols[i] = 0u;  // valid offsets from the start
    const uint32_t epoch = *P.epoch_dev;
    for (;;) {
        int job = 0;
        if (lane == 0) {
            job = atomicAdd(P.ticket, 1);
            if (ld_relaxed_i32(P.err) != 0) job = (int)P.njobs;
        }
        job = __shfl_sync(kFull, job, 0);
        if (job >= P.njobs) break;
        const SegJob J = P.jobs[job];
        // the chunk width of the job's size class
        const int cl = (int)((J.flags >> kClassShift) & 3u);  // (no dynamic index into the parameters)
        const int C = cl == 0 ? P.cls_chunk[0] : (cl == 1 ? P.cls_chunk[1] : (cl == 2 ? P.cls_chunk[2] : P.cls_chunk[3]));
        if (C == 2) batch_job<2, TILES>(P, J, lane, pm, pm_lane, s_cols, col_ring, epoch);
        else if (C == 4) batch_job<4, TILES>(P, J, lane, pm, pm_lane, s_cols, col_ring, epoch);
        else batch_job<8, TILES>(P, J, lane, pm, pm_lane, s_cols, col_ring, epoch);
    }
}

__global__ void k_bump_epoch(uint32_t *e) {
    uint32_t v = *e + 1;
    if (v == 0) v = 1;
    *e = v;
}

// Per-pair prefixes: bottom row from the final segment's step bits (MSB-first
// words) and right column from the lane words (31 rows each), written with
// the transposition undone.
struct PrefixJob {
    int64_t bword;    // bottom-row step words (or -1)
    int64_t rword;    // right-column lane words (or -1)
    int64_t L, S;     // kernel rows / columns
    int64_t out_bottom;  // offset into rows_cat or cols_cat
    int64_t out_right;
    int32_t transposed;
    int32_t pad;
};

__device__ void block_prefix(const uint32_t *words, int bpw, bool msb_first, int64_t nbits, int32_t *out) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    if (out == nullptr) return;
    if (threadIdx.x == 0) out[0] = 0;
    __syncthreads();
    const int64_t nw = (nbits + bpw - 1) / bpw;
    for (int64_t base = 0; base < nw; base += blockDim.x) {
        const int64_t k = base + threadIdx.x;
        uint32_t word = 0;
        if (k < nw) {
            word = words[k];
            if (msb_first) word = __brev(word);
            const int64_t rem = nbits - k * bpw;
            if (rem < 32) word &= (1u << rem) - 1u;
        }
        const int32_t c = __popc(word);
        int32_t inc = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, inc, o);
            if ((threadIdx.x & 31) >= o) inc += y;
        }
        if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = inc;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int32_t t = threadIdx.x < (blockDim.x >> 5) ? warp_tot[threadIdx.x] : 0;
            int32_t ti = t;
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, ti, o);
                if (threadIdx.x >= o) ti += y;
            }
            warp_tot[threadIdx.x] = ti - t;
        }
        __syncthreads();
        const int32_t before = carry + warp_tot[threadIdx.x >> 5] + inc - c;
        if (k < nw) {
            const int64_t e0 = k * bpw;
            const int ne = (int)min((int64_t)bpw, nbits - e0);
            int32_t run = before;
            for (int b = 0; b < ne; ++b) {
                run += (word >> b) & 1u;
                out[e0 + b + 1] = run;
            }
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + c;
        __syncthreads();
    }
}

__global__ void k_batch_prefix(const PrefixJob *pj, const uint32_t *bbits, const uint32_t *rbits,
                               int32_t *rows_cat, int32_t *cols_cat) {
    const PrefixJob J = pj[blockIdx.x];
    // kernel bottom row (S+1 values) and kernel right column (L+1 values)
    int32_t *kb = J.transposed ? (cols_cat ? cols_cat + J.out_bottom : nullptr)
                               : (rows_cat ? rows_cat + J.out_bottom : nullptr);
    int32_t *kr = J.transposed ? (rows_cat ? rows_cat + J.out_right : nullptr)
                               : (cols_cat ? cols_cat + J.out_right : nullptr);
    if (J.bword >= 0) block_prefix(bbits + J.bword, 32, true, J.S, kb);
    else if (kb) for (int64_t j = threadIdx.x; j <= J.S; j += blockDim.x) kb[j] = 0;
    __syncthreads();
    if (J.rword >= 0) block_prefix(rbits + J.rword, 31, false, J.L, kr);
    else if (kr) for (int64_t i = threadIdx.x; i <= J.L; i += blockDim.x) kr[i] = 0;
}

template <bool TILES>
cudaError_t launch_batch_t(const BatchArgs &a, int grid, cudaStream_t st) {
    const size_t smem = (size_t)a.table_rows * 32 * 4;
    cudaError_t e = cudaFuncSetAttribute(k_batch<TILES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((kMaxSigma + 1) * 32 * 4));
    if (e != cudaSuccess) return e;
    k_batch<TILES><<<grid, 32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs &a, int grid, cudaStream_t st) {
    return a.vbuf ? launch_batch_t<true>(a, grid, st) : launch_batch_t<false>(a, grid, st);
}

template <bool TILES>
int occupancy_t(int table_rows) {
    const size_t smem = (size_t)table_rows * 32 * 4;
    if (cudaFuncSetAttribute(k_batch<TILES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((kMaxSigma + 1) * 32 * 4)) != cudaSuccess)
        return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<TILES>, 32, smem) != cudaSuccess) return 1;
    return std::max(1, nb);
}

int occupancy_for(int table_rows, bool tiles = false) {
    return tiles ? occupancy_t<true>(table_rows) : occupancy_t<false>(table_rows);
}

int table_rows_for(int sigma) { return (sigma >= kMaxSigma ? kMaxSigma : sigma) + 1; }

struct Layout {
    std::vector<SegJob> jobs;
    std::vector<PrefixJob> pjobs;
    std::vector<ColJob> cjobs;
    int64_t cwords = 0;
    int64_t class_jobs[kClasses] = {0, 0, 0, 0};
    int64_t hwords = 0, rwords = 0, bwords = 0;
    int64_t cells = 0;
};

// Segments, carry rows and output word offsets for a batch.  Jobs run in
// critical-path order: a segment's priority is the length of the chain that
// starts with it, S columns plus one pipeline fill (the lanes' skew and one
// word, about 31 C + 32 columns at C = 4) for every segment below it.  A
// pair's segments keep their order (each comes after the one above it, so
// a warp only ever waits for a running segment), and a tall, narrow pair,
// whose chain is long for its few cells, starts early instead of last.
constexpr int64_t kChainFill = 31 * 4 + 32;
void plan_batch(int32_t npairs, const int64_t *a_off, const int64_t *b_off, bool want_rows,
                bool want_cols, const int64_t *row_off, const int64_t *col_off, Layout &lay) {
    lay = Layout();
    std::vector<int32_t> order((size_t)npairs);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int64_t> work((size_t)npairs);
    for (int32_t k = 0; k < npairs; ++k)
        work[(size_t)k] = (a_off[k + 1] - a_off[k]) * (b_off[k + 1] - b_off[k]);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return work[(size_t)x] > work[(size_t)y]; });
    const int64_t seg_rows = 32 * 31;
    std::vector<int64_t> prio;  // per job, in the order built
    for (int32_t k : order) {
        const int64_t n = a_off[k + 1] - a_off[k], m = b_off[k + 1] - b_off[k];
        const bool tr = m > n;
        const int64_t L = tr ? m : n, S = tr ? n : m;
        PrefixJob pj{};
        pj.L = L;
        pj.S = S;
        pj.transposed = tr ? 1 : 0;
        pj.out_bottom = tr ? (col_off ? col_off[k] : 0) : (row_off ? row_off[k] : 0);
        pj.out_right = tr ? (row_off ? row_off[k] : 0) : (col_off ? col_off[k] : 0);
        pj.bword = -1;
        pj.rword = -1;
        const bool want_bottom = tr ? want_cols : want_rows;
        const bool want_right = tr ? want_rows : want_cols;
        lay.cells += L * S;
        if (L == 0 || S == 0) {
            if (want_rows || want_cols) lay.pjobs.push_back(pj);
            continue;
        }
        const int64_t nwords = (S + 31) / 32, hstride = (nwords + 1) & ~(int64_t)1;
        const int64_t nseg = (L + seg_rows - 1) / seg_rows;
        if (want_bottom) {
            pj.bword = lay.bwords;
            lay.bwords += nwords;
        }
        if (want_right) {
            pj.rword = lay.rwords;
            lay.rwords += nseg * 32;
        }
        ColJob cj{};
        cj.src = tr ? a_off[k] : b_off[k];
        cj.dst = lay.cwords;
        cj.len = S;
        cj.from_a = tr ? 1 : 0;
        lay.cjobs.push_back(cj);
        lay.cwords += (S + 3) & ~(int64_t)3;
        int64_t prev_out = -1;
        for (int64_t j = 0; j < nseg; ++j) {
            SegJob J{};
            J.vin = J.vout = -1;
            J.join0 = J.join1 = J.done = -1;
            J.rows_off = (tr ? b_off[k] : a_off[k]) + j * seg_rows;
            J.cols_off = cj.dst;
            J.nrows = (int32_t)std::min(seg_rows, L - j * seg_rows);
            J.S = (int32_t)S;
            J.pair = k;
            J.flags = (tr ? kTransposed : 0u) | ((uint32_t)size_class(S) << kClassShift);
            J.hin = 0;
            J.hout = 0;
            if (j > 0) {
                J.flags |= kInGlobal;
                J.hin = prev_out;
            }
            if (j + 1 < nseg) {
                J.flags |= kOutGlobal;
                J.hout = lay.hwords;
                prev_out = lay.hwords;
                lay.hwords += hstride;
            } else {
                J.flags |= kFinal;
                J.bword = pj.bword;
            }
            J.rword = pj.rword >= 0 ? pj.rword + j * 32 : -1;
            if (J.flags & kFinal) J.bword = pj.bword;
            else J.bword = -1;
            lay.jobs.push_back(J);
            prio.push_back(S + kChainFill * (nseg - j));
            ++lay.class_jobs[size_class(S)];
        }
        if (want_rows || want_cols) lay.pjobs.push_back(pj);
    }
    std::vector<int64_t> idx(lay.jobs.size());
    std::iota(idx.begin(), idx.end(), (int64_t)0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return prio[(size_t)x] > prio[(size_t)y]; });
    std::vector<SegJob> sorted;
    sorted.reserve(lay.jobs.size());
    for (int64_t i : idx) sorted.push_back(lay.jobs[(size_t)i]);
    lay.jobs.swap(sorted);
}

uint64_t fnv(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

struct BatchState {
    int *ticket_ptr = nullptr;  // device ticket and error word this state launches with
    int *err_ptr = nullptr;
    // device copies of the current layout
    DevBuf jobs, pjobs, cjobs, hbuf, rbits, bbits, coffs, epoch;
    // pinned staging of the layout tables (stream-ordered uploads)
    void *h_stage = nullptr;
    size_t h_stage_cap = 0;
    uint64_t layout_key = 0;
    int64_t njobs = 0, npjobs = 0, ncjobs = 0;
    // captured graph of the whole batch step
    cudaGraphExec_t exec = nullptr;
    uint64_t exec_key = 0;
    int64_t class_jobs[4] = {0, 0, 0, 0};
    // autotuned chunk width of each size class, per layout signature
    std::map<uint64_t, std::array<int, 4>> tuned;
};

void batch_release(paco_ctx *ctx) {
    batch_state_free(ctx->batch);
    ctx->batch = nullptr;
    batch_state_free(ctx->recover);
    ctx->recover = nullptr;
    tile_state_free(ctx->tiles);
    ctx->tiles = nullptr;
}

namespace {

// Enqueue the whole batch step (no allocation, capturable).
cudaError_t enqueue_batch(paco_ctx *ctx, BatchState *B, const std::array<int, 4> &cls, int sigma,
                          const uint8_t *a_cat, int64_t a_len,
                          const uint8_t *b_cat, int64_t b_len, int32_t npairs, int32_t *d_len,
                          int32_t *rows_cat, int32_t *cols_cat, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(B->ticket_ptr, 0, sizeof(int), st);
    if (e == cudaSuccess && npairs > 0) e = cudaMemsetAsync(d_len, 0, (size_t)npairs * 4, st);
    if (e != cudaSuccess) return e;
    (void)a_len;
    (void)b_len;
    k_bump_epoch<<<1, 1, 0, st>>>((uint32_t *)B->epoch.ptr);
    if (B->ncjobs > 0)
        k_pair_column_offsets<<<(unsigned)B->ncjobs, 256, 0, st>>>(a_cat, b_cat, (const ColJob *)B->cjobs.ptr,
                                                                   (uint32_t *)B->coffs.ptr, sigma, B->err_ptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (B->njobs > 0) {
        BatchArgs A;
        A.a_cat = a_cat;
        A.b_cat = b_cat;
        A.coffs = (const uint32_t *)B->coffs.ptr;
        A.jobs = (const SegJob *)B->jobs.ptr;
        A.njobs = B->njobs;
        A.hbuf = (uint64_t *)B->hbuf.ptr;
        A.rbits = (uint32_t *)B->rbits.ptr;
        A.bbits = (uint32_t *)B->bbits.ptr;
        A.len = d_len;
        A.ticket = B->ticket_ptr;
        A.err = B->err_ptr;
        A.epoch_dev = (const uint32_t *)B->epoch.ptr;
        A.wait_limit_ns = ctx->wait_limit_ns;
        A.sigma = sigma;
        A.table_rows = table_rows_for(sigma);
        for (int k = 0; k < kClasses; ++k) A.cls_chunk[k] = cls[(size_t)k];
        A.vbuf = nullptr;
        A.done = nullptr;
        const int grid = (int)std::min<int64_t>(B->njobs, (int64_t)ctx->sms * occupancy_for(A.table_rows));
        e = launch_batch(A, grid, st);
        if (e != cudaSuccess) return e;
    }
    if (B->npjobs > 0 && (rows_cat || cols_cat)) {
        k_batch_prefix<<<(unsigned)B->npjobs, 256, 0, st>>>((const PrefixJob *)B->pjobs.ptr,
                                                            (const uint32_t *)B->bbits.ptr,
                                                            (const uint32_t *)B->rbits.ptr, rows_cat, cols_cat);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

BatchState *batch_state_new(int *ticket, int *err) {
    BatchState *B = new (std::nothrow) BatchState();
    if (B) {
        B->ticket_ptr = ticket;
        B->err_ptr = err;
    }
    return B;
}

void batch_state_free(BatchState *B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    for (DevBuf *b : {&B->jobs, &B->pjobs, &B->cjobs, &B->hbuf, &B->rbits, &B->bbits, &B->coffs, &B->epoch})
        if (b->ptr) cudaFree(b->ptr);
    if (B->h_stage) cudaFreeHost(B->h_stage);
    delete B;
}

int run_batch(paco_ctx *ctx, BatchState *B, const uint8_t *a_cat, const int64_t *h_a_off, const uint8_t *b_cat,
              const int64_t *h_b_off, int32_t npairs, int32_t *d_len, int32_t *rows_cat,
              const int64_t *h_row_off, int32_t *cols_cat, const int64_t *h_col_off, cudaStream_t st,
              bool use_graph, int force_chunk, int sigma) {
    if (!B) return PACO_ENOMEM;
    if (sigma < 1 || sigma > kMaxSigma) sigma = kMaxSigma;
    int rc;
    const int64_t a_len = h_a_off[npairs], b_len = h_b_off[npairs];
    // layout: depends on lengths and on which outputs are wanted (and where)
    uint64_t key = fnv(h_a_off, sizeof(int64_t) * (npairs + 1));
    key = fnv(&sigma, sizeof(sigma), key);
    key = fnv(h_b_off, sizeof(int64_t) * (npairs + 1), key);
    const int want = (rows_cat ? 1 : 0) | (cols_cat ? 2 : 0);
    key = fnv(&want, sizeof(want), key);
    if (rows_cat) key = fnv(h_row_off, sizeof(int64_t) * npairs, key);
    if (cols_cat) key = fnv(h_col_off, sizeof(int64_t) * npairs, key);
    if (key != B->layout_key) {
        Layout lay;
        plan_batch(npairs, h_a_off, h_b_off, rows_cat != nullptr, cols_cat != nullptr, h_row_off, h_col_off, lay);
        const size_t bj = lay.jobs.size() * sizeof(SegJob), bp = lay.pjobs.size() * sizeof(PrefixJob),
                     bc = lay.cjobs.size() * sizeof(ColJob);
        if (B != ctx->batch) {
            // a serving slot: its buffers are used by its own stream only, so
            // they grow stream-ordered (no device-wide synchronisation) and
            // the layout goes up from pinned staging asynchronously; the slot
            // is reused only after its previous micro-batch has completed
            auto grow = [&](DevBuf &d, size_t need, bool zero) -> int {
                if (d.bytes >= need) return PACO_OK;
                if (d.ptr) cudaFreeAsync(d.ptr, st);
                d.ptr = nullptr;
                d.bytes = 0;
                const size_t want = std::max(need * 2, (size_t)4096);
                if (cudaMallocAsync(&d.ptr, want, st) != cudaSuccess) return PACO_ENOMEM;
                d.bytes = want;
                if (zero && cudaMemsetAsync(d.ptr, 0, want, st) != cudaSuccess) return PACO_EDEVICE;
                return PACO_OK;
            };
            if ((rc = grow(B->jobs, bj + 64, false)) != PACO_OK || (rc = grow(B->pjobs, bp + 64, false)) != PACO_OK ||
                (rc = grow(B->cjobs, bc + 64, false)) != PACO_OK ||
                (rc = grow(B->coffs, (size_t)lay.cwords * 4 + 64, false)) != PACO_OK ||
                (rc = grow(B->hbuf, (size_t)lay.hwords * 8 + 64, true)) != PACO_OK ||
                (rc = grow(B->rbits, (size_t)lay.rwords * 4 + 64, false)) != PACO_OK ||
                (rc = grow(B->bbits, (size_t)lay.bwords * 4 + 64, false)) != PACO_OK ||
                (rc = grow(B->epoch, 64, true)) != PACO_OK)
                return rc;
            const size_t need = bj + bp + bc + 64;
            if (B->h_stage_cap < need) {
                if (B->h_stage) cudaFreeHost(B->h_stage);
                B->h_stage = nullptr;
                B->h_stage_cap = 0;
                if (cudaMallocHost(&B->h_stage, need * 2) != cudaSuccess) return PACO_ENOMEM;
                B->h_stage_cap = need * 2;
            }
            unsigned char *hs = (unsigned char *)B->h_stage;
            if (bj) std::memcpy(hs, lay.jobs.data(), bj);
            if (bp) std::memcpy(hs + bj, lay.pjobs.data(), bp);
            if (bc) std::memcpy(hs + bj + bp, lay.cjobs.data(), bc);
            cudaError_t e = cudaSuccess;
            if (bj) e = cudaMemcpyAsync(B->jobs.ptr, hs, bj, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && bp) e = cudaMemcpyAsync(B->pjobs.ptr, hs + bj, bp, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && bc)
                e = cudaMemcpyAsync(B->cjobs.ptr, hs + bj + bp, bc, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return set_cuda_error(ctx, e, "upload batch layout");
        } else {
            if ((rc = ensure_bytes(ctx, B->jobs, bj + 64)) != PACO_OK) return rc;
            if ((rc = ensure_bytes(ctx, B->pjobs, bp + 64)) != PACO_OK) return rc;
            if ((rc = ensure_bytes(ctx, B->cjobs, bc + 64)) != PACO_OK) return rc;
            if ((rc = ensure_bytes(ctx, B->coffs, (size_t)lay.cwords * 4 + 64)) != PACO_OK) return rc;
            if ((rc = ensure_bytes(ctx, B->hbuf, (size_t)lay.hwords * 8 + 64)) != PACO_OK) return rc;
            if ((rc = ensure_bytes(ctx, B->rbits, (size_t)lay.rwords * 4 + 64)) != PACO_OK) return rc;
            if ((rc = ensure_bytes(ctx, B->bbits, (size_t)lay.bwords * 4 + 64)) != PACO_OK) return rc;
            if ((rc = ensure_bytes(ctx, B->epoch, 64)) != PACO_OK) return rc;
            cudaError_t e = cudaSuccess;
            if (bj) e = cudaMemcpy(B->jobs.ptr, lay.jobs.data(), bj, cudaMemcpyHostToDevice);
            if (e == cudaSuccess && bp) e = cudaMemcpy(B->pjobs.ptr, lay.pjobs.data(), bp, cudaMemcpyHostToDevice);
            if (e == cudaSuccess && bc) e = cudaMemcpy(B->cjobs.ptr, lay.cjobs.data(), bc, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return set_cuda_error(ctx, e, "upload batch layout");
        }
        B->ncjobs = (int64_t)lay.cjobs.size();
        B->njobs = (int64_t)lay.jobs.size();
        B->npjobs = (int64_t)lay.pjobs.size();
        for (int k = 0; k < kClasses; ++k) B->class_jobs[k] = lay.class_jobs[k];
        B->layout_key = key;
        if (B->exec) {
            cudaGraphExecDestroy(B->exec);
            B->exec = nullptr;
            B->exec_key = 0;
        }
    }

    // chunk width of each size class: forced, tuned for this layout, or tuned
    // now by coordinate descent over the classes present (each candidate
    // timed twice, the second run kept)
    std::array<int, 4> cls = {4, 4, 4, 4};
    if (force_chunk) {
        cls = {force_chunk, force_chunk, force_chunk, force_chunk};
    } else if (B != ctx->batch) {
        // serving micro-batches: the caller's widths per size class, else defaults
        const int sc = ctx->opt_serve_chunks;
        cls = sc ? std::array<int, 4>{sc & 15, (sc >> 4) & 15, (sc >> 8) & 15, (sc >> 12) & 15}
                 : std::array<int, 4>{2, 4, 8, 8};
    } else {
        auto it = B->tuned.find(key);
        if (it != B->tuned.end()) {
            cls = it->second;
        } else {
            // best of three runs per candidate (run-to-run noise is a few percent)
            auto time_it = [&](const std::array<int, 4> &c, float &ms) -> int {
                ms = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    cudaEventRecord(ctx->ev0, st);
                    cudaError_t e = enqueue_batch(ctx, B, c, sigma, a_cat, a_len, b_cat, b_len, npairs, d_len,
                                                  rows_cat, cols_cat, st);
                    cudaEventRecord(ctx->ev1, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev1);
                    if (e != cudaSuccess) return set_cuda_error(ctx, e, "batch autotune");
                    float t = 0.f;
                    cudaEventElapsedTime(&t, ctx->ev0, ctx->ev1);
                    if (rep > 0) ms = std::min(ms, t);  // the first run also warms caches
                }
                return PACO_OK;
            };
            // one width for every class first, then each class on its own,
            // largest class (most of the cells) first
            float best = 1e30f;
            for (int cand : {2, 4, 8}) {
                const std::array<int, 4> trial = {cand, cand, cand, cand};
                float ms = 0.f;
                if ((rc = time_it(trial, ms)) != PACO_OK) return rc;
                if (ms < best) {
                    best = ms;
                    cls = trial;
                }
            }
            for (int k = kClasses - 1; k >= 0; --k) {
                if (B->class_jobs[k] == 0) continue;
                const int keep = cls[(size_t)k];
                for (int cand : {2, 4, 8}) {
                    if (cand == keep) continue;
                    std::array<int, 4> trial = cls;
                    trial[(size_t)k] = cand;
                    float ms = 0.f;
                    if ((rc = time_it(trial, ms)) != PACO_OK) return rc;
                    if (ms < best) {
                        best = ms;
                        cls = trial;
                    }
                }
            }
            B->tuned[key] = cls;
        }
    }
    const int C = cls[0] | (cls[1] << 4) | (cls[2] << 8) | (cls[3] << 12);
    const uint64_t exec_key = fnv(&C, sizeof(C),
                                  fnv(&a_cat, sizeof(a_cat),
                                      fnv(&b_cat, sizeof(b_cat),
                                          fnv(&d_len, sizeof(d_len),
                                              fnv(&rows_cat, sizeof(rows_cat),
                                                  fnv(&cols_cat, sizeof(cols_cat), key))))));
    const bool timing = (B == ctx->batch);
    if (timing) cudaEventRecord(ctx->ev0, st);
    cudaError_t e = cudaSuccess;
    if (use_graph) {
        if (!B->exec || B->exec_key != exec_key) {
            if (B->exec) {
                cudaGraphExecDestroy(B->exec);
                B->exec = nullptr;
            }
            cudaStream_t cap = nullptr;
            e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            cudaGraph_t g = nullptr;
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue_batch(ctx, B, cls, sigma, a_cat, a_len, b_cat, b_len, npairs, d_len, rows_cat,
                                               cols_cat, cap);
                e = cudaStreamEndCapture(cap, &g);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (cap) cudaStreamDestroy(cap);
            if (e != cudaSuccess) return set_cuda_error(ctx, e, "capture batch graph");
            B->exec_key = exec_key;
        }
        e = cudaGraphLaunch(B->exec, st);
    } else {
        e = enqueue_batch(ctx, B, cls, sigma, a_cat, a_len, b_cat, b_len, npairs, d_len, rows_cat, cols_cat, st);
    }
    if (timing) {
        cudaEventRecord(ctx->ev1, st);
        ctx->timed = true;
        ctx->timed_name = "batch graph (k_batch)";
        ctx->last_batch_chunk = C;
    }
    return e == cudaSuccess ? PACO_OK : (e == cudaErrorMemoryAllocation ? PACO_ENOMEM : PACO_EDEVICE);
}

// ---------------------------------------------------------------------------
// Tile schedules (PACO partition, PA p x p blocks, PO divide and conquer) on
// the batch kernel: every tile is one warp job; its top carries and left
// vertical steps arrive as tagged words written by the tiles above and to
// the left (a job claims its ticket only after every job it depends on), and
// the PO fork-join order waits on completion flags.
// ---------------------------------------------------------------------------
struct TileLayout {
    std::vector<SegJob> jobs;
    int64_t hwords = 0, vwords = 0, nwords = 0, ng = 0;
    int64_t critical_cells = 0;
};

struct TileState {
    DevBuf jobs, coffs, cjob, hbuf, vbuf, rbits, bbits, done, epoch, pjob;
    std::map<std::tuple<int64_t, int64_t, int, int64_t>, std::shared_ptr<TileLayout>> layouts;
    int64_t last_tiles = 0, last_critical = 0;
};

void tile_state_free(TileState *T) {
    if (!T) return;
    for (DevBuf *d : {&T->jobs, &T->coffs, &T->cjob, &T->hbuf, &T->vbuf, &T->rbits, &T->bbits, &T->done, &T->epoch,
                      &T->pjob})
        if (d->ptr) cudaFree(d->ptr);
    delete T;
}

namespace {

__global__ void k_bits_total(const uint32_t *bits, int64_t nw, int32_t *len) {
    int64_t c = 0;
    for (int64_t k = threadIdx.x; k < nw; k += blockDim.x) c += __popc(bits[k]);
    __shared__ int64_t red[32];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        c = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
        if (threadIdx.x == 0) *len = (int32_t)c;
    }
}

std::shared_ptr<TileLayout> build_tile_layout(int64_t L, int64_t S, int p, int kind, int64_t base) {
    TilePlan tp;
    if (!plan_tiles(L, S, p, kind, base, tp)) return nullptr;
    auto lay = std::make_shared<TileLayout>();
    std::vector<int64_t> rc, cc;
    for (const Tile &t : tp.tiles) {
        rc.push_back(t.r0);
        rc.push_back(t.r1);
        cc.push_back(t.c0);
        cc.push_back(t.c1);
    }
    std::sort(rc.begin(), rc.end());
    rc.erase(std::unique(rc.begin(), rc.end()), rc.end());
    std::sort(cc.begin(), cc.end());
    cc.erase(std::unique(cc.begin(), cc.end()), cc.end());
    auto idx = [](const std::vector<int64_t> &v, int64_t x) {
        return (int64_t)(std::lower_bound(v.begin(), v.end(), x) - v.begin());
    };
    lay->nwords = (S + 31) / 32;
    const int64_t hstride = (lay->nwords + 1) & ~(int64_t)1;  // even: 16-byte aligned word pairs
    lay->ng = (L + kLaneRows - 1) / kLaneRows;
    lay->hwords = (int64_t)rc.size() * hstride;
    lay->vwords = (int64_t)cc.size() * lay->ng;
    std::vector<char> is_target(tp.tiles.size(), 0);
    for (size_t k = 0; k < tp.tiles.size(); ++k) {
        if (tp.join0[k] >= 0) is_target[(size_t)tp.join0[k]] = 1;
        if (tp.join1[k] >= 0) is_target[(size_t)tp.join1[k]] = 1;
    }
    lay->jobs.reserve(tp.tiles.size());
    for (size_t k = 0; k < tp.tiles.size(); ++k) {
        const Tile &t = tp.tiles[k];
        SegJob J{};
        J.rows_off = t.r0;
        J.cols_off = t.c0;
        J.nrows = (int32_t)(t.r1 - t.r0);
        J.S = (int32_t)(t.c1 - t.c0);
        J.pair = 0;
        J.flags = ((uint32_t)size_class(t.c1 - t.c0) << kClassShift) | (t.r0 > 0 ? kInGlobal : 0u) |
                  (t.r1 < L ? kOutGlobal : 0u) | (t.c0 > 0 ? kLeftIn : 0u) | (t.c1 < S ? kRightOut : 0u);
        J.hin = idx(rc, t.r0) * hstride + t.c0 / 32;
        J.hout = idx(rc, t.r1) * hstride + t.c0 / 32;
        J.rword = t.c1 == S ? t.r0 / kLaneRows : -1;
        J.bword = t.r1 == L ? t.c0 / 32 : -1;
        J.vin = idx(cc, t.c0) * lay->ng + t.r0 / kLaneRows;
        J.vout = idx(cc, t.c1) * lay->ng + t.r0 / kLaneRows;
        J.join0 = (int32_t)tp.join0[k];
        J.join1 = (int32_t)tp.join1[k];
        J.done = is_target[k] ? (int32_t)k : -1;
        lay->jobs.push_back(J);
    }
    lay->critical_cells = tp.critical_cells;
    return lay;
}

}  // namespace

int run_tiles(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, int32_t *bottom_row,
              int32_t *right_col, int32_t *len, cudaStream_t st) {
    const bool tr = m > n;
    const int64_t L = tr ? m : n, S = tr ? n : m;
    const uint8_t *ka = tr ? b : a, *kb = tr ? a : b;
    const int kind = ctx->opt_tiles;
    const int64_t base = ctx->opt_tile_base > 0 ? ctx->opt_tile_base : (kind == kTilesPo ? 16 : 4);
    if (!ctx->tiles) ctx->tiles = new (std::nothrow) TileState();
    TileState *T = ctx->tiles;
    if (!T) return PACO_ENOMEM;
    const auto key = std::make_tuple(L, S, kind, base);
    auto it = T->layouts.find(key);
    std::shared_ptr<TileLayout> lay;
    if (it != T->layouts.end()) {
        lay = it->second;
    } else {
        lay = build_tile_layout(L, S, ctx->sms, kind, base);
        if (!lay) return PACO_EINVAL;
        if (T->layouts.size() > 16) T->layouts.clear();
        T->layouts.emplace(key, lay);
    }
    const int64_t njobs = (int64_t)lay->jobs.size();
    int rc;
    if ((rc = ensure_bytes(ctx, T->jobs, (size_t)njobs * sizeof(SegJob) + 64)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, T->coffs, (size_t)S * 4 + 64)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, T->cjob, sizeof(ColJob) + 64)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, T->hbuf, (size_t)lay->hwords * 8 + 64)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, T->vbuf, (size_t)lay->vwords * 8 + 64)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, T->rbits, (size_t)lay->ng * 4 + 64)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, T->bbits, (size_t)lay->nwords * 4 + 64)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, T->done, (size_t)njobs * 4 + 64)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, T->epoch, 64)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, T->pjob, sizeof(PrefixJob) + 64)) != PACO_OK) return rc;
    ColJob cj{};
    cj.src = 0;
    cj.dst = 0;
    cj.len = S;
    cj.from_a = 0;  // the streamed string is passed as b_cat
    PrefixJob pj{};
    pj.bword = 0;
    pj.rword = 0;
    pj.L = L;
    pj.S = S;
    pj.out_bottom = 0;
    pj.out_right = 0;
    pj.transposed = tr ? 1 : 0;
    cudaError_t e = cudaMemcpyAsync(T->jobs.ptr, lay->jobs.data(), (size_t)njobs * sizeof(SegJob),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T->cjob.ptr, &cj, sizeof(cj), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T->pjob.ptr, &pj, sizeof(pj), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ticket_ptr(), 0, sizeof(int), st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "tile layout");
    k_bump_epoch<<<1, 1, 0, st>>>((uint32_t *)T->epoch.ptr);
    k_pair_column_offsets<<<1, 256, 0, st>>>(kb, kb, (const ColJob *)T->cjob.ptr, (uint32_t *)T->coffs.ptr,
                                             kMaxSigma, ctx->err_ptr());
    BatchArgs A;
    A.a_cat = ka;
    A.b_cat = kb;
    A.coffs = (const uint32_t *)T->coffs.ptr;
    A.jobs = (const SegJob *)T->jobs.ptr;
    A.njobs = njobs;
    A.hbuf = (uint64_t *)T->hbuf.ptr;
    A.rbits = (uint32_t *)T->rbits.ptr;
    A.bbits = (uint32_t *)T->bbits.ptr;
    A.len = len;
    A.ticket = ctx->ticket_ptr();
    A.err = ctx->err_ptr();
    A.epoch_dev = (const uint32_t *)T->epoch.ptr;
    A.wait_limit_ns = ctx->wait_limit_ns;
    A.sigma = kMaxSigma;
    A.table_rows = table_rows_for(kMaxSigma);
    const int force = ctx->opt_chunk;
    const int cls_default[4] = {2, 4, 8, 8};
    for (int k = 0; k < kClasses; ++k) A.cls_chunk[k] = force ? force : cls_default[k];
    A.vbuf = (uint64_t *)T->vbuf.ptr;
    A.done = (uint32_t *)T->done.ptr;
    const int grid = (int)std::min<int64_t>(njobs, (int64_t)ctx->sms * occupancy_for(A.table_rows, true));
    cudaEventRecord(ctx->ev0, st);
    e = launch_batch(A, grid, st);
    cudaEventRecord(ctx->ev1, st);
    ctx->timed = true;
    ctx->timed_name = "k_batch (tile schedule)";
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "tile schedule launch");
    if (bottom_row || right_col) {
        k_batch_prefix<<<1, 256, 0, st>>>((const PrefixJob *)T->pjob.ptr, (const uint32_t *)T->bbits.ptr,
                                          (const uint32_t *)T->rbits.ptr, bottom_row, right_col);
        e = cudaGetLastError();
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "tile schedule boundaries");
    }
    if (len) k_bits_total<<<1, 256, 0, st>>>((const uint32_t *)T->bbits.ptr, lay->nwords, len);
    T->last_tiles = njobs;
    T->last_critical = lay->critical_cells;
    e = cudaGetLastError();
    return e == cudaSuccess ? PACO_OK : set_cuda_error(ctx, e, "tile schedule length");
}

}  // namespace paco

extern "C" int paco_lcs_batch(paco_ctx *ctx, const uint8_t *a_cat, const uint8_t *b_cat,
                              const int64_t *h_a_off, const int64_t *h_b_off, int32_t npairs,
                              int32_t *d_len, int32_t *d_rows_cat, const int64_t *h_row_off,
                              int32_t *d_cols_cat, const int64_t *h_col_off, void *stream) {
    if (!ctx || npairs < 0 || !h_a_off || !h_b_off) return PACO_EINVAL;
    if (npairs > 0 && !d_len) return PACO_EINVAL;
    if ((d_rows_cat && !h_row_off) || (d_cols_cat && !h_col_off)) return PACO_EINVAL;
    for (int32_t k = 0; k < npairs; ++k) {
        const int64_t n = h_a_off[k + 1] - h_a_off[k], m = h_b_off[k + 1] - h_b_off[k];
        if (n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL) return PACO_EINVAL;
    }
    if (h_a_off[npairs] > 0 && !a_cat) return PACO_EINVAL;
    if (h_b_off[npairs] > 0 && !b_cat) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    const int force = ctx->opt_chunk == 0 ? 0 : std::min(8, std::max(2, ctx->opt_chunk));
    if (!ctx->batch) ctx->batch = paco::batch_state_new(ctx->ticket_ptr(), ctx->err_ptr());
    return paco::run_batch(ctx, ctx->batch, a_cat, h_a_off, b_cat, h_b_off, npairs, d_len, d_rows_cat, h_row_off,
                           d_cols_cat, h_col_off, (cudaStream_t)stream, true, force, ctx->opt_alphabet);
}
