// Single-pair LCS kernel for sm_103a: the whole path of one table in one
// launch.
//
// The table of Eq. (1) (Tang & Gao, Sec. "PACO LCS") is computed on its
// unit steps: in an LCS table neighbouring entries differ by 0 or 1, so a
// column of R rows is one R-bit word V (bit r set when H[r+1][j] ==
// H[r][j], i.e. no vertical step) and the horizontal step between columns
// at the word's top and bottom rows is one carry bit.  With M the rows whose
// symbol equals b[j], one column of Eq. (1) is
//
//     V' = (V + (V & M) + carry_in) | (V & ~M),   carry_out = carry of the sum
//
// (the bit-vector form of Allison & Dix 1986 / Crochemore et al. 2001 /
// Hyyrö 2004; carry_in is the top row's horizontal step at column j and
// carry_out the bottom row's).  A lane holds R = 31 rows (bit 31 of the word
// stays set, so the carry flag of the 32-bit add is the carry out); a warp
// holds 32 lanes x 31 rows, and each lane hands the carry bits of a chunk of
// C columns to the lane below through __shfl_up_sync.  Warps of one CTA
// strip chain through shared-memory rings, and CTA strips chain through
// global memory with epoch-tagged words.  One extra warp per CTA produces:
// it turns the column string into match-table offsets and delivers the
// strip's input carry words (the strip above's output, or the top boundary's
// steps for the first strip), so the compute warps never wait on global
// memory.  The PACO execution phase (regions run in anti-diagonal order,
// each waiting only on its neighbours, no global barrier) is this pipeline:
// lane g of strip s works on chunk q at step q + 3g.
//
// Everything around the table runs in the same launch:
// - the input boundaries are read as values: each lane turns its rows of the
//   left boundary into its first column's steps, and the first strip's
//   producer turns the top boundary into carry words (both checked to be
//   unit-step boundaries);
// - the right column needs no scan: a warp's first row r0 has
//   H[r0][S] = H[r0][0] + (horizontal steps along row r0), the set bits of the
//   carry words the warp consumed, so each warp writes its own rows of the
//   right column from that base and its lanes' last-column steps;
// - the last strip's producer expands the bottom row's carry words into
//   values as the last warp hands them over, and writes L;
// - the last CTA to leave resets the strip ticket for the next launch.
#include "paco_internal.hpp"
#include "bp_device.cuh"

#include <cuda_runtime.h>
#include <stdint.h>

namespace paco {
namespace {

using namespace dev;

// Lane skew in chunks: lane k works on chunk t - 3k at step t (with two
// words per lane, the lower word one chunk behind the upper, fed by its
// carries in registers).  The carry word a lane receives from the lane above
// (one __shfl_up_sync after each step's columns) was sent kSk - WPL + 1
// steps before it is needed: three with one word per lane, two with two
// words (whose lower word's columns already separate the shuffle from its
// use), which keeps the shuffle's latency off the column chain.
template <int WPL> __host__ __device__ constexpr int lane_skew() { return 3; }
// Chunks the last word of lane 31 trails the first word of lane 0.
template <int WPL> __host__ __device__ constexpr int lane_lag() { return lane_skew<WPL>() * 31 + (WPL - 1); }
// Warp 0's input carry words pass through a ring of tagged 64-bit words
// (the word index + 1 in the high half), so reading one needs no fence.
constexpr int kSrcSlots = 64;
// The compute warps check the column ring's fill level (an acquire load) and
// publish their progress (a release store) once per this many 32-column words.
constexpr int kCheckEvery = 4;
// A match table holds one 32-lane row per symbol and one all-zero row after
// them: columns outside [0, S) (before the first column while the lanes'
// pipeline fills, past the last one while it drains) read that row, so an
// idle lane keeps its state and passes zero carries, and one loop serves
// fill, steady state and drain.
constexpr size_t kPairTableBytes = kTableBytes + 128;
constexpr uint32_t kZeroRow = (uint32_t)kMaxSigma * 128u;
// Column-word lag of the oldest word a warp still reads behind the word its
// lane 0 is on (the lower word reuses the upper word's offsets).
__host__ __device__ constexpr int col_lag_words(int C, int WPL) {
    return (3 * 31 * C + (WPL - 1) * C + 31) / 32 + 1;
}
// Column-offset ring slots (a power of two) for C, W compute warps and WPL
// words per lane: the lag of the last warp behind the first, the in-warp lag,
// the look-ahead of one check period and the staleness of the progress words.
__host__ __device__ constexpr int col_slots(int C, int W, int WPL) {
    const int need = col_lag_words(C, WPL) + 2 * kCheckEvery + 4 + (W - 1) * (col_lag_words(C, WPL) + 2) + 8;
    int r = 32;
    while (r < need) r <<= 1;
    return r;
}

// Shared-memory layout of one CTA: W x WPL match tables, the column-offset
// ring (slots + two mirror slots, so a lane's window of the next 32 + 2C
// columns never wraps), the tagged input ring of warp 0, the tagged rings
// after each warp (the last one carries the bottom row to the producer in the
// last strip), and the counters: the producer's column count, then one
// progress word per compute warp and the producer's bottom-row count.
struct PairSmem {
    uint32_t tables, colring, srcring, rings, ctrl, bytes;
};
__host__ __device__ inline PairSmem pair_smem_layout(int W, int C, int WPL) {
    PairSmem L;
    L.tables = 0;
    L.colring = (uint32_t)(W * WPL * kPairTableBytes);
    L.srcring = L.colring + (uint32_t)(col_slots(C, W, WPL) + 2) * 128u;
    L.rings = L.srcring + (uint32_t)kSrcSlots * 8u;
    L.ctrl = L.rings + (uint32_t)(W * kRing * 8);
    L.bytes = L.ctrl + (uint32_t)(2 + W) * 4u + 16u;
    return L;
}

static __device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Compute warps wait here (uniformly: every lane reads the same word) for the
// column ring.  Bounded: false on a timeout or a raised error.
static __device__ __noinline__ bool wait_cols(uint32_t prod_cols, int need, int *err, long long limit) {
    const uint64_t t0 = global_ns();
    bool ok = true;
    while (ld_acquire_shared(prod_cols) < need) {
        if (ld_relaxed_i32(err) != 0) { ok = false; break; }
        if ((long long)(global_ns() - t0) > limit) {
            raise_error(err, kEtimeout);
            ok = false;
            break;
        }
    }
    return __all_sync(kFull, ok);
}

// ... and for a tagged input word (bounded like every wait): returns the
// word; its tag is still stale only after a timeout or a raised error.
static __device__ __noinline__ uint64_t wait_tagged(const uint64_t *slot, uint32_t tag, int *err, long long limit) {
    const uint64_t t0 = global_ns();
    uint64_t v;
    for (;;) {
        v = *reinterpret_cast<const volatile uint64_t *>(slot);
        if ((uint32_t)(v >> 32) == tag) break;
        if (ld_relaxed_i32(err) != 0) break;
        if ((long long)(global_ns() - t0) > limit) {
            raise_error(err, kEtimeout);
            break;
        }
    }
    return v;
}

// The match words of one chunk: the lane's row bits for each column's symbol.
template <int C>
static __device__ __forceinline__ void match_words(uint32_t pm_lane, const uint32_t (&o)[C], uint32_t (&M)[C]) {
#pragma unroll
    for (int jj = 0; jj < C; ++jj) M[jj] = lds_u32(pm_lane + o[jj]);
}

// Column offsets of one chunk from the ring.
template <int C>
static __device__ __forceinline__ void offs_at(uint32_t addr, uint32_t (&o)[C]) {
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
}

// Rows [row0, row1) of strip s: the PACO p-way first cut in lane granules
// (parts differ by at most one granule), or uniform strips.
static __device__ __forceinline__ void strip_rows(const PairArgs &P, int s, int64_t rows_lane, int64_t &row0,
                                                  int64_t &row1) {
    if (P.uniform_rows > 0) {
        row0 = min(P.L, (int64_t)s * P.uniform_rows);
        row1 = min(P.L, row0 + P.uniform_rows);
    } else {
        const int64_t q = P.granules / P.nstrips, r = P.granules % P.nstrips;
        row0 = min(P.L, rows_lane * ((int64_t)s * q + min((int64_t)s, r)));
        row1 = min(P.L, rows_lane * ((int64_t)(s + 1) * q + min((int64_t)(s + 1), r)));
    }
}

template <int C, int WPL>
__global__ void __launch_bounds__(256, 1) k_pair_bp(const PairArgs P) {
    static_assert(C == 2 || C == 4 || C == 8, "chunk widths 2, 4 and 8");
    static_assert(WPL == 1 || WPL == 2, "one or two words per lane");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_strip;
    const int W = (int)(blockDim.x >> 5) - 1;  // compute warps; warp W produces
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const PairSmem lay = pair_smem_layout(W, C, WPL);
    const int R = col_slots(C, W, WPL);
    const uint32_t sbase = smem_addr(smem);
    const uint32_t col_ring = sbase + lay.colring;
    const uint32_t prod_cols = sbase + lay.ctrl;
    const uint32_t cons_s = prod_cols + 4;  // progress word v (v = 0..W) at cons_s + 4 v
    volatile int *cons = reinterpret_cast<volatile int *>(smem + lay.ctrl + 4);
    uint64_t *srcq = reinterpret_cast<uint64_t *>(smem + lay.srcring);
    uint64_t *rings = reinterpret_cast<uint64_t *>(smem + lay.rings);
    uint64_t *ring_out = rings + (size_t)(w < W ? w : W - 1) * kRing;        // read by warp w+1 / the producer
    const uint32_t ring_out_s = smem_addr(ring_out);
    const uint64_t *ring_in = rings + (size_t)(w > 0 && w < W ? w - 1 : 0) * kRing;  // written by warp w-1
    // where this warp's input carry words arrive: warp 0's from the producer
    const uint32_t in_s = w == 0 ? smem_addr(srcq) : smem_addr(ring_in);
    const uint32_t in_mask = w == 0 ? (uint32_t)(kSrcSlots - 1) : (uint32_t)(kRing - 1);
    // table of word x of this warp (x = 0 upper, 1 lower)
    uint32_t *pm0 = reinterpret_cast<uint32_t *>(smem + (size_t)(w < W ? w * WPL : 0) * kPairTableBytes);
    uint32_t *pm1 = pm0 + (WPL == 2 ? kPairTableBytes / 4 : 0);
    const uint32_t pm_lane0 = smem_addr(pm0 + lane);
    const uint32_t pm_lane1 = smem_addr(pm1 + lane);

    if (w < W)
        for (int c = 0; c < (kMaxSigma + 1) * WPL; ++c) pm0[c * 32 + lane] = 0u;
    // every ring slot holds a valid table offset (the zero row) from the start
    for (int i = threadIdx.x; i < (R + 2) * 32; i += blockDim.x)
        reinterpret_cast<uint32_t *>(smem + lay.colring)[i] = kZeroRow;

    constexpr int K = 32 / C;                       // steps per 32-column word
    constexpr int kSk = lane_skew<WPL>();
    constexpr int kLag = lane_lag<WPL>();           // chunks lane 31's last word trails lane 0
    constexpr int kFlushStep = (kLag - 1) % K;      // step at which lane 31 completes a word
    constexpr int kLagW = col_lag_words(C, WPL);
    constexpr int kRowsLane = kLaneRows * WPL;
    const int nwords = P.nwords;
    // words lane 0 runs over: the real ones, then zero-row words until the
    // last lane has finished the last real word
    const int nouter = (nwords * K + kLag + K - 1) / K;
    const int nvwords = nouter + 2;                 // words the producer writes (with the prefetch)
    const int32_t *top = P.top, *left = P.left;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = atomicAdd(P.ctl, 1);
            if (ld_relaxed_i32(P.err) != 0) s = P.nstrips;
            s_strip = s;
            st_release_shared(prod_cols, 0);
        }
        if (threadIdx.x <= W) cons[threadIdx.x] = 0;
        for (int i = threadIdx.x; i < kSrcSlots + W * kRing; i += blockDim.x) {
            if (i < kSrcSlots) srcq[i] = 0ull;
            else rings[i - kSrcSlots] = 0ull;
        }
        __syncthreads();
        const int s = s_strip;
        if (s >= P.nstrips) break;
        const bool last_strip = s == P.nstrips - 1;
        int64_t row0, row1;
        strip_rows(P, s, kRowsLane, row0, row1);

        if (w == W) {
            // ---------------- producer warp ----------------
            // Column offsets (symbol x 128 bytes) from b into the ring, as far
            // ahead as the slowest compute warp allows; warp 0's input carry
            // words (the strip above's output polled in global memory, or the
            // top boundary's steps) into the tagged input ring; in the last
            // strip, the bottom row's carry words into values.
            int qc = 0, qs = 0, qb = 0;
            int32_t run = 0;  // bottom row: H[L][j] of the last column expanded
            const uint64_t *src_row = P.hbuf + (size_t)s * P.hstride;
            const uint32_t want = (s == P.stall_strip) ? (P.epoch ^ 0x80000000u) : P.epoch;
            uint32_t *ring = reinterpret_cast<uint32_t *>(smem + lay.colring);
            const uint64_t *bq = rings + (size_t)(W - 1) * kRing;
            // the words before column 0 (read while the lanes' pipeline fills): zero rows
            for (int j = 1; j <= kLagW + 1; ++j) ring[(uint32_t)((R - j) & (R - 1)) * 32 + lane] = kZeroRow;
            __syncwarp();
            if (s == 0 && lane == 0) {  // H[0][0] is both boundaries' first value
                const int32_t t0 = top ? top[0] : 0, l0 = left ? left[0] : 0;
                if (t0 != l0) raise_error(P.err, kEinval);
            }
            if (last_strip) {
                run = left ? left[P.L] : 0;
                if (lane == 0 && P.bottom) P.bottom[0] = run;
            }
            int idle = 0;
            uint64_t t_idle = global_ns();
            bool ok = true;
            while (qc < nvwords || qs < nwords || (last_strip && qb < nwords)) {
                bool progress = false;
                int minc = cons[0];
                for (int v = 1; v < W; ++v) minc = min(minc, cons[v]);
                const int lim_c = min(nvwords, minc - 1 - kLagW + R);
                // the strip above's next words: loaded first, so their latency
                // overlaps the column work below
                const int lim_s = min(nwords, cons[0] + kSrcSlots - 1);
                const int qp = qs + lane;
                uint64_t vp = 0;
                if (s > 0 && qp < lim_s) vp = ld_relaxed_u64(src_row + qp);
                if (qc < lim_c) {
                    const int qe = min(lim_c, qc + 8);
                    uint32_t o[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int64_t col = (int64_t)(qc + k) * 32 + lane;
                        o[k] = (qc + k < qe && col < P.S) ? (uint32_t)__ldg(P.b + col) * 128u : kZeroRow;
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        if (qc + k < qe) {
                            const uint32_t slot = (uint32_t)((qc + k) & (R - 1));
                            ring[slot * 32 + lane] = o[k];
                            if (slot < 2) ring[((uint32_t)R + slot) * 32 + lane] = o[k];
                        }
                    }
                    __syncwarp();
                    if (lane == 0) st_release_shared(prod_cols, qe);
                    qc = qe;
                    progress = true;
                }
                if (qs < lim_s) {
                    if (s > 0) {  // the strip above's output words, as they are published
                        const int q = qp;
                        const uint64_t v = vp;
                        const bool rd = q < lim_s && (uint32_t)(v >> 32) == want;
                        const uint32_t bal = __ballot_sync(kFull, rd);
                        const int n = (bal == kFull) ? 32 : (__ffs(~bal) - 1);
                        if (lane < n) srcq[q & (kSrcSlots - 1)] = ((uint64_t)(uint32_t)(q + 1) << 32) | (uint32_t)v;
                        if (n > 0) {
                            qs += n;
                            progress = true;
                        }
                    } else if (top == nullptr) {  // zero top boundary
                        const int q = qs + lane;
                        if (q < lim_s) srcq[q & (kSrcSlots - 1)] = (uint64_t)(uint32_t)(q + 1) << 32;
                        qs = min(lim_s, qs + 32);
                        progress = true;
                    } else {  // the top boundary's steps, MSB first, four words per pass
                        const int qe = min(lim_s, qs + 4);
                        int32_t v0[4], v1[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int64_t col = (int64_t)(qs + k) * 32 + lane;
                            const bool in = qs + k < qe && col < P.S;
                            v0[k] = in ? top[col] : 0;
                            v1[k] = in ? top[col + 1] : 0;
                        }
                        bool bad = false;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int32_t d = v1[k] - v0[k];
                            bad |= (d & ~1) != 0;
                            const uint32_t word = __brev(__ballot_sync(kFull, (d & 1) != 0));
                            if (qs + k < qe && lane == k)
                                srcq[(qs + k) & (kSrcSlots - 1)] = ((uint64_t)(uint32_t)(qs + k + 1) << 32) | word;
                        }
                        if (__any_sync(kFull, bad) && lane == 0) raise_error(P.err, kEinval);
                        qs = qe;
                        progress = true;
                    }
                }
                if (last_strip && qb < nwords) {  // the bottom row from the last warp's words
                    const int q = qb + lane;
                    uint64_t v = 0;
                    bool rd = false;
                    if (q < nwords) {
                        v = *reinterpret_cast<const volatile uint64_t *>(bq + (q & (kRing - 1)));
                        rd = (uint32_t)(v >> 32) == (uint32_t)(q + 1);
                    }
                    const uint32_t bal = __ballot_sync(kFull, rd);
                    const int n = (bal == kFull) ? 32 : (__ffs(~bal) - 1);
                    for (int k = 0; k < n; ++k) {
                        const uint32_t lsb = __brev(__shfl_sync(kFull, (uint32_t)v, k));  // bit t = column 32(qb+k) + t
                        if (P.bottom) {
                            const int64_t col = (int64_t)(qb + k) * 32 + lane;
                            if (col < P.S) P.bottom[col + 1] = run + __popc(lsb & ((2u << lane) - 1u));
                        }
                        run += __popc(lsb);
                    }
                    if (n > 0) {
                        qb += n;
                        __syncwarp();
                        if (lane == 0) st_release_shared(cons_s + 4u * (uint32_t)W, qb);
                        progress = true;
                    }
                }
                if (progress) {
                    t_idle = global_ns();
                    idle = 0;
                } else {
                    ++idle;
                    if ((idle & 15) == 0) {
                        if (ld_relaxed_i32(P.err) != 0) { ok = false; break; }
                        if ((long long)(global_ns() - t_idle) > P.wait_limit_ns) {
                            raise_error(P.err, kEtimeout);
                            ok = false;
                            break;
                        }
                    }
                    // short naps while the strip above is publishing (its next
                    // word is on the critical path), longer ones otherwise
                    if (idle > 4) __nanosleep(idle > 64 && !(s > 0 && qs < nwords && qs > 0) ? 256 : 32);
                }
            }
            if (ok && last_strip && lane == 0 && P.len) P.len[0] = run;
            continue;
        }

        // ---------------- compute warps ----------------
        const int64_t wrow0 = row0 + (int64_t)w * (32 * kRowsLane);  // the warp's first row
        const int64_t lbase = wrow0 + (int64_t)lane * kRowsLane;
        // per word x: first row, real rows, row symbols
        int64_t rbase[WPL];
        int nreal[WPL];
        uint32_t realmask[WPL];
        uint32_t aw[WPL][8];
        uint32_t Sv[WPL], Yv[WPL];
        bool badstep = false;
#pragma unroll
        for (int x = 0; x < WPL; ++x) {
            rbase[x] = lbase + x * kLaneRows;
            const int64_t left_rows = row1 - rbase[x];
            nreal[x] = left_rows <= 0 ? 0 : (left_rows >= kLaneRows ? kLaneRows : (int)left_rows);
            realmask[x] = (1u << nreal[x]) - 1u;
#pragma unroll
            for (int k = 0; k < 8; ++k) aw[x][k] = 0;
#pragma unroll
            for (int r = 0; r < kLaneRows; ++r)
                if (r < nreal[x]) aw[x][r >> 2] |= (uint32_t)__ldg(P.a + rbase[x] + r) << ((r & 3) * 8);
            uint32_t *pmx = x == 0 ? pm0 : pm1;
#pragma unroll
            for (int r = 0; r < kLaneRows; ++r) {
                if (r < nreal[x]) {
                    const uint32_t ch = (aw[x][r >> 2] >> ((r & 3) * 8)) & 0xffu;
                    pmx[ch * 32 + lane] |= 1u << r;
                }
            }
            // V from the first column's vertical steps (the left boundary's
            // unit steps; bit set = no step), padding rows 1, bit 31 held at 1
            uint32_t steps = 0;
            if (left != nullptr && nreal[x] > 0) {
                int32_t prev = left[rbase[x]];
                for (int r = 0; r < nreal[x]; ++r) {
                    const int32_t cur = left[rbase[x] + r + 1];
                    const int32_t d = cur - prev;
                    badstep |= (d & ~1) != 0;
                    steps |= (uint32_t)(d & 1) << r;
                    prev = cur;
                }
            }
            Sv[x] = ~steps;
            Yv[x] = 0;
        }
        if (badstep) raise_error(P.err, kEinval);
        __syncwarp();

        uint32_t cw[WPL], sr[WPL];  // carry-outs (newest in bit 0, never reset); carry-ins (next in bit 31)
#pragma unroll
        for (int x = 0; x < WPL; ++x) {
            cw[x] = 0;
            sr[x] = 0;
        }
        // the lane above's carry words: for this step and the ones after it
        constexpr int kQ = kSk - WPL + 1;
        uint32_t cinq[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) cinq[q] = 0;
        uint32_t Mcur[C];       // the upper word's match words for this step
        uint32_t onext[C];      // the next step's column offsets
        uint32_t oprev[C];      // two words: this step's offsets, for the lower word next step
        uint32_t Mlow[C];       // two words: the lower word's match words for this step
        bool ok = true;
        int cons_seen = 0;      // downstream consumer's progress word, last read
        int cols_seen = 0;      // the producer's column count, last read
        uint32_t steps_in = 0;  // set bits of the input carry words: horizontal steps along row wrow0
        const bool out_shared = (w + 1 < W) || last_strip;
        uint64_t *dst_row = P.hbuf + (size_t)(s + 1) * P.hstride;
        // the input carry word of the next 32-column word, read kPrefetch steps
        // before it is needed (so its load never stalls the column chain)
        constexpr int kPrefetch = K >= 8 ? K - 4 : 0;
        // the producer's count for the next word (acquire), then the vote on
        // the next word's needs, late in the word but a shared load's latency
        // after the loads they test
        constexpr int kAcquireStep = K >= 8 ? K - 3 : 1;
        constexpr int kVoteStep = K >= 8 ? K - 2 : 2;
        auto in_slot = [&](int q) { return in_s + (((uint32_t)q & in_mask) << 3); };
        uint64_t in_next = nwords > 0 ? lds_u64(in_slot(0)) : 0ull;
        {   // the first word's offsets and match words (later words: carried over)
            const uint32_t cb0 = col_ring + (uint32_t)(((-kSk * C * lane) >> 5 & (R - 1)) * 128) +
                                 (uint32_t)(((-kSk * C * lane) & 31) * 4);
            uint32_t o0[C];
            offs_at<C>(cb0, o0);
            match_words<C>(pm_lane0, o0, Mcur);
            if constexpr (WPL == 2) {
                // the lower word's chunk of step 0 (one behind) lies before column 0
#pragma unroll
                for (int jj = 0; jj < C; ++jj) {
                    Mlow[jj] = 0u;
                    oprev[jj] = o0[jj];
                }
            }
            offs_at<C>(cb0 + (uint32_t)(C * 4), onext);
        }
        // Word u needs: the column ring filled up to word u + 1 (the words its
        // lanes read; the producer's count is read with acquire, and the reads
        // of the ring follow it), its input carry word tagged u + 1 (warp 0's
        // from the producer, the others' from the warp above), and, when its
        // lane 31 flushes into a shared ring, that slot read by the consumer
        // (the next warp, or the producer for the bottom row).  The fast loop
        // tests the next word's needs by one vote in the middle of the current
        // word, so the branch at the word boundary finds its predicate ready,
        // and it leaves before the first word that lacks something.  The waits
        // (function calls) sit in the slow path outside it.
        int u = 0;
        for (;;) {
            if (u >= nouter) break;
            {   // the slow path: wait (bounded) for what word u lacks
                const int need_c = min(u + 2, nvwords);
                const int wq_u = ((u * K + kFlushStep - kLag) * C) >> 5;
                const int need_out = out_shared ? min(wq_u, nwords - 1) - kRing + 1 : 0;
                if (!wait_cols(prod_cols, need_c, P.err, P.wait_limit_ns)) {
                    ok = false;
                    break;
                }
                cols_seen = ld_acquire_shared(prod_cols);
                if (u < nwords && !__all_sync(kFull, (uint32_t)(in_next >> 32) == (uint32_t)(u + 1))) {
                    in_next = wait_tagged(reinterpret_cast<const uint64_t *>(smem + (in_slot(u) - sbase)),
                                          (uint32_t)(u + 1), P.err, P.wait_limit_ns);
                    if (!__all_sync(kFull, (uint32_t)(in_next >> 32) == (uint32_t)(u + 1))) {
                        ok = false;
                        break;
                    }
                }
                if (need_out > cons_seen) {
                    if (!__all_sync(kFull, wait_consumed(cons + w + 1, need_out, P.err, P.wait_limit_ns))) {
                        ok = false;
                        break;
                    }
                    cons_seen = cons[w + 1];
                }
            }
            bool stop = false;  // the next word lacks something
            // Words per iteration: a multiple of K steps that is also one of
            // the carry queue's kQ entries, so the queue's rotation ends where
            // it started and the loop's back edge moves no registers (with one
            // word per lane, kQ = 3: three words ran the 131072 pair 3% faster
            // than two; with two words per lane, kQ = 2 and two words stay
            // best).
#pragma unroll(kQ == 3 ? 3 : 2)
            for (; u < nouter;) {
                // the input carry word u (its tag was checked)
                const uint32_t srcw = u < nwords ? (uint32_t)in_next : 0u;
                steps_in += __popc(srcw);
                st_release_shared_if(lane == 0 && (u & (kCheckEvery - 1)) == kCheckEvery - 1, cons_s + 4u * (uint32_t)w,
                                     u + 1);
                const int ubase = u * K;
                // this lane's column of step 0 (upper word) and its place in the ring
                const int c0 = u * 32 - kSk * C * lane;
                const uint32_t cbase = col_ring + (uint32_t)(((c0 >> 5) & (R - 1)) * 128) + (uint32_t)((c0 & 31) * 4);
                if (lane == 0) sr[0] = srcw;
                // Software pipeline: offsets two steps ahead, match words one step
                // ahead, the carry hand-off after the step's columns (its result is
                // used three steps later), so a warp issuing in order never waits on
                // a shared load or a shuffle before a column.  Columns outside
                // [0, S) read the zero row: no per-lane activity tests.
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    uint32_t onext2[C], Mnext[C], Mlow_next[C];
                    offs_at<C>(cbase + (uint32_t)((i + 2) * C * 4), onext2);
                    match_words<C>(pm_lane0, onext, Mnext);
                    if constexpr (WPL == 2) match_words<C>(pm_lane1, oprev, Mlow_next);
                    if (i == kPrefetch) in_next = lds_u64(in_slot(u + 1));  // any slot is readable
                    if (i == kAcquireStep)  // the count the next word's reads follow, once per kCheckEvery words
                        ld_acquire_shared_if(((u + 1) & (kCheckEvery - 1)) == 0, prod_cols, cols_seen);
                    if (i == kVoteStep) {  // the next word's needs
                        const int v1 = u + 1;
                        const int need_c = min(v1 + 2, nvwords);
                        const int wq_v = ((v1 * K + kFlushStep - kLag) * C) >> 5;
                        const int need_out = out_shared ? min(wq_v, nwords - 1) - kRing + 1 : 0;
                        const bool stale = v1 < nwords && (uint32_t)(in_next >> 32) != (uint32_t)(v1 + 1);
                        stop = __any_sync(kFull, cols_seen < need_c || stale || need_out > cons_seen);
                    }
                    if (lane != 0) sr[0] = cinq[0] << (32 - C);
                    if constexpr (WPL == 2) {
                        sr[1] = cw[0] << (32 - C);  // the upper word's carries of the step before
#pragma unroll
                        for (int jj = 0; jj < C; ++jj) {
                            column31c(Sv[0], Yv[0], sr[0], cw[0], Mcur[jj]);
                            column31c(Sv[1], Yv[1], sr[1], cw[1], Mlow[jj]);
                        }
                    } else {
#pragma unroll
                        for (int jj = 0; jj < C; ++jj) column31c(Sv[0], Yv[0], sr[0], cw[0], Mcur[jj]);
                    }
                    const uint32_t recv = __shfl_up_sync(kFull, cw[WPL - 1], 1);
#pragma unroll
                    for (int q = 0; q + 1 < kQ; ++q) cinq[q] = cinq[q + 1];
                    cinq[kQ - 1] = recv;
#pragma unroll
                    for (int jj = 0; jj < C; ++jj) {
                        Mcur[jj] = Mnext[jj];
                        if constexpr (WPL == 2) {
                            Mlow[jj] = Mlow_next[jj];
                            oprev[jj] = onext[jj];
                        }
                        onext[jj] = onext2[jj];
                    }
                    if (i == kFlushStep) {  // lane 31 completes word wq: predicated stores, no branch
                        const int wq = ((ubase + i - kLag) * C) >> 5;
                        const bool fl = lane == 31 && wq >= 0 && wq < nwords;
                        const uint64_t word = ((uint64_t)(uint32_t)(wq + 1) << 32) | cw[WPL - 1];
                        // to the next warp or the producer (the slot was checked free) ...
                        sts_u64_if(fl && out_shared, ring_out_s + (uint32_t)((wq & (kRing - 1)) * 8), word);
                        // ... or to the next strip, tagged with the launch epoch
                        st_relaxed_u64_if(fl && !out_shared, dst_row + (fl ? wq : 0),
                                          ((uint64_t)P.epoch << 32) | cw[WPL - 1]);
                    }
            }
            ++u;
            if (stop) break;
            }
        }
        if (lane == 0) st_release_shared(cons_s + 4u * (uint32_t)w, nouter);
        // The right column: H[i][S] for this warp's rows, from H[wrow0][S] =
        // H[wrow0][0] + (horizontal steps along row wrow0) and the lanes'
        // vertical steps at the last column, in row order (lane-major).
        if (ok && P.right != nullptr && wrow0 < row1) {
            uint32_t vbits[WPL];
            int cnt = 0;
#pragma unroll
            for (int x = 0; x < WPL; ++x) {
                vbits[x] = ~(Sv[x] | Yv[x]) & realmask[x];
                cnt += __popc(vbits[x]);
            }
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += y;
            }
            const int32_t base = (left ? left[wrow0] : 0) + (int32_t)steps_in;
            if (s == 0 && w == 0 && lane == 0) P.right[0] = base;  // H[0][S]
            int32_t val = base + inc - cnt;
#pragma unroll
            for (int x = 0; x < WPL; ++x) {
                for (int r = 0; r < nreal[x]; ++r) {
                    val += (int32_t)((vbits[x] >> r) & 1u);
                    P.right[rbase[x] + r + 1] = val;
                }
            }
        }
#pragma unroll
        for (int x = 0; x < WPL; ++x) {
            uint32_t *pmx = x == 0 ? pm0 : pm1;
#pragma unroll
            for (int r = 0; r < kLaneRows; ++r) {
                if (r < nreal[x]) {
                    const uint32_t ch = (aw[x][r >> 2] >> ((r & 3) * 8)) & 0xffu;
                    pmx[ch * 32 + lane] = 0u;
                }
            }
        }
    }
    // The last CTA to leave resets the strip ticket and the exit count, so the
    // next launch on the stream starts from zero without a separate memset.
    if (threadIdx.x == 0) {
        __threadfence();
        const int d = atomicAdd(P.ctl + 1, 1);
        if (d == (int)gridDim.x - 1) {
            atomicExch(P.ctl, 0);
            atomicExch(P.ctl + 1, 0);
        }
    }
}

__global__ void k_degenerate(const int32_t *top, const int32_t *left, int64_t n, int64_t m,
                             int32_t *bottom_row, int32_t *right_col, int32_t *len, int *err) {
    // n == 0: the table is the single row `top`; m == 0: the single column `left`.
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = tid; j <= m; j += stride) {
        int32_t v;
        if (n == 0) v = top ? top[j] : 0;
        else v = left ? left[n] : 0;  // m == 0: only j == 0
        if (bottom_row) bottom_row[j] = v;
    }
    for (int64_t i = tid; i <= n; i += stride) {
        int32_t v;
        if (m == 0) v = left ? left[i] : 0;
        else v = top ? top[m] : 0;  // n == 0: only i == 0
        if (right_col) right_col[i] = v;
    }
    if (tid == 0) {
        if (top && left && top[0] != left[0]) atomicCAS(err, 0, kEinval);
        if (len) len[0] = (n == 0) ? (top ? top[m] : 0) : (left ? left[n] : 0);
    }
}

// Integer ALU microbenchmark: 8 independent dependency chains per thread.
__global__ void k_int_peak(int op, int iters, uint32_t *sink) {
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 2654435761u + k * 40503u + blockIdx.x;
    const uint32_t m1 = 0x9E3779B9u ^ threadIdx.x, m2 = 0x7F4A7C15u + blockIdx.x;
    if (op == 0) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = x[k] + m1 + (x[k] >> 0);  // 3-input add
        }
    } else if (op == 1) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = (x[k] & m1) ^ (x[k] | m2);  // 3-input logic
        }
    } else if (op == 2) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = max(x[k] ^ 0u, m1 + (uint32_t)i) ;  // max (+ add)
        }
    } else {
        // the column step of the bit-parallel kernel, 8 independent lanes' worth
        uint32_t y[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) y[k] = 0;
        for (int i = 0; i < iters; ++i) {
            const uint32_t M = m1 * (uint32_t)i;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t V = x[k] | y[k];
                const uint32_t X = V & M;
                y[k] = V & ~M;
                const uint64_t s = (uint64_t)V + X + (i & 1);
                x[k] = (uint32_t)s + (uint32_t)(s >> 32);
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc ^= x[k];
    if (acc == 0x12345678u) sink[blockIdx.x] = acc;  // keep the chains live
}

}  // namespace

size_t pair_smem_bytes(int warps, int C, int wpl) { return pair_smem_layout(warps, C, wpl).bytes; }

int pair_max_warps(int wpl) {
    int w = 1;  // the widest chunk (largest column ring) bounds every configuration
    while (w < 7 && pair_smem_bytes(w + 1, 8, wpl) <= 227 * 1024 - 64) ++w;
    return w;
}

template <int C, int WPL>
static cudaError_t launch_cw(const PairArgs &p, int warps, int grid, cudaStream_t st) {
    const size_t smem = pair_smem_bytes(warps, C, WPL);
    cudaError_t e = cudaFuncSetAttribute(k_pair_bp<C, WPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_pair_bp<C, WPL><<<grid, (warps + 1) * 32, smem, st>>>(p);  // + the producer warp
    return cudaGetLastError();
}

template <int C, int WPL>
static int occ_cw(int warps) {
    const size_t smem = pair_smem_bytes(warps, C, WPL);
    if (cudaFuncSetAttribute(k_pair_bp<C, WPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pair_bp<C, WPL>, (warps + 1) * 32, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

int pair_occupancy(int C, int warps, int wpl) {
    if (wpl == 2) {
        switch (C) {
            case 2: return occ_cw<2, 2>(warps);
            case 4: return occ_cw<4, 2>(warps);
            case 8: return occ_cw<8, 2>(warps);
            default: return 0;
        }
    }
    switch (C) {
        case 2: return occ_cw<2, 1>(warps);
        case 4: return occ_cw<4, 1>(warps);
        case 8: return occ_cw<8, 1>(warps);
        default: return 0;
    }
}

cudaError_t launch_pair_bp(const PairArgs &p, int C, int warps, int wpl, int grid, cudaStream_t st) {
    if (warps < 1 || warps > 7 || grid < 1 || p.nstrips < 1) return cudaErrorInvalidValue;
    if (wpl == 2) {
        switch (C) {
            case 2: return launch_cw<2, 2>(p, warps, grid, st);
            case 4: return launch_cw<4, 2>(p, warps, grid, st);
            case 8: return launch_cw<8, 2>(p, warps, grid, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (C) {
        case 2: return launch_cw<2, 1>(p, warps, grid, st);
        case 4: return launch_cw<4, 1>(p, warps, grid, st);
        case 8: return launch_cw<8, 1>(p, warps, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_degenerate(const int32_t *top, const int32_t *left, int64_t n, int64_t m,
                              int32_t *bottom_row, int32_t *right_col, int32_t *len, int *err,
                              cudaStream_t st) {
    const int64_t mx = (n > m ? n : m) + 1;
    const int grid = (int)min((int64_t)1024, (mx + 255) / 256);
    k_degenerate<<<grid, 256, 0, st>>>(top, left, n, m, bottom_row, right_col, len, err);
    return cudaGetLastError();
}

cudaError_t launch_int_peak(int op, int grid, int block, int iters, uint32_t *sink, cudaStream_t st) {
    k_int_peak<<<grid, block, 0, st>>>(op, iters, sink);
    return cudaGetLastError();
}

}  // namespace paco
