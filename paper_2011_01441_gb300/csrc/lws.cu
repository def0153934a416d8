// The 1D problem of Sec. "PACO 1D" (least weight subsequence, Eq. 1D):
// D[j] = min_{i<j} D[i] + w(i, j).  Block kernel, host launch and the C ABI
// of include/paco_lws.h.
//
// Layout.  The outputs are cut into blocks of kLwsBlock consecutive j (a
// CTA of kLwsBlock threads works on one block at a time, thread t <-> j =
// block start + t).  The work of the recurrence is the triangle
// {(i, j): i < j}, cut into the squares (a, b) of block pairs a < b and the
// diagonal triangles of the blocks, like the quadrants of the paper's
// recursion.  Jobs, in the order a CTA takes them from an atomic ticket:
//
//   T(0), T(1), S(0, 2), T(2), S(0, 3), S(1, 3), T(3), ...
//
// (every job after the jobs it waits for, so a job only ever waits for a
// running or finished one; the order is computed from the ticket number).
// S(a, b) folds min_i D[i] + w(i, j) over block a into block b's running
// minima P[j] with atomicMin and counts itself done.  T(b) folds block b - 1
// in itself 32 values at a time as they are finished (so that square
// overlaps T(b - 1)), then waits for its b - 1 squares and takes their
// minima, then solves its diagonal triangle 32 values at a time: warp s finishes its values by a sequential
// sweep in which every lane carries the chain D[k] -> D[k+1] itself (the
// running minimum of lane k + 1 is shuffled a step early), and the later
// warps fold those 32 values in before their own turn.  Finished values are
// published as 64-bit words (launch tag in the high half, D in the low
// half), written and read as single accesses, so a reader can tell them
// from stale words without fences or flags.  Every wait is bounded.
#include "../../include/paco_lws.h"
#include "bp_device.cuh"
#include "ctx.hpp"
#include "paco_internal.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

namespace paco {
namespace {

constexpr int kLwsBlock = 256;            // outputs per block = threads per CTA
constexpr int kLwsWarps = kLwsBlock / 32;
constexpr int kLwsMaxSms = 1024;          // entries of the per-SM busy counters (a power of two)
constexpr long long kLwsYieldNs = 50000;  // longest a square waits for a triangle job on its SM
constexpr size_t kLwsWeightBytes = (size_t)kLwsWarps * 2 * 32 * 32 * sizeof(int);   // 64 KB
constexpr int kLwsInf = 0x3f3f3f3f;       // above every D (D < 2^29 + 2^24 + 256 by the argument checks);
                                          // its byte pattern lets a memset fill P

struct LwsArgs {
    int64_t n;
    int d0;
    int T;
    uint32_t seed;
    uint32_t noise_mask;   // 255 or 0
    int32_t *D;            // n + 1 outputs
    uint64_t *hand;        // n + 1 tagged words (tag << 32 | D)
    int *P;                // n + 1 running minima from the squares (kLwsInf before launch)
    int *done;             // per block: squares folded into it (0 before launch)
    int *busy;             // per SM: triangle jobs running their chain part (0 before launch)
    unsigned long long *ticket;
    int64_t njobs;
    uint32_t tag;          // nonzero tag of this launch
    int nblocks;
    int *err;
    long long wait_limit_ns;
    int stall_block;       // tests: block whose triangle waits for words that never come (-1: none)
};

static __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// w(i, j) with jt = j - T and js = j ^ seed precomputed by the caller.
static __device__ __forceinline__ int lws_w(int i, int jt, uint32_t js, uint32_t noise_mask) {
    const int d = jt - i;
    const int q = (d > -4096 && d < 4096) ? d * d : (1 << 24);
    return q + (int)(fmix32(((uint32_t)i * 0x9E3779B1u) ^ js) & noise_mask);
}

// The hashed byte of w(i, j) alone (js = j ^ seed).
static __device__ __forceinline__ int lws_noise(int i, uint32_t js, uint32_t noise_mask) {
    return (int)(fmix32(((uint32_t)i * 0x9E3779B1u) ^ js) & noise_mask);
}

// Folds the staged values s[0..count) of i0 .. i0 + count - 1 into best.
// FAR: every jump of the tile is at least 4096 away from T, so the squared
// term is the constant 2^24 for all of them and is added once.
template <bool FAR, int COUNT>
static __device__ __forceinline__ int fold_tile(int best, const int *s, int i0, int jt, uint32_t js,
                                                uint32_t noise_mask) {
    if (FAR) {
        int m = kLwsInf;
#pragma unroll 8
        for (int k = 0; k < COUNT; ++k) m = min(m, s[k] + lws_noise(i0 + k, js, noise_mask));
        return min(best, m + (1 << 24));
    }
#pragma unroll 8
    for (int k = 0; k < COUNT; ++k) best = min(best, s[k] + lws_w(i0 + k, jt, js, noise_mask));
    return best;
}

static __device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Stages `count` finished values starting at word `i0` into s_val: threads
// t < count load a word each and reload until every word carries `tag`
// (bounded wait).  CTA-uniform; false on timeout or a raised error.
static __device__ __noinline__ bool stage_values(const uint64_t *hand, int64_t i0, int count, uint32_t tag,
                                                 int *err, long long limit, int *s_val, int *s_bad) {
    const int t = threadIdx.x;
    uint64_t w = 0;
    if (t < count) w = dev::ld_relaxed_u64(hand + i0 + t);
    bool ready = t >= count || (uint32_t)(w >> 32) == tag;
    if (!__syncthreads_and(ready)) {
        // poll the stale words; the error word and the clock are looked at
        // every 32 rounds, and the CTA sleeps between rounds only after 64
        const uint64_t t0 = dev::global_ns();
        for (int spin = 1;; ++spin) {
            if (t == 0 && (spin & 31) == 0) {
                int bad = 0;
                if (dev::ld_relaxed_i32(err) != 0) {
                    bad = 1;
                } else if ((long long)(dev::global_ns() - t0) > limit) {
                    dev::raise_error(err, kEtimeout);
                    bad = 1;
                }
                *s_bad = bad;
            }
            if (spin > 64) __nanosleep(64);
            if (!ready) {
                w = dev::ld_relaxed_u64(hand + i0 + t);
                ready = (uint32_t)(w >> 32) == tag;
            }
            const bool all = __syncthreads_and(ready);   // also orders *s_bad
            if (all) break;
            if ((spin & 31) == 0 && *s_bad) return false;
        }
    }
    if (t < count) s_val[t] = (int)(uint32_t)w;
    __syncthreads();
    return true;
}

// Like stage_values for a word w each thread t < count loaded earlier:
// checks the tags, reloads the stale words (bounded wait) and stages the
// values into s_val.  CTA-uniform; false on timeout or a raised error.
static __device__ __noinline__ bool settle_values(const uint64_t *hand, int64_t i0, int count, uint32_t tag,
                                                  int *err, long long limit, uint64_t w, int *s_val, int *s_bad) {
    const int t = threadIdx.x;
    bool ready = t >= count || (uint32_t)(w >> 32) == tag;
    if (!__syncthreads_and(ready)) {
        const uint64_t t0 = dev::global_ns();
        for (int spin = 1;; ++spin) {
            if (t == 0 && (spin & 31) == 0) {
                int bad = 0;
                if (dev::ld_relaxed_i32(err) != 0) {
                    bad = 1;
                } else if ((long long)(dev::global_ns() - t0) > limit) {
                    dev::raise_error(err, kEtimeout);
                    bad = 1;
                }
                *s_bad = bad;
            }
            if (spin > 64) __nanosleep(64);
            if (!ready) {
                w = dev::ld_relaxed_u64(hand + i0 + t);
                ready = (uint32_t)(w >> 32) == tag;
            }
            const bool all = __syncthreads_and(ready);   // also orders *s_bad
            if (all) break;
            if ((spin & 31) == 0 && *s_bad) return false;
        }
    }
    if (t < count) s_val[t] = (int)(uint32_t)w;
    __syncthreads();
    return true;
}

// Job of ticket x: sets *a (-1 for a triangle) and *b.  Level b >= 1 holds
// S(0, b) .. S(b - 2, b), T(b) and starts at ticket 1 + b (b - 1) / 2.
static __device__ __forceinline__ void lws_job(int64_t x, int *a, int *b) {
    if (x == 0) {
        *a = -1;
        *b = 0;
        return;
    }
    int64_t lv = (int64_t)((1.0 + sqrt(8.0 * (double)(x - 1) + 1.0)) * 0.5);
    while (1 + lv * (lv - 1) / 2 > x) --lv;
    while (1 + (lv + 1) * lv / 2 <= x) ++lv;
    const int64_t idx = x - (1 + lv * (lv - 1) / 2);
    *b = (int)lv;
    *a = idx < lv - 1 ? (int)idx : -1;
}

static __device__ __forceinline__ int smid() {
    int v;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
    return v;
}

static __device__ __forceinline__ int ld_acquire_i32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ int ld_relaxed_l2(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits (bounded) until *cnt >= need; CTA-uniform result.
static __device__ __noinline__ bool wait_count(const int *cnt, int need, int *err, long long limit, int *s_bad) {
    if (threadIdx.x == 0) {
        int bad = 0;
        if (ld_acquire_i32(cnt) < need) {
            const uint64_t t0 = dev::global_ns();
            for (int spin = 0;; ++spin) {
                if (spin > 8) __nanosleep(64);
                if (ld_acquire_i32(cnt) >= need) break;
                if (dev::ld_relaxed_i32(err) != 0) {
                    bad = 1;
                    break;
                }
                if ((long long)(dev::global_ns() - t0) > limit) {
                    dev::raise_error(err, kEtimeout);
                    bad = 1;
                    break;
                }
            }
        }
        *s_bad = bad;
    }
    __syncthreads();
    return *s_bad == 0;
}

__global__ void __launch_bounds__(kLwsBlock, 3) k_lws(LwsArgs P) {
    extern __shared__ int s_wts[];   // per warp: [2][32 k][32 lanes] weights of the triangle
    __shared__ int s_D[kLwsBlock];
    __shared__ int s_sub[2][32];
    __shared__ int64_t s_ticket;
    __shared__ int s_bad;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    for (;;) {
        // a raised error ends every CTA at its next job
        if (t == 0) s_ticket = dev::ld_relaxed_i32(P.err) != 0 ? P.njobs : (int64_t)atomicAdd(P.ticket, 1ull);
        __syncthreads();
        const int64_t x = s_ticket;
        __syncthreads();
        if (x >= P.njobs) return;
        int a, b;
        lws_job(x, &a, &b);
        const int64_t j64 = (int64_t)b * kLwsBlock + t;
        const int j = (int)j64;
        const int jt = j - P.T;
        const uint32_t js = (uint32_t)j ^ P.seed;

        if (a >= 0) {
            // S(a, b): fold the whole block a (a < b - 1, a full block).  A
            // square yields its SM while a triangle job there runs its part of
            // the chain (at most kLwsYieldNs): the chain sets the pace.
            if (t == 0) {
                const int *bz = P.busy + (smid() & (kLwsMaxSms - 1));
                if (dev::ld_relaxed_i32(bz) > 0) {
                    const uint64_t t0 = dev::global_ns();
                    while (dev::ld_relaxed_i32(bz) > 0 && (long long)(dev::global_ns() - t0) < kLwsYieldNs)
                        __nanosleep(256);
                }
            }
            __syncthreads();
            const int i0 = a * kLwsBlock;
            if (!stage_values(P.hand, i0, kLwsBlock, P.tag, P.err, P.wait_limit_ns, s_D, &s_bad)) return;
            // jumps of this square span [b start - T - (i0 + 255), b end - T - i0]
            const int64_t dlo = (int64_t)b * kLwsBlock - P.T - (i0 + kLwsBlock - 1);
            const int64_t dhi = (int64_t)b * kLwsBlock + kLwsBlock - 1 - P.T - i0;
            const bool far = dlo >= 4096 || dhi <= -4096;
            const int best = far ? fold_tile<true, kLwsBlock>(kLwsInf, s_D, i0, jt, js, P.noise_mask)
                                 : fold_tile<false, kLwsBlock>(kLwsInf, s_D, i0, jt, js, P.noise_mask);
            if (j64 <= P.n) atomicMin(P.P + j64, best);
            __threadfence();
            __syncthreads();
            if (t == 0) atomicAdd(P.done + b, 1);
            continue;
        }

        // T(b).  First, while the inputs are still coming: each lane's weights
        // of its own warp's 32 values (the sweep) and of the warp before's 32
        // values (the fold on the triangle's critical path), into this lane's
        // column of the warp's shared tables.
        const int i0 = b * kLwsBlock;
        {
            int *sw = s_wts + warp * (2 * 32 * 32);
            const int ib = i0 + 32 * warp;
#pragma unroll 4
            for (int k = 0; k < 32; ++k) {
                sw[k * 32 + lane] = lws_w(ib + k, jt, js, P.noise_mask);
                sw[32 * 32 + k * 32 + lane] = lws_w(ib - 32 + k, jt, js, P.noise_mask);
            }
        }
        int best = j == 0 ? P.d0 : kLwsInf;
        int *bz = P.busy + (smid() & (kLwsMaxSms - 1));
        if (t == 0) atomicAdd(bz, 1);
        // square (b - 1, b), 32 values at a time as T(b - 1) finishes them;
        // the words of the next 32 are loaded before this 32 are folded, so
        // a word is mostly checked after it has arrived
        if (b > 0) {
            const uint32_t want = b == P.stall_block ? P.tag ^ 0x80000000u : P.tag;
            const int64_t h0 = (int64_t)(b - 1) * kLwsBlock;
            uint64_t pre = t < 32 ? dev::ld_relaxed_u64(P.hand + h0 + t) : 0;
            for (int s = 0; s < kLwsWarps; ++s) {
                const int i0 = (b - 1) * kLwsBlock + 32 * s;
                int *sv = s_sub[s & 1];
                if (!settle_values(P.hand, h0 + 32 * s, 32, want, P.err, P.wait_limit_ns, pre, sv, &s_bad)) {
                    if (t == 0) atomicSub(bz, 1);
                    return;
                }
                if (s + 1 < kLwsWarps && t < 32) pre = dev::ld_relaxed_u64(P.hand + h0 + 32 * (s + 1) + t);
                best = fold_tile<false, 32>(best, sv, i0, jt, js, P.noise_mask);
            }
        }
        // then the squares (a, b), a < b - 1, which are in P once all have
        // counted: waiting for them only after block b - 1 is folded keeps that
        // fold overlapped with T(b - 1) (the square (b - 2, b) starts only when
        // block b - 2 is final, and often ends after T(b - 1) does)
        if (b >= 2) {
            if (!wait_count(P.done + b, b - 1, P.err, P.wait_limit_ns, &s_bad)) {
                if (t == 0) atomicSub(bz, 1);
                return;
            }
            if (j64 <= P.n) best = min(best, ld_relaxed_l2(P.P + j64));
        }

        // the diagonal triangle of block b, 32 values at a time
        const int *sw = s_wts + warp * (2 * 32 * 32) + lane;
        // lane l's weight of the jump from its predecessor, w(j - 1, j): the
        // chain D[k] -> D[k+1] of the sweeps below takes it by one shuffle
        const int wstep = lws_w(j - 1, jt, js, P.noise_mask);
        for (int s = 0; s < kLwsWarps; ++s) {
            if (warp == s) {
                // lane k's minimum is final once lanes < k are folded in; every
                // lane carries D[ib + k] itself, and the running minimum of
                // lane k + 1 (folded up to D[ib + k - 1]) is shuffled a step early
                const int ib = i0 + 32 * s;
                int dk = __shfl_sync(dev::kFull, best, 0);
#pragma unroll
                for (int k = 0; k < 31; ++k) {
                    const int xk = __shfl_sync(dev::kFull, best, k + 1);
                    const int wk = __shfl_sync(dev::kFull, wstep, k + 1);
                    if (lane > k) best = min(best, dk + sw[k * 32]);
                    dk = min(xk, dk + wk);
                }
                s_D[t] = best;
                if (j64 <= P.n) {
                    P.D[j64] = best;
                    st_relaxed_u64(P.hand + j64, ((uint64_t)P.tag << 32) | (uint32_t)best);
                }
            }
            __syncthreads();
            if (warp == s + 1) {   // the next sweep's warp: its weights are in the table
#pragma unroll 8
                for (int k = 0; k < 32; ++k) best = min(best, s_D[32 * s + k] + sw[32 * 32 + k * 32]);
            } else if (warp > s + 1) {
                best = fold_tile<false, 32>(best, s_D + 32 * s, i0 + 32 * s, jt, js, P.noise_mask);
            }
        }
        __syncthreads();
        if (t == 0) atomicSub(bz, 1);
    }
}

}  // namespace

// Scratch of the 1D path, owned by the context.
struct LwsState {
    DevBuf ticket, hand, part, done, busy;
    uint32_t tag = 0;   // tag of the last launch (0: none yet)
};

void lws_state_free(LwsState *L) {
    if (!L) return;
    for (DevBuf *d : {&L->ticket, &L->hand, &L->part, &L->done, &L->busy})
        if (d->ptr) cudaFree(d->ptr);
    delete L;
}

}  // namespace paco

using namespace paco;

extern "C" int paco_lws(paco_ctx *ctx, int64_t n, int32_t d0, const paco_lws_weight *w, int32_t *d_D, void *stream) {
    if (!ctx || !w || !d_D || n < 0 || n > (int64_t(1) << 30) || d0 < 0 || d0 >= (1 << 29)) return PACO_EINVAL;
    if (w->T < -(1 << 20) || w->T > (1 << 20) || (w->noise != 0 && w->noise != 1)) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->lws) ctx->lws = new (std::nothrow) LwsState();
    LwsState *L = ctx->lws;
    if (!L) return PACO_ENOMEM;
    const int nblocks = (int)((n + 1 + kLwsBlock - 1) / kLwsBlock);
    int rc = ensure_bytes(ctx, L->ticket, 16);
    if (rc == PACO_OK) rc = ensure_bytes(ctx, L->hand, ((size_t)n + 1) * sizeof(uint64_t));
    if (rc == PACO_OK) rc = ensure_bytes(ctx, L->part, ((size_t)n + 1) * sizeof(int));
    if (rc == PACO_OK) rc = ensure_bytes(ctx, L->done, (size_t)nblocks * sizeof(int));
    if (rc == PACO_OK) rc = ensure_bytes(ctx, L->busy, (size_t)kLwsMaxSms * sizeof(int));
    if (rc != PACO_OK) return rc;
    // a new tag per launch: words of older launches never carry it (the
    // buffer is zeroed when it grows and cleared when the tag wraps)
    L->tag = L->tag == 0xffffffffu ? 1u : L->tag + 1u;
    cudaError_t e = cudaSuccess;
    if (L->tag == 1) e = cudaMemsetAsync(L->hand.ptr, 0, L->hand.bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->ticket.ptr, 0, sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->part.ptr, 0x3f, ((size_t)n + 1) * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->done.ptr, 0, (size_t)nblocks * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->busy.ptr, 0, (size_t)kLwsMaxSms * sizeof(int), st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "lws set-up");
    LwsArgs P{};
    P.n = n;
    P.d0 = d0;
    P.T = w->T;
    P.seed = w->seed;
    P.noise_mask = w->noise ? 255u : 0u;
    P.D = d_D;
    P.hand = (uint64_t *)L->hand.ptr;
    P.ticket = (unsigned long long *)L->ticket.ptr;
    P.P = (int *)L->part.ptr;
    P.done = (int *)L->done.ptr;
    P.busy = (int *)L->busy.ptr;
    P.njobs = 1 + (int64_t)nblocks * (nblocks - 1) / 2;
    P.tag = L->tag;
    P.nblocks = nblocks;
    P.err = ctx->err_ptr();
    P.wait_limit_ns = ctx->wait_limit_ns;
    P.stall_block = ctx->test_stall;
    int per_sm = 0;
    e = cudaFuncSetAttribute(k_lws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLwsWeightBytes);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lws, kLwsBlock, kLwsWeightBytes);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "lws occupancy");
    const int grid = (int)std::min<int64_t>(P.njobs, (int64_t)ctx->sms * std::max(per_sm, 1));
    cudaEventRecord(ctx->ev0, st);
    k_lws<<<grid, kLwsBlock, kLwsWeightBytes, st>>>(P);
    e = cudaGetLastError();
    cudaEventRecord(ctx->ev1, st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "k_lws");
    ctx->timed = true;
    ctx->timed_name = "k_lws";
    return PACO_OK;
}
