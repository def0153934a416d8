// The 1D problem of Sec. "PACO 1D" (least weight subsequence, Eq. 1D):
// D[j] = min_{i<j} D[i] + w(i, j).  Block kernel, host launch and the C ABI
// of include/paco_lws.h.
//
// Layout.  The outputs are cut into blocks of kLwsBlock consecutive j; one
// CTA of kLwsBlock threads owns one block (thread t <-> j = block start + t,
// its running minimum in a register).  The work of the recurrence is the
// triangle {(i, j): i < j}; the CTA of block b walks its column of that
// triangle from the left: for every earlier block a it waits for a's flag,
// stages a's finished D in shared memory and folds min_i D[i] + w(i, j) into
// its minima (the square (a, b) of the paper's quadrant structure), then
// solves its own diagonal triangle in sub-blocks of 32: warp s finishes its
// 32 values by a sequential sweep over its lanes (a shuffle per value), and
// the later warps fold those 32 values in before their own turn.  Finished
// blocks publish D and set a flag with release semantics.  Blocks are taken
// from an atomic ticket, so a CTA only ever waits for a block held by a
// running CTA; every wait is bounded.
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
constexpr int kLwsInf = 0x3fffffff;       // above every D (D < 2^29 + 2^24 + 256 by the argument checks)

struct LwsArgs {
    int64_t n;
    int d0;
    int T;
    uint32_t seed;
    uint32_t noise_mask;   // 255 or 0
    int32_t *D;            // n + 1 outputs
    int *flags;            // [0] ticket, [1 + b] block b finished (this launch's tag)
    int tag;               // nonzero tag of this launch
    int nblocks;
    int *err;
    long long wait_limit_ns;
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

static __device__ __forceinline__ int ld_acquire_flag(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits (bounded) for a block's flag `f` to carry `tag`; the
// result is CTA-uniform (scalar arguments keep the caller's state in
// registers).
static __device__ __noinline__ bool wait_block(const int *f, int tag, int *err, long long limit, int *s_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire_flag(f) != tag) {
            const uint64_t t0 = dev::global_ns();
            for (int spin = 0;; ++spin) {
                if (spin > 8) __nanosleep(64);
                if (ld_acquire_flag(f) == tag) break;
                if (dev::ld_relaxed_i32(err) != 0) {
                    ok = 0;
                    break;
                }
                if ((long long)(dev::global_ns() - t0) > limit) {
                    dev::raise_error(err, kEtimeout);
                    ok = 0;
                    break;
                }
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__global__ void __launch_bounds__(kLwsBlock) k_lws(LwsArgs P) {
    __shared__ int s_D[kLwsBlock];
    __shared__ int s_ticket, s_ok;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    for (;;) {
        if (t == 0) s_ticket = atomicAdd(P.flags, 1);
        __syncthreads();
        const int b = s_ticket;
        __syncthreads();
        if (b >= P.nblocks) return;
        const int64_t j64 = (int64_t)b * kLwsBlock + t;
        const int j = (int)j64;
        const int jt = j - P.T;
        const uint32_t js = (uint32_t)j ^ P.seed;
        int best = j == 0 ? P.d0 : kLwsInf;

        // squares (a, b) for every earlier block a
        for (int a = 0; a < b; ++a) {
            if (!wait_block(P.flags + 1 + a, P.tag, P.err, P.wait_limit_ns, &s_ok)) return;
            s_D[t] = P.D[(int64_t)a * kLwsBlock + t];   // blocks below b are full (a < b <= last)
            __syncthreads();
            const int i0 = a * kLwsBlock;
#pragma unroll 8
            for (int k = 0; k < kLwsBlock; ++k) best = min(best, s_D[k] + lws_w(i0 + k, jt, js, P.noise_mask));
            __syncthreads();
        }

        // the diagonal triangle of block b, 32 values at a time
        const int i0 = b * kLwsBlock;
        for (int s = 0; s < kLwsWarps; ++s) {
            if (warp == s) {
                // sequential sweep: lane k's minimum is final once lanes < k are folded in
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const int dk = __shfl_sync(dev::kFull, best, k);
                    if (lane > k) best = min(best, dk + lws_w(i0 + 32 * s + k, jt, js, P.noise_mask));
                }
                s_D[t] = best;
                if (j64 <= P.n) P.D[j64] = best;
            }
            __syncthreads();
            if (warp > s) {
                const int ib = i0 + 32 * s;
#pragma unroll 8
                for (int k = 0; k < 32; ++k) best = min(best, s_D[32 * s + k] + lws_w(ib + k, jt, js, P.noise_mask));
            }
        }
        // publish: every thread's store is ordered before the flag by the
        // CTA barrier and thread 0's release fence
        __syncthreads();
        if (t == 0) {
            __threadfence();
            asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(P.flags + 1 + b), "r"(P.tag) : "memory");
        }
    }
}

}  // namespace

// Scratch of the 1D path, owned by the context.
struct LwsState {
    DevBuf flags;
    int tag = 0;   // tag of the last launch (0: none yet)
};

void lws_state_free(LwsState *L) {
    if (!L) return;
    if (L->flags.ptr) cudaFree(L->flags.ptr);
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
    int rc = ensure_bytes(ctx, L->flags, ((size_t)nblocks + 1) * sizeof(int));
    if (rc != PACO_OK) return rc;
    // a new tag per launch; flags of older launches never match it (the
    // buffer is cleared when the tag wraps, and zeroed when it grows)
    L->tag = L->tag >= (1 << 30) ? 1 : L->tag + 1;
    cudaError_t e = cudaSuccess;
    if (L->tag == 1) e = cudaMemsetAsync(L->flags.ptr, 0, L->flags.bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->flags.ptr, 0, sizeof(int), st);  // ticket
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "lws set-up");
    LwsArgs P{};
    P.n = n;
    P.d0 = d0;
    P.T = w->T;
    P.seed = w->seed;
    P.noise_mask = w->noise ? 255u : 0u;
    P.D = d_D;
    P.flags = (int *)L->flags.ptr;
    P.tag = L->tag;
    P.nblocks = nblocks;
    P.err = ctx->err_ptr();
    P.wait_limit_ns = ctx->wait_limit_ns;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lws, kLwsBlock, 0);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "lws occupancy");
    const int grid = std::min(nblocks, ctx->sms * std::max(per_sm, 1));
    cudaEventRecord(ctx->ev0, st);
    k_lws<<<grid, kLwsBlock, 0, st>>>(P);
    e = cudaGetLastError();
    cudaEventRecord(ctx->ev1, st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "k_lws");
    ctx->timed = true;
    ctx->timed_name = "k_lws";
    return PACO_OK;
}
