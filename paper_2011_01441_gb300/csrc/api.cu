// C ABI of the LCS library (include/paco_lcs.h): context, argument checks,
// the single-pair planner and launches, and measurement helpers.
#include "../../include/paco_lcs.h"
#include "paco_internal.hpp"
#include "plan.hpp"
#include "ctx.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace paco;

namespace paco {

int set_cuda_error(paco_ctx *ctx, cudaError_t e, const char *where) {
    if (e == cudaSuccess) return PACO_OK;
    if (ctx) {
        std::snprintf(ctx->last_error, sizeof(ctx->last_error), "%s: %s", where, cudaGetErrorString(e));
    }
    return e == cudaErrorMemoryAllocation ? PACO_ENOMEM : PACO_EDEVICE;
}

int ensure_bytes(paco_ctx *ctx, DevBuf &buf, size_t bytes) {
    if (buf.bytes >= bytes) return PACO_OK;
    if (buf.ptr) {
        // the previous owner may still be in use by enqueued work
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "sync before regrow");
        cudaFree(buf.ptr);
        buf.ptr = nullptr;
        buf.bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)4096);
    want = (want + 4095) / 4096 * 4096;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaMalloc scratch");
    e = cudaMemset(p, 0, want);
    if (e != cudaSuccess) {
        cudaFree(p);
        return set_cuda_error(ctx, e, "cudaMemset scratch");
    }
    buf.ptr = p;
    buf.bytes = want;
    return PACO_OK;
}

uint32_t next_epoch(paco_ctx *ctx) {
    ctx->epoch += 1;
    if (ctx->epoch == 0 || ctx->epoch == 0x80000000u) ctx->epoch += 1;
    return ctx->epoch;
}

}  // namespace paco

static bool bad_len(int64_t x) { return x < 0 || x > 0x7fffffffLL; }

extern "C" {

const char *paco_strerror(int status) {
    switch (status) {
        case PACO_OK: return "ok";
        case PACO_PENDING: return "pending";
        case PACO_EINVAL: return "invalid argument";
        case PACO_ENOMEM: return "out of memory";
        case PACO_ETIMEOUT: return "device wait timed out";
        case PACO_EDEVICE: return "CUDA error";
        case PACO_EBUSY: return "busy";
        case PACO_ENOTFOUND: return "unknown ticket";
        default: return "unknown status";
    }
}

const char *paco_last_error(paco_ctx *ctx) { return ctx ? ctx->last_error : "no context"; }

int paco_ctx_create(int device, size_t mem_budget_bytes, paco_ctx **out) {
    if (!out) return PACO_EINVAL;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return set_cuda_error(nullptr, e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return PACO_EINVAL;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return set_cuda_error(nullptr, e, "cudaSetDevice");
    paco_ctx *ctx = new (std::nothrow) paco_ctx();
    if (!ctx) return PACO_ENOMEM;
    ctx->device = device;
    ctx->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)8 << 30;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete ctx;
        return set_cuda_error(nullptr, e, "cudaGetDeviceProperties");
    }
    ctx->sms = prop.multiProcessorCount;
    int rc = ensure_bytes(ctx, ctx->small, 65536);
    if (rc != PACO_OK) {
        delete ctx;
        return rc;
    }
    e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        paco_ctx_destroy(ctx);
        return set_cuda_error(nullptr, e, "ctx events/stream");
    }
    *out = ctx;
    return PACO_OK;
}

void paco_ctx_destroy(paco_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    serve_shutdown(ctx);
    cudaDeviceSynchronize();
    batch_release(ctx);
    affine_state_free(ctx->affine);
    ctx->affine = nullptr;
    lws_state_free(ctx->lws);
    ctx->lws = nullptr;
    for (DevBuf *b : {&ctx->small, &ctx->hbuf,
                      &ctx->h_a, &ctx->h_b, &ctx->h_top, &ctx->h_left, &ctx->h_row, &ctx->h_col,
                      &ctx->h_len}) {
        if (b->ptr) cudaFree(b->ptr);
        b->ptr = nullptr;
    }
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

int paco_ctx_set_option(paco_ctx *ctx, int option, int64_t value) {
    if (!ctx) return PACO_EINVAL;
    switch (option) {
        case PACO_OPT_ENGINE:
            if (value < 0 || value > 1) return PACO_EINVAL;
            ctx->opt_engine = (int)value;
            return PACO_OK;
        case PACO_OPT_CHUNK:
            if (!(value == 0 || value == 2 || value == 4 || value == 8))
                return PACO_EINVAL;
            ctx->opt_chunk = (int)value;
            return PACO_OK;
        case PACO_OPT_WARPS:  // the planner clamps to what fits in shared memory
            if (value < 0 || value > 7) return PACO_EINVAL;
            ctx->opt_warps = (int)value;
            return PACO_OK;
        case PACO_OPT_WAIT_LIMIT_NS:
            if (value < 1000 || value > 600LL * 1000000000LL) return PACO_EINVAL;
            ctx->wait_limit_ns = value;
            return PACO_OK;
        case PACO_OPT_ORIENT:
            if (value < 0 || value > 2) return PACO_EINVAL;
            ctx->opt_orient = (int)value;
            return PACO_OK;
        case PACO_OPT_SCHEDULE:
            if (value < 0 || value > 1) return PACO_EINVAL;
            ctx->opt_schedule = (int)value;
            return PACO_OK;
        case PACO_OPT_ALPHABET:
            if (value < 1 || value > 256) return PACO_EINVAL;
            ctx->opt_alphabet = (int)value;
            return PACO_OK;
        case PACO_OPT_WORDS_PER_LANE:
            if (value < 0 || value > 2) return PACO_EINVAL;
            ctx->opt_wpl = (int)value;
            return PACO_OK;
        case PACO_OPT_TILES:
            if (value < 0 || value > 3) return PACO_EINVAL;
            ctx->opt_tiles = (int)value;
            return PACO_OK;
        case PACO_OPT_TILE_BASE:
            if (value < 0 || value > (1 << 20)) return PACO_EINVAL;
            ctx->opt_tile_base = value;
            return PACO_OK;
        case PACO_OPT_AFFINE_ROWS:
            if (!(value == 0 || value == 2 || value == 4 || value == 8)) return PACO_EINVAL;
            ctx->opt_affine_rows = (int)value;
            return PACO_OK;
        case PACO_OPT_SERVE_CHUNKS:
            if (value != 0) {
                for (int k = 0; k < 4; ++k) {
                    const int64_t c = (value >> (4 * k)) & 15;
                    if (!(c == 2 || c == 4 || c == 8)) return PACO_EINVAL;
                }
                if (value >> 16) return PACO_EINVAL;
            }
            ctx->opt_serve_chunks = (int)value;
            return PACO_OK;
        case PACO_OPT_TEST_STALL:
            if (value < -1 || value > 0x7fffffff) return PACO_EINVAL;
            ctx->test_stall = (int)value;
            return PACO_OK;
        default:
            return PACO_EINVAL;
    }
}

int paco_ctx_get_option(paco_ctx *ctx, int option, int64_t *value) {
    if (!ctx || !value) return PACO_EINVAL;
    switch (option) {
        case PACO_OPT_ENGINE: *value = ctx->opt_engine; return PACO_OK;
        case PACO_OPT_CHUNK: *value = ctx->opt_chunk; return PACO_OK;
        case PACO_OPT_WARPS: *value = ctx->opt_warps; return PACO_OK;
        case PACO_OPT_WAIT_LIMIT_NS: *value = ctx->wait_limit_ns; return PACO_OK;
        case PACO_OPT_ORIENT: *value = ctx->opt_orient; return PACO_OK;
        case PACO_OPT_SCHEDULE: *value = ctx->opt_schedule; return PACO_OK;
        case PACO_OPT_ALPHABET: *value = ctx->opt_alphabet; return PACO_OK;
        case PACO_OPT_WORDS_PER_LANE: *value = ctx->opt_wpl; return PACO_OK;
        case PACO_OPT_TILES: *value = ctx->opt_tiles; return PACO_OK;
        case PACO_OPT_TILE_BASE: *value = ctx->opt_tile_base; return PACO_OK;
        case PACO_OPT_BATCH_CHUNKS: *value = ctx->last_batch_chunk; return PACO_OK;
        case PACO_OPT_AFFINE_ROWS: *value = ctx->opt_affine_rows; return PACO_OK;
        case PACO_OPT_SERVE_CHUNKS: *value = ctx->opt_serve_chunks; return PACO_OK;
        case PACO_OPT_TEST_STALL: *value = ctx->test_stall; return PACO_OK;
        default: return PACO_EINVAL;
    }
}

int paco_ctx_sync(paco_ctx *ctx, void *stream) {
    if (!ctx) return PACO_EINVAL;
    cudaSetDevice(ctx->device);
    cudaError_t e;
    if (stream) e = cudaStreamSynchronize((cudaStream_t)stream);
    else e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "sync");
    int err = 0;
    e = cudaMemcpy(&err, ctx->err_ptr(), sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "read error word");
    if (err != 0) {
        e = cudaMemset(ctx->err_ptr(), 0, sizeof(int));
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "clear error word");
        return err;
    }
    return PACO_OK;
}

int paco_lcs_boundaries(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                        const int32_t *d_top_in, const int32_t *d_left_in, int32_t *d_bottom_row,
                        int32_t *d_right_col, int32_t *d_len, void *stream) {
    if (!ctx || bad_len(n) || bad_len(m)) return PACO_EINVAL;
    if ((n > 0 && !a) || (m > 0 && !b)) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    return run_pair(ctx, a, n, b, m, d_top_in, d_left_in, d_bottom_row, d_right_col, d_len,
                    (cudaStream_t)stream);
}

int paco_lcs_length(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                    int32_t *d_len, void *stream) {
    if (!d_len) return PACO_EINVAL;
    return paco_lcs_boundaries(ctx, a, n, b, m, nullptr, nullptr, nullptr, nullptr, d_len, stream);
}

int paco_lcs_boundaries_host(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                             const int32_t *top_in, const int32_t *left_in, int32_t *bottom_row,
                             int32_t *right_col, int32_t *len, void *stream) {
    if (!ctx || bad_len(n) || bad_len(m)) return PACO_EINVAL;
    if ((n > 0 && !a) || (m > 0 && !b)) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->own_stream;
    int rc;
    if ((rc = ensure_bytes(ctx, ctx->h_a, (size_t)n + 16)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, ctx->h_b, (size_t)m + 16)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, ctx->h_row, ((size_t)m + 1) * 4)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, ctx->h_col, ((size_t)n + 1) * 4)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, ctx->h_len, 16)) != PACO_OK) return rc;
    if (top_in && (rc = ensure_bytes(ctx, ctx->h_top, ((size_t)m + 1) * 4)) != PACO_OK) return rc;
    if (left_in && (rc = ensure_bytes(ctx, ctx->h_left, ((size_t)n + 1) * 4)) != PACO_OK) return rc;
    cudaError_t e = cudaSuccess;
    if (n) e = cudaMemcpyAsync(ctx->h_a.ptr, a, (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(ctx->h_b.ptr, b, (size_t)m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && top_in)
        e = cudaMemcpyAsync(ctx->h_top.ptr, top_in, ((size_t)m + 1) * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && left_in)
        e = cudaMemcpyAsync(ctx->h_left.ptr, left_in, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "host inputs to device");
    rc = run_pair(ctx, (const uint8_t *)ctx->h_a.ptr, n, (const uint8_t *)ctx->h_b.ptr, m,
                  top_in ? (const int32_t *)ctx->h_top.ptr : nullptr,
                  left_in ? (const int32_t *)ctx->h_left.ptr : nullptr,
                  bottom_row ? (int32_t *)ctx->h_row.ptr : nullptr,
                  right_col ? (int32_t *)ctx->h_col.ptr : nullptr, (int32_t *)ctx->h_len.ptr, st);
    if (rc != PACO_OK) return rc;
    if (bottom_row)
        e = cudaMemcpyAsync(bottom_row, ctx->h_row.ptr, ((size_t)m + 1) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && right_col)
        e = cudaMemcpyAsync(right_col, ctx->h_col.ptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost, st);
    int32_t hl = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hl, ctx->h_len.ptr, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "device outputs to host");
    if (len) *len = hl;
    int err = 0;
    e = cudaMemcpy(&err, ctx->err_ptr(), sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "read error word");
    if (err != 0) {
        cudaMemset(ctx->err_ptr(), 0, sizeof(int));
        return err;
    }
    return PACO_OK;
}

int paco_measure_int_peak(paco_ctx *ctx, int op, double *ops_per_s, void *stream) {
    if (!ctx || !ops_per_s || op < 0 || op > 3) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->own_stream;
    const int block = 256, per_sm = 8, iters = 1 << 14;
    const int grid = ctx->sms * per_sm;
    uint32_t *sink = ctx->sink_ptr();
    cudaError_t e = launch_int_peak(op, grid, block, 64, sink, st);  // warm-up
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "int peak warm-up");
    cudaEventRecord(ctx->ev0, st);
    e = launch_int_peak(op, grid, block, iters, sink, st);
    cudaEventRecord(ctx->ev1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev1);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "int peak");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    // lane-ops per chain step: op 0: 1 three-input add; op 1: 1 three-input
    // logic op (and/xor/or fuse to one); op 2: 1 add + 1 max; op 3: the
    // column step, 4 lane-ops (or, and, andnot, add-with-carry).
    const double per_step[4] = {1.0, 1.0, 2.0, 4.0};
    const double ops = (double)grid * block * 8.0 * iters * per_step[op];
    *ops_per_s = ops / (ms * 1e-3);
    return PACO_OK;
}

int paco_last_kernel_ms(paco_ctx *ctx, double *ms, const char **name) {
    if (!ctx || !ms) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->timed) return PACO_EINVAL;
    cudaError_t e = cudaEventSynchronize(ctx->ev1);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "event sync");
    float f = 0.f;
    e = cudaEventElapsedTime(&f, ctx->ev0, ctx->ev1);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "event elapsed");
    *ms = f;
    if (name) *name = ctx->timed_name;
    return PACO_OK;
}

}  // extern "C"
