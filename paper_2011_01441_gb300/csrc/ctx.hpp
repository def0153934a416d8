// The context object behind the opaque paco_ctx handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "plan.hpp"

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

namespace paco {
struct BatchState;
struct ServeEngine;
struct TileState;
struct AffineState;
struct LwsState;

// A pair plan (the strips' rows are computed in the kernel from its counts).
struct CachedPairPlan {
    PairPlan plan;
};
}  // namespace paco

struct paco_ctx {
    int device = 0;
    int sms = 0;
    size_t budget = 0;
    std::mutex mu;
    // small: [0] error word, [1] batch ticket, [4..5] the pair kernel's strip ticket and exit
    // count (zero between launches), sink from byte 1024
    DevBuf small;
    // single-pair scratch: the strips' tagged carry rows
    DevBuf hbuf;
    // staging for the host-buffer entry point
    DevBuf h_a, h_b, h_top, h_left, h_row, h_col, h_len;
    uint32_t epoch = 0;
    int opt_engine = 0, opt_chunk = 0, opt_warps = 0, opt_orient = 0, opt_schedule = 0, opt_wpl = 0;
    int opt_tiles = 0;            // single pair: 0 = strip pipeline, 1..3 = tile schedule (PACO, PA, PO)
    int64_t opt_tile_base = 0;    // tile schedules: smallest tile side in granules (0 = per schedule)
    int opt_affine_rows = 0;      // affine alignment: rows per lane, 4 or 8 (0 = 4)
    int opt_serve_chunks = 0;     // serving micro-batches: packed chunk width per size class (0 = defaults)
    int test_stall = -1;
    int opt_alphabet = 256;
    long long wait_limit_ns = 2000000000LL;
    char last_error[256] = {0};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
    int last_batch_chunk = 0;
    const char *timed_name = "";
    cudaStream_t own_stream = nullptr;
    std::map<std::tuple<int64_t, int64_t, int, int, int, int>, std::unique_ptr<paco::CachedPairPlan>> plans;
    paco::BatchState *batch = nullptr;
    paco::BatchState *recover = nullptr;  // the subsequence recovery's batch engine state
    paco::TileState *tiles = nullptr;     // tile schedules: layouts and buffers
    paco::AffineState *affine = nullptr;  // affine alignment: band plans and buffers
    paco::LwsState *lws = nullptr;        // 1D problem: block flags
    paco::ServeEngine *serve = nullptr;

    int *err_ptr() { return (int *)small.ptr; }
    int *ticket_ptr() { return (int *)small.ptr + 1; }
    int *pair_ctl_ptr() { return (int *)small.ptr + 4; }
    uint32_t *sink_ptr() { return (uint32_t *)((char *)small.ptr + 1024); }
};

namespace paco {
int set_cuda_error(paco_ctx *ctx, cudaError_t e, const char *where);
int ensure_bytes(paco_ctx *ctx, DevBuf &buf, size_t bytes);
uint32_t next_epoch(paco_ctx *ctx);
// Enqueue one pair (device pointers) on `st`; ctx->mu must be held.
int run_pair(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
             const int32_t *top, const int32_t *left, int32_t *bottom_row, int32_t *right_col,
             int32_t *len, cudaStream_t st);
const CachedPairPlan *get_pair_plan(paco_ctx *ctx, int64_t n, int64_t m, int *rc);
// Enqueue a batch (device strings, host offsets); ctx->mu must be held.
BatchState *batch_state_new(int *ticket, int *err);
void batch_state_free(BatchState *B);
int run_batch(paco_ctx *ctx, BatchState *B, const uint8_t *a_cat, const int64_t *h_a_off, const uint8_t *b_cat,
              const int64_t *h_b_off, int32_t npairs, int32_t *d_len, int32_t *rows_cat,
              const int64_t *h_row_off, int32_t *cols_cat, const int64_t *h_col_off, cudaStream_t st,
              bool use_graph, int force_chunk, int sigma);
void serve_shutdown(paco_ctx *ctx);
// A tile schedule (ctx->opt_tiles) of one pair with zero boundaries.
int run_tiles(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, int32_t *bottom_row,
              int32_t *right_col, int32_t *len, cudaStream_t st);
void tile_state_free(TileState *T);
void affine_state_free(AffineState *A);
void lws_state_free(LwsState *L);
void batch_release(paco_ctx *ctx);
}  // namespace paco
