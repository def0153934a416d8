// Host driver of the single-pair path: plan lookup, scratch sizing and the
// one launch of the strip pipeline (which also converts the boundaries and
// writes L, the last row and the last column).
#include "../../include/paco_lcs.h"
#include "ctx.hpp"
#include "paco_internal.hpp"

#include <algorithm>
#include <cstdio>

namespace paco {

const CachedPairPlan *get_pair_plan(paco_ctx *ctx, int64_t n, int64_t m, int *rc) {
    const auto key = std::make_tuple(n, m, ctx->opt_chunk, ctx->opt_warps, ctx->opt_orient,
                                     ctx->opt_schedule * 4 + ctx->opt_wpl);
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        *rc = PACO_OK;
        return it->second.get();
    }
    if (ctx->plans.size() > 256) ctx->plans.clear();  // host memory only
    PairPlanOptions o;
    o.chunk = ctx->opt_chunk;
    o.warps = ctx->opt_warps;
    o.orient = ctx->opt_orient;
    o.schedule = ctx->opt_schedule;
    o.wpl = ctx->opt_wpl;
    o.max_warps = pair_max_warps(1);
    o.max_warps_wpl2 = pair_max_warps(2);
    auto cp = std::make_unique<CachedPairPlan>();
    // resident CTAs for the chosen chunk width; plan once to learn C and W
    if (!plan_pair(n, m, ctx->sms, o, cp->plan)) {
        *rc = PACO_EINVAL;
        return nullptr;
    }
    o.resident = ctx->sms * std::max(1, pair_occupancy(cp->plan.C, cp->plan.W, cp->plan.wpl));
    if (!plan_pair(n, m, ctx->sms, o, cp->plan)) {
        *rc = PACO_EINVAL;
        return nullptr;
    }
    // the planner may have raised W; the grid must fit what is resident
    const int occ = std::max(1, pair_occupancy(cp->plan.C, cp->plan.W, cp->plan.wpl));
    cp->plan.grid = std::min(cp->plan.nstrips, ctx->sms * occ);
    const CachedPairPlan *res = cp.get();
    ctx->plans.emplace(key, std::move(cp));
    *rc = PACO_OK;
    return res;
}

int run_pair(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
             const int32_t *top, const int32_t *left, int32_t *bottom_row, int32_t *right_col,
             int32_t *len, cudaStream_t st) {
    cudaError_t e;
    if (n == 0 || m == 0) {
        e = launch_degenerate(top, left, n, m, bottom_row, right_col, len, ctx->err_ptr(), st);
        ctx->timed = false;
        return set_cuda_error(ctx, e, "degenerate table");
    }
    if (ctx->opt_tiles) {  // a tile schedule instead of the strip pipeline
        if (top || left) {
            std::snprintf(ctx->last_error, sizeof(ctx->last_error), "tile schedules take zero boundaries only");
            return PACO_EINVAL;
        }
        return run_tiles(ctx, a, n, b, m, bottom_row, right_col, len, st);
    }
    int rc = PACO_OK;
    const CachedPairPlan *cp = get_pair_plan(ctx, n, m, &rc);
    if (!cp) return rc;
    const PairPlan &pl = cp->plan;
    const int64_t L = pl.L, S = pl.S;
    const int64_t nwords = (S + 31) / 32;
    const int64_t hstride = (nwords + 1) & ~(int64_t)1;
    if ((rc = ensure_bytes(ctx, ctx->hbuf, (size_t)(pl.nstrips + 1) * hstride * 8 + 16)) != PACO_OK) return rc;

    PairArgs P;
    // kernel view: rows = a (bits), columns = b; transposed when bits run along b
    P.a = pl.transpose ? b : a;
    P.b = pl.transpose ? a : b;
    P.L = L;
    P.S = S;
    P.nwords = (int32_t)nwords;
    P.hstride = hstride;
    P.granules = (L + 31 * pl.wpl - 1) / (31 * pl.wpl);
    P.uniform_rows = ctx->opt_schedule == 1 ? (int64_t)pl.W * 32 * 31 * pl.wpl : 0;
    P.nstrips = pl.nstrips;
    P.top = pl.transpose ? left : top;   // S+1 values along the kernel's columns
    P.left = pl.transpose ? top : left;  // L+1 values along the kernel's rows
    P.bottom = pl.transpose ? right_col : bottom_row;
    P.right = pl.transpose ? bottom_row : right_col;
    P.len = len;
    P.hbuf = (uint64_t *)ctx->hbuf.ptr;
    P.ctl = ctx->pair_ctl_ptr();
    P.err = ctx->err_ptr();
    P.epoch = next_epoch(ctx);
    P.wait_limit_ns = ctx->wait_limit_ns;
    P.stall_strip = ctx->test_stall;
    cudaEventRecord(ctx->ev0, st);
    e = launch_pair_bp(P, pl.C, pl.W, pl.wpl, pl.grid, st);
    cudaEventRecord(ctx->ev1, st);
    ctx->timed = true;
    ctx->timed_name = "k_pair_bp";
    return set_cuda_error(ctx, e, "strip pipeline launch");
}

}  // namespace paco
