// Host driver of the single-pair path: plan lookup, scratch sizing, and the
// launch sequence  boundary bits -> strip pipeline -> boundary prefixes.
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
    if (ctx->plans.size() > 256) {
        cudaDeviceSynchronize();
        for (auto &kv : ctx->plans)
            if (kv.second->d_row0.ptr) cudaFree(kv.second->d_row0.ptr);
        ctx->plans.clear();
    }
    PairPlanOptions o;
    o.chunk = ctx->opt_chunk;
    o.warps = ctx->opt_warps;
    o.orient = ctx->opt_orient;
    o.schedule = ctx->opt_schedule;
    o.wpl = ctx->opt_wpl;
    o.max_warps = pair_max_warps(o.wpl == 2 ? 2 : 1);
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
    const size_t bytes = cp->plan.row0.size() * sizeof(int64_t);
    cudaError_t e = cudaMalloc(&cp->d_row0.ptr, bytes);
    if (e == cudaSuccess)
        e = cudaMemcpy(cp->d_row0.ptr, cp->plan.row0.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (cp->d_row0.ptr) cudaFree(cp->d_row0.ptr);
        *rc = set_cuda_error(ctx, e, "upload plan");
        return nullptr;
    }
    cp->d_row0.bytes = bytes;
    const CachedPairPlan *res = cp.get();
    ctx->plans.emplace(key, std::move(cp));
    *rc = PACO_OK;
    return res;
}

int run_pair(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
             const int32_t *top, const int32_t *left, int32_t *bottom_row, int32_t *right_col,
             int32_t *len, cudaStream_t st) {
    if (ctx->opt_engine == 2) {
        std::snprintf(ctx->last_error, sizeof(ctx->last_error), "cell-wise engine: not in this build");
        return PACO_EINVAL;
    }
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
    // kernel view: rows = ka (bits), columns = kb; transposed when bits run along b
    const uint8_t *ka = pl.transpose ? b : a;
    const uint8_t *kb = pl.transpose ? a : b;
    const int32_t *ktop = pl.transpose ? left : top;   // S+1 values along the kernel's columns
    const int32_t *kleft = pl.transpose ? top : left;  // L+1 values along the kernel's rows
    int32_t *kbottom = pl.transpose ? right_col : bottom_row;
    int32_t *kright = pl.transpose ? bottom_row : right_col;

    const int64_t nwords = (S + 31) / 32;
    const int64_t hstride = (nwords + 1) & ~(int64_t)1;
    const int64_t lwords = (L + 31) / 32;
    const int64_t rwords = (L + 30) / 31;
    const int64_t maxbits = std::max(L, S);
    const int64_t nblocks = ((maxbits + 30) / 31 + 1023) / 1024 + 1;
    if ((rc = ensure_bytes(ctx, ctx->hbuf, (size_t)(pl.nstrips + 1) * hstride * 8 + 16)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, ctx->lbits, (size_t)lwords * 4 + 16)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, ctx->rbits, (size_t)rwords * 4 + 16)) != PACO_OK) return rc;
    if ((rc = ensure_bytes(ctx, ctx->sums, (size_t)nblocks * 8 * 2)) != PACO_OK) return rc;

    const uint32_t epoch = next_epoch(ctx);
    uint64_t *hbuf = (uint64_t *)ctx->hbuf.ptr;
    e = launch_boundary_bits(kleft, L, (uint32_t *)ctx->lbits.ptr, nullptr, epoch, nullptr,
                             ctx->err_ptr(), st);
    if (e == cudaSuccess)
        e = launch_boundary_bits(ktop, S, nullptr, hbuf, epoch, kleft, ctx->err_ptr(), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ticket_ptr(), 0, sizeof(int), st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "prepare boundaries");

    PairArgs P;
    P.a = ka;
    P.b = kb;
    P.L = L;
    P.S = S;
    P.nwords = nwords;
    P.hstride = hstride;
    P.strip_row0 = (const int64_t *)cp->d_row0.ptr;
    P.granules = 0;
    P.nstrips = pl.nstrips;
    P.sigma = kMaxSigma;
    P.left_bits = (const uint32_t *)ctx->lbits.ptr;
    P.right_bits = (uint32_t *)ctx->rbits.ptr;
    P.hbuf = hbuf;
    P.ticket = ctx->ticket_ptr();
    P.err = ctx->err_ptr();
    P.epoch = epoch;
    P.wait_limit_ns = ctx->wait_limit_ns;
    P.stall_strip = ctx->test_stall;
    cudaEventRecord(ctx->ev0, st);
    e = launch_pair_bp(P, pl.C, pl.W, pl.wpl, pl.grid, st);
    cudaEventRecord(ctx->ev1, st);
    ctx->timed = true;
    ctx->timed_name = "k_pair_bp";
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "strip pipeline launch");

    PrefixScratch scr{(int64_t *)ctx->sums.ptr, nblocks};
    // kernel bottom row: the last strip's carries (tagged row nstrips), base H[L][0] = kleft[L]
    e = launch_bits_prefix(nullptr, hbuf + (size_t)pl.nstrips * hstride, S, 32, kleft, L, kbottom,
                           len, scr, st);
    if (e == cudaSuccess && kright != nullptr) {
        PrefixScratch scr2{(int64_t *)ctx->sums.ptr + nblocks, nblocks};
        // kernel right column: vertical steps of the last column, base H[0][S] = ktop[S]
        e = launch_bits_prefix((const uint32_t *)ctx->rbits.ptr, nullptr, L, 31, ktop, S, kright,
                               nullptr, scr2, st);
    }
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "boundary prefixes");
    return PACO_OK;
}

}  // namespace paco
