// C ABI of the planner (include/paco_plan.h); host only.
#include "../../include/paco_plan.h"
#include "plan.hpp"

#include <vector>

extern "C" {

int paco_plan_partition(int64_t n, int64_t m, int32_t p, int64_t base, paco_tile *out, int64_t cap,
                        int64_t *count) {
    std::vector<paco::Tile> tiles;
    if (!paco::paco_partition(n, m, p, base, tiles)) return -1;
    if (count) *count = (int64_t)tiles.size();
    if (out) {
        const int64_t k = (int64_t)tiles.size() < cap ? (int64_t)tiles.size() : cap;
        for (int64_t i = 0; i < k; ++i) {
            const paco::Tile &t = tiles[(size_t)i];
            out[i].r0 = t.r0;
            out[i].r1 = t.r1;
            out[i].c0 = t.c0;
            out[i].c1 = t.c1;
            out[i].label = t.label;
            out[i].owner = t.owner;
            out[i].order = t.order;
        }
    }
    return 0;
}

int paco_plan_partition_deps(int64_t n, int64_t m, int32_t p, int64_t base, int64_t *dep_off,
                             int64_t *dep_idx, int64_t cap_idx, int64_t *n_idx) {
    std::vector<paco::Tile> tiles;
    if (!paco::paco_partition(n, m, p, base, tiles)) return -1;
    std::vector<std::vector<int64_t>> deps;
    paco::tile_deps(tiles, deps);
    int64_t pos = 0;
    for (size_t k = 0; k < tiles.size(); ++k) {
        if (dep_off) dep_off[k] = pos;
        for (int64_t d : deps[k]) {
            if (dep_idx && pos < cap_idx) dep_idx[pos] = d;
            ++pos;
        }
    }
    if (dep_off) dep_off[tiles.size()] = pos;
    if (n_idx) *n_idx = pos;
    return 0;
}

int paco_plan_pair(int64_t n, int64_t m, int32_t sms, int32_t chunk, int32_t warps, int32_t orient,
                   int32_t schedule, int32_t words_per_lane, paco_pair_plan *out, int64_t *row0,
                   int64_t cap) {
    if (!out) return -1;
    paco::PairPlanOptions o;
    o.chunk = chunk;
    o.warps = warps;
    o.orient = orient;
    o.schedule = schedule;
    o.wpl = words_per_lane;
    paco::PairPlan pl;
    if (!paco::plan_pair(n, m, sms, o, pl)) return -1;
    out->transpose = pl.transpose ? 1 : 0;
    out->chunk = pl.C;
    out->warps = pl.W;
    out->nstrips = pl.nstrips;
    out->words_per_lane = pl.wpl;
    out->pad = 0;
    out->L = pl.L;
    out->S = pl.S;
    if (row0)
        for (size_t k = 0; k < pl.row0.size() && (int64_t)k < cap; ++k) row0[k] = pl.row0[k];
    return 0;
}

int paco_plan_tiles(int64_t n, int64_t m, int32_t p, int32_t kind, int64_t base, paco_tile *out,
                    int64_t cap, int64_t *count, int64_t *dep_off, int64_t *dep_idx, int64_t cap_idx,
                    int64_t *n_idx, int64_t *critical_cells) {
    paco::TilePlan tp;
    if (!paco::plan_tiles(n, m, p, kind, base, tp)) return -1;
    const int64_t T = (int64_t)tp.tiles.size();
    if (count) *count = T;
    if (n_idx) *n_idx = (int64_t)tp.dep_idx.size();
    if (critical_cells) *critical_cells = tp.critical_cells;
    for (int64_t k = 0; out && k < T && k < cap; ++k) {
        const paco::Tile &t = tp.tiles[(size_t)k];
        out[k].r0 = t.r0;
        out[k].r1 = t.r1;
        out[k].c0 = t.c0;
        out[k].c1 = t.c1;
        out[k].label = 0;
        out[k].owner = 0;
        out[k].order = k;
    }
    if (dep_off && cap >= T)
        for (int64_t k = 0; k <= T; ++k) dep_off[k] = tp.dep_off[(size_t)k];
    for (int64_t k = 0; dep_idx && k < (int64_t)tp.dep_idx.size() && k < cap_idx; ++k)
        dep_idx[k] = tp.dep_idx[(size_t)k];
    return 0;
}

int paco_plan_shard(const int64_t *a_off, const int64_t *b_off, int64_t npairs, int32_t ranks, int32_t *owner,
                    int64_t *rank_cells) {
    if (npairs > 0 && !owner) return -1;
    std::vector<int32_t> own;
    std::vector<int64_t> rc;
    if (!paco::plan_shard(a_off, b_off, npairs, ranks, own, rc)) return -1;
    for (int64_t k = 0; k < npairs; ++k) owner[k] = own[(size_t)k];
    if (rank_cells)
        for (int32_t r = 0; r < ranks; ++r) rank_cells[r] = rc[(size_t)r];
    return 0;
}

}  // extern "C"
