// Host-side planner (see plan.hpp).
#include "plan.hpp"

#include <algorithm>
#include <utility>
#include <cmath>
#include <map>
#include <queue>
#include <tuple>

namespace paco {

std::vector<int64_t> balanced_split(int64_t total, int64_t parts) {
    std::vector<int64_t> sizes;
    if (parts <= 0) return sizes;
    sizes.resize((size_t)parts, total / parts);
    for (int64_t k = 0; k < total % parts; ++k) sizes[(size_t)k] += 1;
    return sizes;
}

namespace {

struct Reg {
    int64_t r0, r1, c0, c1;
    int64_t gi, gj;  // grid index at the region's level
};

bool divisible(const Reg &r, int64_t base) {
    return (r.r1 - r.r0) >= 2 * base && (r.c1 - r.c0) >= 2 * base;
}

}  // namespace

bool paco_partition(int64_t n, int64_t m, int32_t p, int64_t base, std::vector<Tile> &tiles) {
    tiles.clear();
    if (n <= 0 || m <= 0 || p <= 0 || base <= 0) return false;
    // Step 1: the p-way division in both dimensions (balanced integer split).
    const int64_t pr = std::min<int64_t>(p, n), pc = std::min<int64_t>(p, m);
    const std::vector<int64_t> hs = balanced_split(n, pr), ws = balanced_split(m, pc);
    std::vector<Reg> un;
    un.reserve((size_t)(pr * pc));
    int64_t r = 0;
    for (int64_t i = 0; i < pr; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < pc; ++j) {
            un.push_back({r, r + hs[(size_t)i], c, c + ws[(size_t)j], i, j});
            c += ws[(size_t)j];
        }
        r += hs[(size_t)i];
    }
    int32_t label = 1;
    int64_t rr = 0;  // round-robin counter of base-case assignments
    while (!un.empty()) {
        // group by anti-diagonal of the level grid; within one, ascending column
        std::map<int64_t, std::vector<Reg>> diag;
        for (const Reg &x : un) diag[x.gi + x.gj].push_back(x);
        std::vector<Reg> left;
        bool assigned_any = false;
        for (auto &kv : diag) {
            std::vector<Reg> &v = kv.second;
            std::sort(v.begin(), v.end(), [](const Reg &a, const Reg &b) { return a.gj < b.gj; });
            size_t take = v.size() >= (size_t)p ? (size_t)p : 0;
            for (size_t k = 0; k < take; ++k)
                tiles.push_back({v[k].r0, v[k].r1, v[k].c0, v[k].c1, label, (int32_t)k, 0});
            if (take) assigned_any = true;
            for (size_t k = take; k < v.size(); ++k) left.push_back(v[k]);
        }
        // base-case regions (cannot be halved): all of them round-robin
        std::vector<Reg> next;
        bool base_assigned = false;
        std::sort(left.begin(), left.end(), [](const Reg &a, const Reg &b) {
            return std::make_tuple(a.gi + a.gj, a.gj) < std::make_tuple(b.gi + b.gj, b.gj);
        });
        for (const Reg &x : left) {
            if (!divisible(x, base)) {
                tiles.push_back({x.r0, x.r1, x.c0, x.c1, label, (int32_t)(rr % p), 0});
                ++rr;
                base_assigned = true;
            } else {
                const int64_t hm = x.r0 + (x.r1 - x.r0) / 2, wm = x.c0 + (x.c1 - x.c0) / 2;
                next.push_back({x.r0, hm, x.c0, wm, 2 * x.gi, 2 * x.gj});
                next.push_back({x.r0, hm, wm, x.c1, 2 * x.gi, 2 * x.gj + 1});
                next.push_back({hm, x.r1, x.c0, wm, 2 * x.gi + 1, 2 * x.gj});
                next.push_back({hm, x.r1, wm, x.c1, 2 * x.gi + 1, 2 * x.gj + 1});
            }
        }
        if (assigned_any || base_assigned) ++label;
        un.swap(next);
    }
    // time line: Kahn's algorithm over the region DAG, earliest anti-diagonal first
    std::vector<std::vector<int64_t>> deps;
    tile_deps(tiles, deps);
    const size_t T = tiles.size();
    std::vector<std::vector<int64_t>> succ(T);
    std::vector<int64_t> indeg(T, 0);
    for (size_t k = 0; k < T; ++k) {
        indeg[k] = (int64_t)deps[k].size();
        for (int64_t d : deps[k]) succ[(size_t)d].push_back((int64_t)k);
    }
    using Key = std::tuple<int64_t, int64_t, int64_t>;  // (2*center anti-diagonal, r0, index)
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> ready;
    auto key = [&](size_t k) {
        const Tile &t = tiles[k];
        return Key{t.r0 + t.r1 + t.c0 + t.c1, t.r0, (int64_t)k};
    };
    for (size_t k = 0; k < T; ++k)
        if (indeg[k] == 0) ready.push(key(k));
    int64_t pos = 0;
    std::vector<Tile> ordered;
    ordered.reserve(T);
    while (!ready.empty()) {
        const size_t k = (size_t)std::get<2>(ready.top());
        ready.pop();
        tiles[k].order = pos++;
        ordered.push_back(tiles[k]);
        for (int64_t s : succ[k])
            if (--indeg[(size_t)s] == 0) ready.push(key((size_t)s));
    }
    if (ordered.size() != T) return false;  // a cycle cannot happen for a partition
    tiles.swap(ordered);
    return true;
}

void tile_deps(const std::vector<Tile> &tiles, std::vector<std::vector<int64_t>> &deps) {
    const size_t T = tiles.size();
    deps.assign(T, {});
    // index tiles by bottom edge (sorted by c0) and by right edge (sorted by r0)
    std::map<int64_t, std::vector<int64_t>> by_r1, by_c1;
    for (size_t k = 0; k < T; ++k) {
        by_r1[tiles[k].r1].push_back((int64_t)k);
        by_c1[tiles[k].c1].push_back((int64_t)k);
    }
    for (auto &kv : by_r1)
        std::sort(kv.second.begin(), kv.second.end(),
                  [&](int64_t a, int64_t b) { return tiles[(size_t)a].c0 < tiles[(size_t)b].c0; });
    for (auto &kv : by_c1)
        std::sort(kv.second.begin(), kv.second.end(),
                  [&](int64_t a, int64_t b) { return tiles[(size_t)a].r0 < tiles[(size_t)b].r0; });
    for (size_t k = 0; k < T; ++k) {
        const Tile &t = tiles[k];
        std::vector<int64_t> &d = deps[k];
        if (t.r0 > 0) {  // tiles above, columns [c0-1, c1)
            auto it = by_r1.find(t.r0);
            if (it != by_r1.end()) {
                const int64_t lo = std::max<int64_t>(0, t.c0 - 1), hi = t.c1;
                for (int64_t x : it->second) {
                    const Tile &u = tiles[(size_t)x];
                    if (u.c0 >= hi) break;
                    if (u.c1 > lo) d.push_back(x);
                }
            }
        }
        if (t.c0 > 0) {  // tiles to the left, rows [r0-1, r1)
            auto it = by_c1.find(t.c0);
            if (it != by_c1.end()) {
                const int64_t lo = std::max<int64_t>(0, t.r0 - 1), hi = t.r1;
                for (int64_t x : it->second) {
                    const Tile &u = tiles[(size_t)x];
                    if (u.r0 >= hi) break;
                    if (u.r1 > lo) d.push_back(x);
                }
            }
        }
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
    }
}

bool plan_pair(int64_t n, int64_t m, int sms, const PairPlanOptions &o, PairPlan &out) {
    if (n <= 0 || m <= 0 || sms <= 0) return false;
    out = PairPlan();
    out.transpose = o.orient == 2 || (o.orient == 0 && m > n);
    out.L = out.transpose ? m : n;
    out.S = out.transpose ? n : m;
    // chunk width: lane k of a strip trails lane 0 by a few chunks, so the
    // pipeline's fill grows with C while the per-chunk overhead shrinks;
    // measured on GB300, C = 2 wins from a 4096-column streamed side up.
    out.C = o.chunk ? o.chunk : ((out.S >= 64) ? 2 : 4);
    // words per lane: each lane streams all S columns after a fill of
    // (lanes x skew x C) column steps; two words per lane halve the lanes and
    // take a longer step (the same skew of 3 chunks; the step's time ratio is
    // measured on GB300).  Pick the smaller modelled time.
    if (o.wpl == 1 || o.wpl == 2) {
        out.wpl = o.wpl;
    } else {
        auto cost = [&](int wpl) {
            const double lanes = (double)((out.L + kPlanLaneRows * wpl - 1) / (kPlanLaneRows * wpl));
            const double skew = 3.0, step = wpl == 1 ? 1.0 : 1.18;
            return step * ((double)out.S + lanes * skew * out.C);
        };
        out.wpl = cost(2) < cost(1) ? 2 : 1;
    }
    const int64_t warp_rows = kPlanWarpRows * out.wpl, lane_rows = kPlanLaneRows * out.wpl;
    const int64_t warps_total = (out.L + warp_rows - 1) / warp_rows;
    // one warp per CTA strip unless the strips would not all be resident at once
    const int max_w = out.wpl == 2 ? o.max_warps_wpl2 : o.max_warps;
    int W = o.warps > 0 ? o.warps : 1;
    W = std::max(1, std::min(W, max_w));
    if ((int64_t)W > warps_total) W = (int)warps_total;
    int64_t nstrips = (warps_total + W - 1) / W;
    if (o.warps == 0 && o.resident > 0 && nstrips > o.resident) {
        // keep every strip resident when shared memory allows taller CTA strips
        const int64_t need = (warps_total + o.resident - 1) / o.resident;
        if (need <= max_w) {
            W = (int)need;
            nstrips = (warps_total + W - 1) / W;
        }
    }
    out.W = W;
    if (o.schedule == 1) {
        const int64_t h = (int64_t)W * warp_rows;
        nstrips = (out.L + h - 1) / h;
        out.row0.resize((size_t)nstrips + 1);
        for (int64_t k = 0; k <= nstrips; ++k) out.row0[(size_t)k] = std::min(out.L, k * h);
    } else {
        // the p-way first division of the PACO partition on rows, p = nstrips,
        // in lane granules of 31 * wpl rows (parts differ by at most one granule)
        const int64_t G = (out.L + lane_rows - 1) / lane_rows;
        const std::vector<int64_t> parts = balanced_split(G, nstrips);
        out.row0.resize((size_t)nstrips + 1);
        int64_t acc = 0;
        out.row0[0] = 0;
        for (int64_t k = 0; k < nstrips; ++k) {
            acc += parts[(size_t)k];
            out.row0[(size_t)k + 1] = std::min(out.L, acc * lane_rows);
        }
    }
    out.nstrips = (int)nstrips;
    out.grid = o.resident > 0 ? (int)std::min<int64_t>(nstrips, o.resident) : (int)nstrips;
    return true;
}

bool plan_shard(const int64_t *a_off, const int64_t *b_off, int64_t npairs, int ranks,
                std::vector<int32_t> &owner, std::vector<int64_t> &rank_cells) {
    if (npairs < 0 || ranks < 1 || (npairs > 0 && (!a_off || !b_off))) return false;
    std::vector<int64_t> cells((size_t)npairs);
    for (int64_t k = 0; k < npairs; ++k) {
        const int64_t n = a_off[k + 1] - a_off[k], m = b_off[k + 1] - b_off[k];
        if (n < 0 || m < 0) return false;
        cells[(size_t)k] = n * m;
    }
    std::vector<int64_t> order((size_t)npairs);
    for (int64_t k = 0; k < npairs; ++k) order[(size_t)k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t x, int64_t y) { return cells[(size_t)x] > cells[(size_t)y]; });
    owner.assign((size_t)npairs, 0);
    rank_cells.assign((size_t)ranks, 0);
    // least-loaded rank first; ties to the lowest rank
    using Item = std::pair<int64_t, int32_t>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int32_t r = 0; r < ranks; ++r) heap.push({0, r});
    for (int64_t k : order) {
        const Item it = heap.top();
        heap.pop();
        owner[(size_t)k] = it.second;
        rank_cells[(size_t)it.second] += cells[(size_t)k];
        heap.push({it.first + cells[(size_t)k], it.second});
    }
    return true;
}

namespace {

struct GTile {  // a tile in granules
    int64_t r0, r1, c0, c1;
};

// PO recursion: base tiles in fork-join order; returns (first, last) tile
// index of the node, and adds the join dependencies.
std::pair<int64_t, int64_t> po_node(int64_t r0, int64_t r1, int64_t c0, int64_t c1, int64_t base,
                                    std::vector<GTile> &out, std::vector<std::vector<int64_t>> &joins) {
    const bool split_r = (r1 - r0) > base, split_c = (c1 - c0) > base;
    if (!split_r && !split_c) {
        out.push_back({r0, r1, c0, c1});
        joins.emplace_back();
        const int64_t k = (int64_t)out.size() - 1;
        return {k, k};
    }
    const int64_t rm = split_r ? r0 + (r1 - r0) / 2 : r1, cm = split_c ? c0 + (c1 - c0) / 2 : c1;
    auto dep = [&](int64_t first, int64_t on) { joins[(size_t)first].push_back(on); };
    if (split_r && split_c) {
        auto x11 = po_node(r0, rm, c0, cm, base, out, joins);
        auto x12 = po_node(r0, rm, cm, c1, base, out, joins);
        dep(x12.first, x11.second);
        auto x21 = po_node(rm, r1, c0, cm, base, out, joins);
        dep(x21.first, x11.second);
        auto x22 = po_node(rm, r1, cm, c1, base, out, joins);
        dep(x22.first, x12.second);
        dep(x22.first, x21.second);
        return {x11.first, x22.second};
    }
    auto h1 = split_r ? po_node(r0, rm, c0, c1, base, out, joins) : po_node(r0, r1, c0, cm, base, out, joins);
    auto h2 = split_r ? po_node(rm, r1, c0, c1, base, out, joins) : po_node(r0, r1, cm, c1, base, out, joins);
    dep(h2.first, h1.second);
    return {h1.first, h2.second};
}

}  // namespace

bool plan_tiles(int64_t n, int64_t m, int p, int kind, int64_t base, TilePlan &out) {
    out = TilePlan();
    if (n <= 0 || m <= 0 || p <= 0 || base <= 0) return false;
    const int64_t ng = (n + kTileRowGranule - 1) / kTileRowGranule;
    const int64_t mg = (m + kTileColGranule - 1) / kTileColGranule;
    std::vector<GTile> g;
    std::vector<std::vector<int64_t>> joins;  // extra dependencies (PO), by granule tile
    if (kind == kTilesPaco) {
        std::vector<Tile> t;
        if (!paco_partition(ng, mg, p, base, t)) return false;
        for (const Tile &x : t) g.push_back({x.r0, x.r1, x.c0, x.c1});
    } else if (kind == kTilesPa) {
        const std::vector<int64_t> hs = balanced_split(ng, std::min<int64_t>(p, ng));
        const std::vector<int64_t> ws = balanced_split(mg, std::min<int64_t>(p, mg));
        std::vector<int64_t> r(hs.size() + 1, 0), c(ws.size() + 1, 0);
        for (size_t i = 0; i < hs.size(); ++i) r[i + 1] = r[i] + hs[i];
        for (size_t j = 0; j < ws.size(); ++j) c[j + 1] = c[j] + ws[j];
        const int64_t P = (int64_t)hs.size(), Q = (int64_t)ws.size();
        for (int64_t d = 0; d <= P + Q - 2; ++d)
            for (int64_t i = std::max<int64_t>(0, d - Q + 1); i <= std::min<int64_t>(d, P - 1); ++i)
                g.push_back({r[(size_t)i], r[(size_t)i + 1], c[(size_t)(d - i)], c[(size_t)(d - i) + 1]});
    } else if (kind == kTilesPo) {
        po_node(0, ng, 0, mg, base, g, joins);
    } else {
        return false;
    }
    if (joins.empty()) joins.resize(g.size());
    // bands of at most one warp's rows, in order; a join dependency moves to
    // the first band of its tile and points at the last band of the other
    std::vector<int64_t> first_band(g.size()), last_band(g.size());
    std::vector<Tile> tiles;
    for (size_t k = 0; k < g.size(); ++k) {
        first_band[k] = (int64_t)tiles.size();
        for (int64_t r = g[k].r0; r < g[k].r1; r += kTileMaxRowGranules) {
            const int64_t re = std::min(g[k].r1, r + kTileMaxRowGranules);
            Tile t{};
            t.r0 = std::min(n, r * kTileRowGranule);
            t.r1 = std::min(n, re * kTileRowGranule);
            t.c0 = std::min(m, g[k].c0 * kTileColGranule);
            t.c1 = std::min(m, g[k].c1 * kTileColGranule);
            t.order = (int64_t)tiles.size();
            tiles.push_back(t);
        }
        last_band[k] = (int64_t)tiles.size() - 1;
    }
    std::vector<std::vector<int64_t>> deps;
    tile_deps(tiles, deps);
    out.join0.assign(tiles.size(), -1);
    out.join1.assign(tiles.size(), -1);
    for (size_t k = 0; k < g.size(); ++k) {
        const size_t fb = (size_t)first_band[k];
        for (int64_t on : joins[k]) {
            const int64_t target = last_band[(size_t)on];
            deps[fb].push_back(target);
            if (out.join0[fb] < 0) out.join0[fb] = target;
            else if (out.join1[fb] < 0 && out.join0[fb] != target) out.join1[fb] = target;
            else if (out.join0[fb] != target && out.join1[fb] != target) return false;  // at most two
        }
    }
    out.dep_off.assign(tiles.size() + 1, 0);
    std::vector<int64_t> finish(tiles.size(), 0);
    for (size_t k = 0; k < tiles.size(); ++k) {
        std::vector<int64_t> &d = deps[k];
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
        int64_t start = 0;
        for (int64_t x : d) {
            if (x >= (int64_t)k) return false;  // not a topological order
            out.dep_idx.push_back(x);
            start = std::max(start, finish[(size_t)x]);
        }
        out.dep_off[k + 1] = (int64_t)out.dep_idx.size();
        const Tile &t = tiles[k];
        finish[k] = start + (t.r1 - t.r0) * (t.c1 - t.c0);
        out.critical_cells = std::max(out.critical_cells, finish[k]);
    }
    out.tiles.swap(tiles);
    return true;
}

}  // namespace paco
