// Host-side planner: the PACO partition of the LCS table (Sec. "PACO LCS")
// and the strip plan the bit-parallel pipeline executes.  Pure C++ (no CUDA),
// so it is testable on a machine without a GPU through include/paco_plan.h.
#pragma once

#include <stdint.h>

#include <vector>

namespace paco {

// Rows held by one lane of the bit-parallel tile (bit 31 is its carry slot)
// and by one warp of 32 lanes.
constexpr int64_t kPlanLaneRows = 31;
constexpr int64_t kPlanWarpRows = 31 * 32;

// ---- the paper's partition, re-derived for an n x m table and any p ----
//
// Step 1 (the proof's simplification, "the first step of partitioning makes
// a p-way division"): rows and columns are each cut p ways by the balanced
// integer split (parts differ by at most one row/column).  Then, repeatedly:
// group the unassigned regions of the current level by anti-diagonal (equal
// row-index + column-index of the level's grid); every anti-diagonal holding
// at least p of them gets p regions assigned round-robin to processors
// 0..p-1 (the p with the smallest column index); when no unassigned region
// can be halved any more (a side would drop below `base`), all remaining
// ones are assigned round-robin; otherwise each unassigned region is divided
// 2-way in both dimensions (a quadtree step) and the next level starts.
struct Tile {
    int64_t r0, r1, c0, c1;  // rows [r0, r1), columns [c0, c1) of the DP cells (0-based)
    int32_t label;           // assignment round, 1 = first (largest regions)
    int32_t owner;           // processor 0..p-1
    int64_t order;           // position in the execution time line (topological)
};

// Returns false on bad arguments.  `tiles` receives the regions in time-line
// order (each region after every region it depends on).
bool paco_partition(int64_t n, int64_t m, int32_t p, int64_t base, std::vector<Tile> &tiles);

// Dependencies of tile k: every tile whose bottom edge touches k's top edge,
// whose right edge touches k's left edge, or that holds the cell diagonally
// above-left of k's corner.
void tile_deps(const std::vector<Tile> &tiles, std::vector<std::vector<int64_t>> &deps);

// ---- the strip plan of the bit-parallel pipeline ----
struct PairPlan {
    bool transpose = false;  // true: bits along b (rows of the kernel = b)
    int C = 8;               // columns per lane hand-off
    int W = 4;               // warps per CTA strip
    int wpl = 1;             // 31-row words per lane (a lane holds 31 * wpl rows)
    int nstrips = 1;         // CTA strips (the p of the balanced split)
    int grid = 1;            // CTAs launched (<= nstrips)
    int64_t L = 0, S = 0;    // kernel rows (bit dimension) and streamed columns
    std::vector<int64_t> row0;  // nstrips+1 offsets, multiples of 31 * wpl, row0[nstrips] = L
};

struct PairPlanOptions {
    int chunk = 0;      // 0: cost model
    int warps = 0;      // 0: default
    int orient = 0;     // 0: bits along the longer string; 1: along a; 2: along b
    int schedule = 0;   // 0: balanced strips (p-way split); 1: uniform strips of W*992*wpl rows
    int wpl = 0;        // 31-row words per lane: 0 = planner, 1 or 2
    int max_warps = 7;       // shared-memory limit per CTA with one word per lane
    int max_warps_wpl2 = 3;  // ... and with two words per lane (twice the match tables)
    int resident = 0;   // CTAs that fit on the device at once (0: unknown)
};

bool plan_pair(int64_t n, int64_t m, int sms, const PairPlanOptions &o, PairPlan &out);

// Size-balanced greedy assignment of independent pairs to `ranks`: largest
// cells first, each to the least-loaded rank (ties: lowest rank).  Returns
// false on bad arguments.
bool plan_shard(const int64_t *a_off, const int64_t *b_off, int64_t npairs, int ranks,
                std::vector<int32_t> &owner, std::vector<int64_t> &rank_cells);

// Balanced integer split of `total` units into `parts` (first total%parts get one more).
std::vector<int64_t> balanced_split(int64_t total, int64_t parts);

// ---- tile schedules: the paper's comparison (PACO against PA and PO) ----
//
// All three cut the table into tiles on a grid of 31-row x 64-column
// granules (a lane's rows, two carry words' columns) and run them as a
// dataflow: a tile starts when the tiles it depends on are done.
//   kTilesPaco: the PACO partition above, computed on the granule grid.
//   kTilesPa:   the processor-aware p-way division of Chowdhury and
//               Ramachandran: a p x p grid of blocks in anti-diagonal order,
//               critical path (2p - 1) blocks of n m / p^2 cells.
//   kTilesPo:   the processor-oblivious 2-way divide and conquer: X11, then
//               X12 and X21, then X22, recursively down to base tiles, with
//               the fork-join order as extra dependencies (a quadrant starts
//               only when the quadrants before it are complete).
// Tiles taller than one warp (32 granules = 992 rows) are cut into bands.
enum TileKind { kTilesPaco = 1, kTilesPa = 2, kTilesPo = 3 };
struct TilePlan {
    std::vector<Tile> tiles;           // execution order; rows/columns in cells
    std::vector<int64_t> dep_off;      // tiles.size()+1 offsets into dep_idx
    std::vector<int64_t> dep_idx;      // each dependency precedes its tile
    std::vector<int64_t> join0, join1; // per tile: fork-join dependencies (PO), -1 if none
    int64_t critical_cells = 0;        // heaviest dependency path, in cells
};
constexpr int64_t kTileRowGranule = 31;
constexpr int64_t kTileColGranule = 64;
constexpr int64_t kTileMaxRowGranules = 32;  // one warp's rows
// base: the smallest tile side in granules (PACO stop, PO base).
bool plan_tiles(int64_t n, int64_t m, int p, int kind, int64_t base, TilePlan &out);

}  // namespace paco
