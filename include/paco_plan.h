/*
 * paco_plan.h - host-only planner introspection (no GPU needed).
 *
 * The partition follows the PACO LCS partitioning phase of Tang & Gao,
 * Sec. "PACO LCS" (and its proof's simplification that the first step is a
 * p-way division): the table is cut p ways in each dimension, then regions
 * are repeatedly halved in both dimensions; whenever an anti-diagonal holds
 * at least p unassigned regions, p of them are assigned round-robin to the
 * p processors; regions that can no longer be halved (a side below 2*base)
 * are assigned round-robin.  Regions are returned in time-line order: each
 * after every region it depends on (its neighbours above and to the left).
 *
 * The pair plan is what the bit-parallel strip pipeline executes for one
 * table: the p-way balanced split of the rows into CTA strips.
 */
#ifndef PACO_PLAN_H
#define PACO_PLAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct paco_tile {
    int64_t r0, r1, c0, c1; /* DP cells: rows [r0, r1), columns [c0, c1), 0-based */
    int32_t label;          /* assignment round (1 = the first p-way regions)      */
    int32_t owner;          /* processor 0..p-1                                      */
    int64_t order;          /* position in the time line                             */
} paco_tile;

/* Partition an n x m table for p processors, stopping at regions whose
 * sides cannot be halved without dropping below `base`.  Writes up to `cap`
 * tiles to `out` (may be NULL to query the count) and the total to *count.
 * Returns 0, or -1 (PACO_EINVAL) for n, m, p, base <= 0. */
int paco_plan_partition(int64_t n, int64_t m, int32_t p, int64_t base, paco_tile *out, int64_t cap,
                        int64_t *count);

/* Dependencies of every tile of the partition above, as a CSR list over
 * the returned order: dep_off[k]..dep_off[k+1] index dep_idx.  dep_off has
 * count+1 entries; dep_idx capacity `cap_idx`.  Returns 0 or -1. */
int paco_plan_partition_deps(int64_t n, int64_t m, int32_t p, int64_t base, int64_t *dep_off,
                             int64_t *dep_idx, int64_t cap_idx, int64_t *n_idx);

typedef struct paco_pair_plan {
    int32_t transpose;  /* 1: bits run along b                                 */
    int32_t chunk;      /* columns per lane hand-off                          */
    int32_t warps;      /* warps per CTA strip                                */
    int32_t nstrips;    /* CTA strips (the p of the balanced row split)       */
    int32_t words_per_lane; /* 31-row words per lane (1 or 2)                 */
    int32_t pad;
    int64_t L, S;       /* kernel rows (bit dimension) and streamed columns   */
} paco_pair_plan;

/* Plan one pair for a device with `sms` multiprocessors.  chunk/warps 0 =
 * planner's choice; orient 0 = bits along the longer string, 1 = along a,
 * 2 = along b; schedule 0 = balanced strips, 1 = uniform strips;
 * words_per_lane 0 = planner, 1 or 2 (a lane holds 31 or 62 rows).
 * row0 (capacity cap, may be NULL) receives nstrips+1 strip row offsets.
 * Returns 0 or -1. */
int paco_plan_pair(int64_t n, int64_t m, int32_t sms, int32_t chunk, int32_t warps, int32_t orient,
                   int32_t schedule, int32_t words_per_lane, paco_pair_plan *out, int64_t *row0,
                   int64_t cap);

/* Tile schedules for the comparison the paper runs (PACO against the
 * processor-aware PA and the processor-oblivious PO divide and conquer),
 * all on a grid of 31-row x 64-column granules, tiles at most 992 rows:
 *   kind 1 = PACO: the partition above on the granule grid (base in granules);
 *   kind 2 = PA: a p x p grid of blocks in anti-diagonal order;
 *   kind 3 = PO: 2-way divide and conquer down to base x base granules, with
 *            the fork-join order (X11; X12 and X21; X22) as dependencies.
 * Writes up to `cap` tiles in execution order (label/owner unused: 0), the
 * dependency CSR (dep_off[count+1], dep_idx up to cap_idx), the number of
 * tiles and dependency entries, and the heaviest dependency path in cells
 * (*critical_cells; the paper's critical-path measure).  Returns 0 or -1. */
int paco_plan_tiles(int64_t n, int64_t m, int32_t p, int32_t kind, int64_t base, paco_tile *out,
                    int64_t cap, int64_t *count, int64_t *dep_off, int64_t *dep_idx, int64_t cap_idx,
                    int64_t *n_idx, int64_t *critical_cells);

/* PACO 1D (Sec. "PACO 1D"): the work of Eq. (1D) over outputs and inputs
 * 0..n is the triangle {(i, j): i < j}.  The recursion on an output range
 * runs the left half's triangle, the square updating the right half from
 * the left half, and the right half's triangle; each square is cut along
 * its longer side in the ratio floor(p'/2) : ceil(p'/2) together with its
 * processor list of p' processors, down to one processor per rectangle.
 * A cut along the input side gives the second part temporary space (one
 * value per output column of the part) merged by a min after the phase.
 * Triangles at most `base` wide are base cases on processor 0.
 * Task kinds: 0 = base triangle (outputs [j0, j1), inputs i < j in the same
 * range), 1 = rectangle (outputs [j0, j1) x inputs [i0, i1)).  Tasks of one
 * phase run concurrently; phases run in order.  merge_group = -1 when the
 * rectangle writes the outputs, else the temporary buffer it writes. */
typedef struct paco_1d_task {
    int64_t j0, j1, i0, i1;
    int32_t proc, phase, merge_group, kind;
} paco_1d_task;

/* Writes up to `cap` tasks in order, the task count, the number of phases
 * and the temporary words the input-side cuts need.  Returns 0 or -1. */
int paco_plan_1d(int64_t n, int32_t p, int64_t base, paco_1d_task *out, int64_t cap, int64_t *count,
                 int32_t *phases, int64_t *temp_words);

/* Shard a batch of independent pairs over `ranks` GPUs (one process per
 * GPU).  The pairs of a batch share nothing, so the split needs no exchange
 * of intermediate data: each rank runs its pairs with paco_lcs_batch and the
 * results are gathered.  The split balances work the way the paper's
 * partition balances its regions, here by size-balanced greedy assignment:
 * pairs in decreasing order of cells n_k * m_k, each to the rank with the
 * fewest cells so far (ties to the lowest rank; equal pairs keep index
 * order).  Every rank's total then exceeds the smallest total by at most
 * the largest single pair.
 *   a_off, b_off : int64[npairs+1] offsets (pair k is n_k = a_off[k+1] -
 *                  a_off[k] by m_k = b_off[k+1] - b_off[k]), host memory
 *   owner        : int32[npairs] out: the rank of each pair
 *   rank_cells   : int64[ranks] out (may be NULL): cells per rank
 * Returns 0, or -1 for npairs < 0, ranks < 1, NULL arrays or decreasing
 * offsets. */
int paco_plan_shard(const int64_t *a_off, const int64_t *b_off, int64_t npairs, int32_t ranks, int32_t *owner,
                    int64_t *rank_cells);

#ifdef __cplusplus
}
#endif

#endif /* PACO_PLAN_H */
