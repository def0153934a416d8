// Internal declarations shared by the host API and the CUDA kernels.
// Not part of the public ABI (include/paco_lcs.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace paco {

// Error words written by device code (same values as paco_status).
enum : int { kOk = 0, kEinval = -1, kEnomem = -2, kEtimeout = -3, kEdevice = -4, kEbusy = -5 };

// Maximum alphabet a bit-parallel match table covers (bytes).
constexpr int kMaxSigma = 256;
// Slots of the shared-memory ring that hands carry words from one warp of a
// CTA strip to the next.
constexpr int kRing = 32;

// ---------------------------------------------------------------------------
// Single pair, bit-parallel strip pipeline (one launch for the whole path).
//
// The table is processed with its rows along bits: row string `a` (length
// L), column string `b` (length S).  Rows are cut into `nstrips` CTA strips
// (balanced granules of one lane's rows, 31 x words per lane); CTA strip s
// is W warps x 32 lanes x (31 x words per lane) rows.  Columns are cut into
// chunks of C columns; a lane hands the C carry bits of a chunk (the
// horizontal steps of the table at the lane's last row) to the next lane.
// Between CTA strips, the carries of the strip's last row travel through
// `hbuf`, tagged with the launch epoch so a consumer can tell a published
// word from a stale one without a separate flag.  The boundaries in and out
// are plain int32 values; the kernel converts them itself.
// ---------------------------------------------------------------------------
struct PairArgs {
    const uint8_t *a;            // row string (bits), length L
    const uint8_t *b;            // column string (streamed), length S
    int64_t L, S;
    int32_t nwords;              // ceil(S / 32): words per carry row
    int64_t hstride;             // words between carry rows (nwords rounded up to even)
    int64_t granules;            // lane granules (31 * wpl rows) over L: strip s starts at granule
                                 //   s * (granules / nstrips) + min(s, granules % nstrips)
    int64_t uniform_rows;        // > 0: strips of this many rows instead (the last one shorter)
    int nstrips;
    const int32_t *top;          // S + 1 values of the first row, or NULL (zeros)
    const int32_t *left;         // L + 1 values of the first column, or NULL (zeros)
    int32_t *bottom;             // S + 1 values of the last row out, or NULL
    int32_t *right;              // L + 1 values of the last column out, or NULL
    int32_t *len;                // H[L][S] out, or NULL
    uint64_t *hbuf;              // (nstrips+1) x hstride tagged carry words; row s = strip s's input
    int *ctl;                    // [0] strip ticket, [1] exit count: zero between launches (the
                                 //   kernel's last CTA resets them)
    int *err;                    // device error word
    uint32_t epoch;              // tag of this launch (never 0)
    long long wait_limit_ns;     // bounded-wait limit
    int stall_strip;             // tests: strip whose input never arrives (-1: none)
};

// Launch helpers (defined in pair_kernels.cu).
// wpl: 31-row words per lane (1 or 2)
size_t pair_smem_bytes(int warps, int C, int wpl);  // dynamic shared memory of one CTA
int pair_max_warps(int wpl);
int pair_occupancy(int C, int warps, int wpl);  // resident CTAs per SM
cudaError_t launch_pair_bp(const PairArgs &p, int C, int warps, int wpl, int grid, cudaStream_t st);

// n == 0 or m == 0 tables: copy/zero the boundaries.
cudaError_t launch_degenerate(const int32_t *top, const int32_t *left, int64_t n, int64_t m,
                              int32_t *bottom_row, int32_t *right_col, int32_t *len,
                              int *err, cudaStream_t st);

// Integer ALU microbenchmark (roofline denominator).
cudaError_t launch_int_peak(int op, int grid, int block, int iters, uint32_t *sink,
                            cudaStream_t st);

}  // namespace paco
