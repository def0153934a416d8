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
// Single pair, bit-parallel strip pipeline.
//
// The table is processed with its rows along bits: row string `a` (length
// L), column string `b` (length S).  Rows are cut into `nstrips` CTA strips
// (balanced granules of one lane's rows, 31 x words per lane); CTA strip s
// is W warps x 32 lanes x (31 x words per lane) rows.  Columns are cut into
// chunks of C columns; a lane hands the C carry bits of a chunk (the
// horizontal steps of the table at the lane's last row) to the next lane.
// Between CTA strips, the carries of the strip's last row travel through
// `hbuf`, tagged with the launch epoch so a consumer can tell a published
// word from a stale one without a separate flag.
// ---------------------------------------------------------------------------
struct PairArgs {
    const uint8_t *a;            // row string (bits), length L
    const uint8_t *b;            // column string (streamed), length S
    int64_t L, S;
    int64_t nwords;              // ceil(S / 32): words per carry row
    int64_t hstride;             // words between carry rows (nwords rounded up to even)
    const int64_t *strip_row0;   // nstrips+1 row offsets (multiples of 31 * wpl, last = L), or NULL:
    int64_t granules;            //   then strip s starts at 31*wpl*(s*(granules/nstrips) + min(s, granules%nstrips))
    int nstrips;
    int sigma;                   // match-table rows (symbols must be < sigma)
    const uint32_t *left_bits;   // L bits: vertical steps of the first column
    uint32_t *right_bits;        // ceil(L/31) lane words out: vertical steps of the last column
    uint64_t *hbuf;              // (nstrips+1) x hstride tagged carry words; row 0 = input top
    int *ticket;                 // strip ticket counter (zeroed before launch)
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

// Input boundary (int32, len+1 values) -> step bits (len bits) with checks.
cudaError_t launch_boundary_bits(const int32_t *v, int64_t len, uint32_t *bits,
                                 uint64_t *tagged, uint32_t epoch,
                                 const int32_t *other, int *err, cudaStream_t st);
// Bits (tagged or plain) -> int32 prefix output with a base value.
struct PrefixScratch { int64_t *block_sums; int64_t cap; };
// bpw: elements per word (32: packed bit rows; 31: lane words).
cudaError_t launch_bits_prefix(const uint32_t *bits, const uint64_t *tagged, int64_t nbits, int bpw,
                               const int32_t *base_ptr, int64_t base_index,
                               int32_t *out, int32_t *len_out,
                               PrefixScratch &scr, cudaStream_t st);
// n == 0 or m == 0 tables: copy/zero the boundaries.
cudaError_t launch_degenerate(const int32_t *top, const int32_t *left, int64_t n, int64_t m,
                              int32_t *bottom_row, int32_t *right_col, int32_t *len,
                              int *err, cudaStream_t st);

// Integer ALU microbenchmark (roofline denominator).
cudaError_t launch_int_peak(int op, int grid, int block, int iters, uint32_t *sink,
                            cudaStream_t st);

}  // namespace paco
