/*
 * paco_lcs.h - C ABI of the GB300 LCS wavefront library.
 *
 * The library fills the longest-common-subsequence table of Eq. (1) in
 * Tang & Gao, "Balanced Partitioning of Several Cache-Oblivious Algorithms"
 * (Sec. "PACO LCS"):
 *
 *   H[i][0] = left[i], H[0][j] = top[j]   (zeros when not given, as in Eq. (1))
 *   H[i][j] = H[i-1][j-1] + 1               if a[i-1] == b[j-1]
 *           = max(H[i-1][j], H[i][j-1])     otherwise
 *
 * for byte strings a (n rows) and b (m columns), and returns the LCS length
 * L = H[n][m] together with the table's last row bottom_row[j] = H[n][j]
 * (j = 0..m) and last column right_col[i] = H[i][m] (i = 0..n).  Those two
 * boundaries are exactly what the paper's execution phase hands from one
 * region to its neighbours (Sec. "PACO LCS": each sub-region depends only on
 * its neighbouring regions), so a caller can chain calls over a larger table.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Symbols are raw bytes compared by equality; 0 is an ordinary symbol.
 * - Lengths n, m are in [0, 2^31 - 1]; anything else returns PACO_EINVAL.
 * - Device pointers are CUDA global-memory pointers on the context's device.
 *   `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Device entry points are stream ordered: they return after
 *   enqueueing; results are valid once the stream reaches that point.
 * - The caller owns every input and output buffer.  Inputs are never
 *   written.  The context owns all scratch memory (flags, boundary bit
 *   buffers, plans) and grows it on demand; scratch is reused across calls,
 *   so calls on one context must be serialised on one stream (or synchronised
 *   by the caller).
 * - Return values: PACO_OK (0), PACO_PENDING (1, poll only) or a negative
 *   paco_status.  A device-side failure (a bounded wait that timed out)
 *   cannot be seen at enqueue time: it is recorded in a device error word and
 *   returned by the next paco_ctx_sync (sticky until then).
 * - Input boundaries `top`/`left` must be valid LCS boundaries: top[0] ==
 *   left[0], and each is non-decreasing with steps in {0, 1}.  Every row and
 *   column of a true LCS table has this property (it is what one region
 *   receives from its neighbours).  Device-side inputs are checked on the
 *   device; a violation is reported as PACO_EINVAL by paco_ctx_sync.
 */
#ifndef PACO_LCS_H
#define PACO_LCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct paco_ctx paco_ctx;

typedef enum paco_status {
    PACO_OK = 0,
    PACO_PENDING = 1,     /* paco_lcs_poll: request not finished yet        */
    PACO_EINVAL = -1,     /* bad argument or invalid boundary               */
    PACO_ENOMEM = -2,     /* device or host allocation failed               */
    PACO_ETIMEOUT = -3,   /* a device wait exceeded its limit               */
    PACO_EDEVICE = -4,    /* a CUDA call failed (message: paco_last_error)  */
    PACO_EBUSY = -5,      /* serving queue full / budget exhausted          */
    PACO_ENOTFOUND = -6   /* unknown serving ticket                         */
} paco_status;

/* ---- context --------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `mem_budget_bytes` bounds the
 * device memory the serving path may hold for admitted requests (0 = 8 GiB).
 * Writes the new context to *out.  Errors: PACO_EINVAL (out == NULL or bad
 * device), PACO_EDEVICE, PACO_ENOMEM. */
int paco_ctx_create(int device, size_t mem_budget_bytes, paco_ctx **out);

/* Destroy a context: drains its streams and the serving loop, frees its
 * scratch.  NULL is ignored. */
void paco_ctx_destroy(paco_ctx *ctx);

/* Human-readable name of a status code (static string). */
const char *paco_strerror(int status);

/* Last CUDA/diagnostic message recorded on the context (static per ctx). */
const char *paco_last_error(paco_ctx *ctx);

/* Wait for all work the context enqueued on `stream` (NULL: all of the
 * context's streams and the caller's last stream) and return the first
 * sticky device error (PACO_ETIMEOUT, PACO_EINVAL), clearing it.  The stream
 * argument lets a caller that keeps several streams wait for one of them
 * without draining the others (the bounded waits of the paper's execution
 * phase, Sec. "PACO LCS", report their timeouts here). */
int paco_ctx_sync(paco_ctx *ctx, void *stream);

/* Tunables (engine choice, chunk width, warps per CTA, wait limit ...).
 * See PACO_OPT_* below.  Returns PACO_EINVAL for an unknown option or a
 * value out of range. */
int paco_ctx_set_option(paco_ctx *ctx, int option, int64_t value);
int paco_ctx_get_option(paco_ctx *ctx, int option, int64_t *value);

enum paco_option {
    PACO_OPT_ENGINE = 1,        /* 0 = auto, 1 = bit-parallel (the only engine) */
    PACO_OPT_CHUNK = 2,         /* columns per lane hand-off: 2, 4 or 8 (0 = planner) */
    PACO_OPT_WARPS = 3,         /* compute warps per CTA strip, 0..7 (0 = planner); more
                                   than fit in shared memory are clamped */
    PACO_OPT_WAIT_LIMIT_NS = 4, /* bounded-wait limit per wait, ns (default 2e9) */
    PACO_OPT_ORIENT = 5,        /* 0 = planner, 1 = bits along a, 2 = along b  */
    PACO_OPT_SCHEDULE = 6,      /* 0 = PACO balanced strips, 1 = uniform strips */
    PACO_OPT_ALPHABET = 7,      /* batch and serving: symbols are < this (1..256, default
                                   256); a smaller alphabet shrinks the per-warp match
                                   table and raises occupancy.  A symbol outside it never
                                   matches and the call reports PACO_EINVAL */
    PACO_OPT_BATCH_CHUNKS = 8,  /* read only: chunk widths the last paco_lcs_batch call ran
                                   with, one per size class of the streamed side
                                   (< 256, < 1024, < 4096, >= 4096 columns), 4 bits each,
                                   smallest class in the low bits */
    PACO_OPT_WORDS_PER_LANE = 9, /* single pair: 31-row words per lane, 1 or 2 (0 =
                                   planner); two words give each lane two
                                   dependency chains and halve the strips */
    PACO_OPT_TILES = 10,        /* single pair: 0 = strip pipeline; 1, 2, 3 = the tile
                                   schedules of include/paco_plan.h (PACO partition, PA
                                   p x p blocks, PO divide and conquer) on the batch
                                   kernel, for the paper's comparison; zero boundaries only */
    PACO_OPT_TILE_BASE = 11,    /* tile schedules: smallest tile side in 31-row / 64-column
                                   granules (0 = 4 for PACO, 16 for PO) */
    PACO_OPT_AFFINE_ROWS = 12,  /* affine alignment (include/paco_affine.h): rows per
                                   lane of a row band, 2, 4 or 8 (0 = 4) */
    PACO_OPT_SERVE_CHUNKS = 13, /* serving: chunk width per size class for the
                                   micro-batches, packed like PACO_OPT_BATCH_CHUNKS
                                   (each 2, 4 or 8); 0 = the defaults 2, 4, 8, 8.  A
                                   caller can pass the widths the batch autotuner
                                   picked on a batch of the same mix */
    PACO_OPT_TEST_STALL = 100   /* tests only: make one strip (pair kernel), one
                                   band job (affine) or one block (1D problem) wait
                                   for input that never arrives (exercises the
                                   bounded wait) */
};

/* ---- single pair ------------------------------------------------------ */

/* LCS length only: L = H[n][m] of Eq. (1), the quantity the paper's LCS
 * section computes (Sec. "PACO LCS").  a: device uint8[n]; b: device uint8[m];
 * d_len: device int32[1] receiving L.  Errors: PACO_EINVAL (NULL pointer with a non-zero
 * length, negative or too-large length), PACO_ENOMEM, PACO_EDEVICE. */
int paco_lcs_length(paco_ctx *ctx, const uint8_t *a, int64_t n,
                    const uint8_t *b, int64_t m, int32_t *d_len, void *stream);

/* Length plus boundaries: the whole table of Eq. (1) with the given first
 * row and column, returning its last row and column, i.e. one region of the
 * paper's execution phase (Sec. "PACO LCS": a region needs only the
 * boundaries its neighbours above and to the left hand it, and hands its own
 * last row and column on).  The table is split across the GPU's SMs by the
 * p-way first cut of the PACO partition (rows in balanced strips), and runs
 * in one launch.  d_top_in: device int32[m+1] or NULL (zeros);
 * d_left_in: device int32[n+1] or NULL (zeros); d_bottom_row: device
 * int32[m+1] or NULL; d_right_col: device int32[n+1] or NULL; d_len: device
 * int32[1] or NULL.  Output buffers must not overlap inputs. */
int paco_lcs_boundaries(paco_ctx *ctx, const uint8_t *a, int64_t n,
                        const uint8_t *b, int64_t m,
                        const int32_t *d_top_in, const int32_t *d_left_in,
                        int32_t *d_bottom_row, int32_t *d_right_col,
                        int32_t *d_len, void *stream);

/* The same computation (Eq. (1), Sec. "PACO LCS") from HOST buffers
 * (pageable or pinned): copies a, b
 * (and the optional host boundaries) to the device, runs, copies the
 * requested outputs back, and returns when they are in host memory.  Any
 * output pointer may be NULL. */
int paco_lcs_boundaries_host(paco_ctx *ctx, const uint8_t *a, int64_t n,
                             const uint8_t *b, int64_t m,
                             const int32_t *top_in, const int32_t *left_in,
                             int32_t *bottom_row, int32_t *right_col,
                             int32_t *len, void *stream);

/* Length plus boundaries with NO device allocation, for callers that cannot
 * allocate device memory where they need the result: e.g. code running as a
 * plugin or callback inside another framework that owns every device
 * allocation through its own pool, or a latency-critical loop in which a
 * cudaMalloc/cudaFree would synchronise the device.  There is no counterpart
 * in the paper; this is a deployment variant of paco_lcs_boundaries with
 * zero first row and column (top = left = 0) and the planner's defaults.
 *
 * No context is used: all scratch (step bits, carry rows, prefix-sum
 * partials, ticket and error words) lives in one fixed 32 MiB __device__
 * array inside this library, which every GPU that loads the library keeps
 * until the process exits.  The call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).
 *   a, b        : device uint8[n], uint8[m]
 *   d_bottom_row: device int32[m+1] or NULL;  d_right_col: int32[n+1] or NULL
 *   d_len       : device int32[1], required (NULL is PACO_EINVAL); receives
 *                 L, or a negative paco_status (PACO_ETIMEOUT) when a device
 *                 wait timed out, in which case the boundaries are void
 * Every buffer must be on the CURRENT device: the call takes the scratch of
 * the device that is current (cudaGetDevice) and launches on `stream`, which
 * must belong to that device.  Stream ordered (stream = cudaStream_t or
 * NULL).  Each call looks up the array's device address on the current
 * device (cudaGetSymbolAddress, no allocation); the first lookup on a device
 * loads the library's device code there, so make the first call on each
 * device before any stream capture.
 * All calls on a device share the one array and keep the previous call's
 * contents (each call clears what must start at zero): calls that overlap on
 * the GPU race, so serialise them.  Returns PACO_EINVAL for bad arguments or
 * when the table needs more than the 32 MiB of scratch, PACO_EDEVICE for a
 * CUDA error.  The scratch is mostly the strips' carry rows, (strips + 1) x
 * S / 4 bytes with S the shorter side and about one strip per 992 rows of
 * the longer side (fewer, taller strips once they would not all be
 * resident): square tables fit up to about 360,000 per side. */
int paco_lcs_boundaries_static(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                               int32_t *d_bottom_row, int32_t *d_right_col, int32_t *d_len,
                               void *stream);

/* ---- batch of independent pairs ---------------------------------------- */

/* npairs independent tables of Eq. (1) in one persistent launch; the balanced
 * share of work per SM that the PACO partition gives one table (Sec. "PACO
 * LCS") is here a longest-first order of warp jobs over many tables.  The
 * offsets are HOST arrays because the planner needs the lengths before
 * anything is launched (reading device offsets would cost a copy and a
 * synchronisation per call).  The whole step (column
 * tables, the persistent warp-job kernel, the boundary prefixes) is captured
 * once into a CUDA graph per context, layout and output pointers, then
 * replayed; the chunk width is autotuned once per layout (PACO_OPT_CHUNK
 * forces one).
 *   a_cat, b_cat      : device uint8, all strings concatenated
 *   h_a_off, h_b_off  : HOST int64[npairs+1]; pair k is a_cat[h_a_off[k] ..
 *                       h_a_off[k+1]) x b_cat[h_b_off[k] .. h_b_off[k+1])
 *   d_len             : device int32[npairs], receives L_k
 *   d_rows_cat        : device int32 or NULL; pair k's bottom row H[n_k][0..m_k]
 *                       (m_k+1 values) at offset h_row_off[k]
 *   h_row_off         : HOST int64[npairs] (ignored when d_rows_cat is NULL)
 *   d_cols_cat        : device int32 or NULL; pair k's right column
 *                       H[0..n_k][m_k] (n_k+1 values) at offset h_col_off[k]
 *   h_col_off         : HOST int64[npairs]
 * The host arrays are read during the call (the planner needs the lengths).
 * Errors: PACO_EINVAL (negative or oversized length, NULL with work to do),
 * PACO_ENOMEM, PACO_EDEVICE. */
int paco_lcs_batch(paco_ctx *ctx, const uint8_t *a_cat, const uint8_t *b_cat,
                   const int64_t *h_a_off, const int64_t *h_b_off, int32_t npairs,
                   int32_t *d_len, int32_t *d_rows_cat, const int64_t *h_row_off,
                   int32_t *d_cols_cat, const int64_t *h_col_off, void *stream);

/* ---- serving: continuous batching ------------------------------------- */

/* Serving (continuous batching of tables of Eq. (1); not in the paper):
 * submit one request from HOST memory.  The library copies the strings
 * before returning (the caller may free them).  The request is admitted to
 * the device when the context's memory budget allows, runs in a micro-batch
 * with whatever else is admitted, and is retrieved with paco_lcs_poll.
 * want_boundaries != 0 keeps bottom_row/right_col for poll.  Writes a ticket.
 * Errors: PACO_EINVAL, PACO_EBUSY (a single request larger than the budget,
 * or the host queue or string arena is full: retry after polling),
 * PACO_ENOMEM. */
int paco_lcs_submit(paco_ctx *ctx, const uint8_t *a, int64_t n,
                    const uint8_t *b, int64_t m, int want_boundaries,
                    uint64_t *ticket);

/* Poll a ticket.  PACO_PENDING while queued or running; PACO_OK when done,
 * after writing *len and (if the request kept them and the pointers are not
 * NULL) HOST row_out[m+1] / col_out[n+1]; the ticket is then released.
 * PACO_ENOTFOUND for an unknown or already released ticket; a device error
 * of the request's micro-batch is returned once (and the ticket released). */
int paco_lcs_poll(paco_ctx *ctx, uint64_t ticket, int32_t *len,
                  int32_t *row_out, int32_t *col_out);

/* Submit `count` requests at once: request k is a_cat[a_off[k] ..
 * a_off[k+1]) against b_cat[b_off[k] .. b_off[k+1]), all HOST buffers
 * copied before the call returns (a submission of several MiB is copied by
 * the calling thread and a few helper threads); lengths only (no
 * boundaries).  Requests are published to the engine in groups of up to 512
 * as their strings are copied, so the engine starts on the first group
 * while later ones are copied.  tickets[count] receives the tickets.
 * Returns PACO_OK, PACO_EINVAL for a bad argument (nothing submitted), or
 * PACO_EBUSY when a request does not fit the budget, or the queue or string
 * arena is full: then *n_submitted (if not NULL) tells how many of the
 * first requests were taken, and the caller submits the rest after polling. */
int paco_lcs_submit_many(paco_ctx *ctx, const uint8_t *a_cat, const int64_t *a_off,
                         const uint8_t *b_cat, const int64_t *b_off, int64_t count,
                         uint64_t *tickets, int64_t *n_submitted);

/* Poll `count` length-only tickets at once: for each finished one, len[k]
 * and status[k] (PACO_OK or its device error) are written and the ticket is
 * released; unfinished ones get status[k] = PACO_PENDING, unknown ones
 * PACO_ENOTFOUND.  *n_done (if not NULL) receives the number finished. */
int paco_lcs_poll_many(paco_ctx *ctx, const uint64_t *tickets, int64_t count, int32_t *len,
                       int32_t *status, int64_t *n_done);

/* Serving statistics since the context was created: requests submitted and
 * completed, cells computed, queue and in-flight counts, micro-batches
 * launched, device bytes held and the budget, and the worker threads' host
 * time (ns, summed over the workers) spent preparing and launching
 * micro-batches and collecting their results. */
typedef struct paco_serve_stats {
    uint64_t submitted, completed, cells_done;
    uint64_t queued_now, inflight_now, batches_launched;
    uint64_t bytes_in_use, bytes_budget;
    uint64_t host_launch_ns, host_complete_ns;
    uint64_t host_stage_ns, host_batch_ns;  /* parts of host_launch_ns: staging the strings, and
                                               planning and enqueueing the batch */
} paco_serve_stats;
int paco_serve_get_stats(paco_ctx *ctx, paco_serve_stats *out);

/* ---- subsequence recovery -------------------------------------------- */

/* One longest common subsequence of a (n, DEVICE) and b (m, DEVICE), not only
 * its length: the paper computes the length and names recovering the
 * subsequence as the harder variant (Sec. "PACO LCS", footnote to Eq. (1)).
 * Recovery is Hirschberg's linear-space divide and conquer (CACM 18(6),
 * 1975): each level cuts every subproblem at its middle row and finds the
 * best column of the cut from the forward bottom row of the upper half and
 * the bottom row of the reversed lower half, all subproblems of a level in
 * one batch launch; about 2 n m cells in all, O(n + m) device memory.
 * Output: *d_len = L, and DEVICE d_ai[0, L), d_bj[0, L) (capacity min(n, m))
 * with a[d_ai[k]] == b[d_bj[k]], both strictly increasing.  Which of the
 * longest subsequences is returned is fixed (the smallest best column at
 * every cut, the first equal column for a single row) but not part of the
 * contract.  Synchronous: returns when the result is in the buffers (the
 * call synchronises `stream` once per level); like every call on a context,
 * order it with the context's other calls. */
int paco_lcs_subsequence(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                         int32_t *d_ai, int32_t *d_bj, int32_t *d_len, void *stream);

/* ---- measurement helpers ---------------------------------------------- */

/* Device microbenchmark of the 32-bit integer ALU issue rate used as the
 * roofline denominator: runs independent chains of `op` (0 = IADD3-class
 * add, 1 = LOP3-class logic, 2 = integer max, 3 = the bit-parallel column
 * step mix) on every SM and writes lane-operations per second to *out. */
int paco_measure_int_peak(paco_ctx *ctx, int op, double *ops_per_s, void *stream);

/* Kernel time (ms, CUDA events on the launching stream) of the dominant
 * kernel of the last paco_lcs_* call on this context, and its name. */
int paco_last_kernel_ms(paco_ctx *ctx, double *ms, const char **name);

#ifdef __cplusplus
}
#endif

#endif /* PACO_LCS_H */
