// Serving: continuous batching of LCS requests under a device-memory budget.
//
// paco_lcs_submit copies a request's strings into pinned host arenas (one
// for the a strings, one for the b strings, each a FIFO ring) and returns a
// ticket (paco_lcs_submit_many copies a large submission's strings with a
// few helper threads).  One worker thread per stream slot (kStreams of them)
// admits queued requests while the device budget allows, packs them into a
// micro-batch and launches it (the batch engine, one persistent launch) on
// its slot's stream, so micro-batches overlap on the device and their host
// preparation runs in parallel.  Requests are admitted in submission order, so a
// micro-batch's strings are one or two contiguous runs of each arena and go
// to the device in as many copies, straight from where submit put them.
// When a micro-batch's completion event fires its results are copied into
// the requests, their budget is released and their arena space reclaimed;
// paco_lcs_poll returns PACO_PENDING until then.
#include "../../include/paco_lcs.h"
#include "ctx.hpp"
#include "paco_internal.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace paco {

namespace {

constexpr int kStreams = 8;
constexpr size_t kMaxQueued = 1u << 20;
constexpr int32_t kMaxBatchPairs = 8192;
// Up to ~2.5 ms of device work per micro-batch at the batch kernel's rate on
// the serving mix.  A micro-batch lasts at least as long as its longest
// chain of segments (a tall pair), so small ones leave the device idle
// around that chain: on the 100k-request serving mix, caps of 2e10 / 6e10 /
// 2e11 cells served 52 / 62 / 64 TCUPS at the saturating rate, with lower
// latency too (p99 at 0.9 of it 40 / 27 / 26 ms).  Under light load the cap
// does not bind: a worker takes what has arrived.
constexpr int64_t kMaxBatchCells = 200000000000LL;
// Pinned arena per string side (a, b).
constexpr size_t kArenaBytes = (size_t)256 << 20;

enum ReqState { kQueued, kRunning, kDone };

struct Request {
    uint64_t ticket = 0;
    uint64_t a_pos = 0, b_pos = 0;  // logical arena positions of the strings
    int64_t n = 0, m = 0;
    bool want = false;
    ReqState state = kQueued;
    int status = PACO_OK;
    int32_t len = 0;
    std::vector<int32_t> row, col;
    size_t bytes = 0;
};

// Device bytes a request holds while admitted: its strings, column-table
// offsets, carry rows and (optionally) its boundaries and step words.
size_t request_bytes(int64_t n, int64_t m, bool want) {
    const int64_t L = n > m ? n : m, S = n > m ? m : n;
    size_t b = (size_t)(n + m) * 5 + 256;
    b += (size_t)((L + 991) / 992) * (size_t)(((S + 31) / 32 + 2) * 8);
    if (want) b += (size_t)(n + m + 2) * 4 + (size_t)((L + 30) / 31 + 32) * 4 + (size_t)(S / 8 + 8);
    return b;
}

// A FIFO ring of pinned host memory.  Positions are logical (they only
// grow); a string never straddles the physical end: when it would, the rest
// of the lap is skipped.  `tail` is the oldest byte still needed.
struct Arena {
    uint8_t *mem = nullptr;
    size_t cap = 0;
    uint64_t head = 0;
    uint64_t tail = 0;
    // Reserve n contiguous bytes; false when the ring is full.
    bool reserve(int64_t n, uint64_t *pos) {
        uint64_t p = head;
        if ((size_t)(p % cap) + (size_t)n > cap) p += cap - (size_t)(p % cap);  // skip to the next lap
        if (p + (uint64_t)n - tail > cap) return false;
        *pos = p;
        head = p + (uint64_t)n;
        return true;
    }
    uint8_t *at(uint64_t pos) { return mem + (size_t)(pos % cap); }
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    BatchState *B = nullptr;
    DevBuf small;             // ticket + error word
    DevBuf a, b, len, rows, cols;
    // pinned results
    int32_t *h_len = nullptr, *h_rows = nullptr, *h_cols = nullptr;
    int *h_err = nullptr;
    size_t cap_rows = 0, cap_cols = 0, cap_pairs = 0;
    std::vector<Request *> reqs;
    std::vector<int64_t> a_off, b_off, row_off, col_off;
    bool busy = false;
    size_t bytes = 0;
    uint64_t seq = 0;  // admission number of the micro-batch (arena reclaim order)
};

// The string copies of a large submission.  Copying the strings into the
// pinned arenas is the ingest path's main cost (one core copies about
// 10 GB/s, which capped serving near 600k requests/s on the serving mix), so
// a submission of many bytes is copied by the submitting thread and
// kCopyThreads helpers together, in pieces of at most kCopyPiece bytes taken
// from one atomic counter.
constexpr int kCopyThreads = 3;
constexpr size_t kCopyPiece = (size_t)1 << 20;
constexpr size_t kCopyParallelMin = (size_t)4 << 20;  // smaller submissions copy on the caller's thread
constexpr int64_t kSubmitGroup = 512;                  // requests published together (workers start early)

struct CopyPiece {
    uint8_t *dst;
    const uint8_t *src;
    size_t n;
};

struct CopyPool {
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::thread th[kCopyThreads];
    const std::vector<CopyPiece> *pieces = nullptr;
    std::atomic<size_t> next{0};
    int pending = 0;   // helpers still on the current generation
    uint64_t gen = 0;
    bool stop = false;
    void work() {
        const std::vector<CopyPiece> &p = *pieces;
        for (;;) {
            const size_t i = next.fetch_add(1, std::memory_order_relaxed);
            if (i >= p.size()) break;
            std::memcpy(p[i].dst, p[i].src, p[i].n);
        }
    }
    void helper() {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || gen != seen; });
                if (stop) return;
                seen = gen;
            }
            work();
            std::lock_guard<std::mutex> lk(mu);
            if (--pending == 0) done_cv.notify_all();
        }
    }
    void start() {
        for (auto &t : th) t = std::thread(&CopyPool::helper, this);
    }
    void run(const std::vector<CopyPiece> &p) {  // the caller copies too; returns when every piece is done
        {
            std::lock_guard<std::mutex> lk(mu);
            pieces = &p;
            next.store(0, std::memory_order_relaxed);
            pending = kCopyThreads;
            ++gen;
        }
        cv.notify_all();
        work();
        std::unique_lock<std::mutex> lk(mu);
        done_cv.wait(lk, [&] { return pending == 0; });
        pieces = nullptr;
    }
    void shutdown() {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_all();
        for (auto &t : th)
            if (t.joinable()) t.join();
    }
};

// Arena space of one admitted micro-batch, reclaimed in admission order.
struct Held {
    uint64_t seq, a_end, b_end;
    bool done;
};

}  // namespace

struct ServeEngine {
    paco_ctx *ctx = nullptr;
    std::mutex mu;       // queue, request table, budget, stats, arena tails, reclaim list
    std::mutex sub_mu;   // submitters: arena reservation and copy, in ticket order
    std::condition_variable cv;
    std::deque<Request *> queue;
    // every live request, indexed by ticket: tickets are handed out in
    // order, so the table is a deque whose front is ticket `base`; released
    // entries become null and the front is trimmed
    std::deque<std::unique_ptr<Request>> table;
    uint64_t base = 1;
    Request *find(uint64_t t) {
        if (t < base || t - base >= table.size()) return nullptr;
        return table[(size_t)(t - base)].get();
    }
    void release(uint64_t t) {
        table[(size_t)(t - base)].reset();
        while (!table.empty() && !table.front()) {
            table.pop_front();
            ++base;
        }
    }
    uint64_t next_ticket = 1;
    Arena arena_a, arena_b;   // heads move under sub_mu and mu, tails under mu
    std::deque<Held> held;
    uint64_t next_seq = 0;
    size_t budget = 0, in_use = 0;
    bool stop = false;
    std::thread workers[kStreams];
    Slot slots[kStreams];
    CopyPool copier;   // used under sub_mu
    paco_serve_stats stats{};
    int init_status = PACO_OK;
};

namespace {

int grow_pinned(void **p, size_t *cap, size_t need) {
    if (*cap >= need) return PACO_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    size_t want = need < 4096 ? 4096 : need * 2;
    if (cudaMallocHost(p, want) != cudaSuccess) {
        *cap = 0;
        return PACO_ENOMEM;
    }
    *cap = want;
    return PACO_OK;
}

// Stream-ordered growth of a slot's device buffer (no device-wide sync).
int grow_dev(DevBuf &d, size_t need, cudaStream_t st) {
    if (d.bytes >= need) return PACO_OK;
    if (d.ptr) cudaFreeAsync(d.ptr, st);
    d.ptr = nullptr;
    d.bytes = 0;
    size_t want = need < 4096 ? 4096 : need * 2;
    if (cudaMallocAsync(&d.ptr, want, st) != cudaSuccess) return PACO_ENOMEM;
    d.bytes = want;
    return PACO_OK;
}

// One side's strings of a micro-batch to the device: the runs of requests
// whose strings follow each other in the arena, one copy per run.  A run
// ends at the arena's physical end: a string that starts a new lap at
// offset 0 follows the previous one logically but not in memory.
cudaError_t copy_side(Arena &ar, const std::vector<Request *> &reqs, bool side_a, uint8_t *dst, cudaStream_t st) {
    size_t k = 0, out = 0;
    while (k < reqs.size()) {
        const uint64_t start = side_a ? reqs[k]->a_pos : reqs[k]->b_pos;
        uint64_t end = start;
        size_t j = k;
        while (j < reqs.size()) {
            const uint64_t p = side_a ? reqs[j]->a_pos : reqs[j]->b_pos;
            const int64_t len = side_a ? reqs[j]->n : reqs[j]->m;
            if (p != end || (j > k && p % ar.cap == 0)) break;
            end = p + (uint64_t)len;
            ++j;
        }
        if (end > start) {
            cudaError_t e = cudaMemcpyAsync(dst + out, ar.at(start), (size_t)(end - start), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return e;
            out += (size_t)(end - start);
        }
        k = j;
    }
    return cudaSuccess;
}

// Launch slot s with the admitted requests in it (engine lock not held).
int launch_slot(ServeEngine *E, Slot &S, uint64_t *stage_ns, uint64_t *batch_ns) {
    const auto t_stage = std::chrono::steady_clock::now();
    const int32_t np = (int32_t)S.reqs.size();
    S.a_off.assign((size_t)np + 1, 0);
    S.b_off.assign((size_t)np + 1, 0);
    S.row_off.assign((size_t)np, 0);
    S.col_off.assign((size_t)np, 0);
    bool any_want = false;
    int64_t rows_tot = 0, cols_tot = 0;
    for (int32_t k = 0; k < np; ++k) {
        Request *r = S.reqs[(size_t)k];
        S.a_off[(size_t)k + 1] = S.a_off[(size_t)k] + r->n;
        S.b_off[(size_t)k + 1] = S.b_off[(size_t)k] + r->m;
        S.row_off[(size_t)k] = rows_tot;
        S.col_off[(size_t)k] = cols_tot;
        rows_tot += r->m + 1;
        cols_tot += r->n + 1;
        any_want |= r->want;
    }
    const size_t na = (size_t)S.a_off[(size_t)np], nb = (size_t)S.b_off[(size_t)np];
    size_t cap = S.cap_pairs;
    if (grow_pinned((void **)&S.h_len, &cap, (size_t)np * 4 + 16) != PACO_OK) return PACO_ENOMEM;
    S.cap_pairs = cap;
    if (any_want) {
        cap = S.cap_rows;
        if (grow_pinned((void **)&S.h_rows, &cap, (size_t)rows_tot * 4 + 16) != PACO_OK) return PACO_ENOMEM;
        S.cap_rows = cap;
        cap = S.cap_cols;
        if (grow_pinned((void **)&S.h_cols, &cap, (size_t)cols_tot * 4 + 16) != PACO_OK) return PACO_ENOMEM;
        S.cap_cols = cap;
    }
    if (grow_dev(S.a, na + 16, S.stream) != PACO_OK || grow_dev(S.b, nb + 16, S.stream) != PACO_OK ||
        grow_dev(S.len, (size_t)np * 4 + 16, S.stream) != PACO_OK)
        return PACO_ENOMEM;
    if (any_want && (grow_dev(S.rows, (size_t)rows_tot * 4 + 16, S.stream) != PACO_OK ||
                     grow_dev(S.cols, (size_t)cols_tot * 4 + 16, S.stream) != PACO_OK))
        return PACO_ENOMEM;
    cudaError_t e = copy_side(E->arena_a, S.reqs, true, (uint8_t *)S.a.ptr, S.stream);
    if (e == cudaSuccess) e = copy_side(E->arena_b, S.reqs, false, (uint8_t *)S.b.ptr, S.stream);
    if (e != cudaSuccess) return PACO_EDEVICE;
    const auto t_batch = std::chrono::steady_clock::now();
    *stage_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(t_batch - t_stage).count();
    int rc = run_batch(E->ctx, S.B, (const uint8_t *)S.a.ptr, S.a_off.data(), (const uint8_t *)S.b.ptr,
                       S.b_off.data(), np, (int32_t *)S.len.ptr, any_want ? (int32_t *)S.rows.ptr : nullptr,
                       S.row_off.data(), any_want ? (int32_t *)S.cols.ptr : nullptr, S.col_off.data(), S.stream,
                       false, 0, E->ctx->opt_alphabet);
    *batch_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() -
                                                                               t_batch).count();
    if (rc != PACO_OK) return rc;
    e = cudaMemcpyAsync(S.h_len, S.len.ptr, (size_t)np * 4, cudaMemcpyDeviceToHost, S.stream);
    if (e == cudaSuccess && any_want)
        e = cudaMemcpyAsync(S.h_rows, S.rows.ptr, (size_t)rows_tot * 4, cudaMemcpyDeviceToHost, S.stream);
    if (e == cudaSuccess && any_want)
        e = cudaMemcpyAsync(S.h_cols, S.cols.ptr, (size_t)cols_tot * 4, cudaMemcpyDeviceToHost, S.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.h_err, (int *)S.small.ptr + 1, sizeof(int), cudaMemcpyDeviceToHost, S.stream);
    if (e == cudaSuccess) e = cudaEventRecord(S.done, S.stream);
    return e == cudaSuccess ? PACO_OK : PACO_EDEVICE;
}

void complete_slot(ServeEngine *E, Slot &S, int launch_rc) {
    const int dev_err = (launch_rc == PACO_OK && S.h_err) ? *S.h_err : 0;
    if (dev_err != 0) cudaMemsetAsync((int *)S.small.ptr + 1, 0, sizeof(int), S.stream);
    // The slot's requests are this worker's until they are marked done, so
    // their results are filled in without the engine lock (which the
    // submitters and pollers need).
    uint64_t cells = 0;
    for (size_t k = 0; k < S.reqs.size(); ++k) {
        Request *r = S.reqs[k];
        r->status = launch_rc != PACO_OK ? launch_rc : dev_err;
        if (r->status == PACO_OK) {
            r->len = S.h_len[k];
            if (r->want) {
                r->row.assign(S.h_rows + S.row_off[k], S.h_rows + S.row_off[k] + r->m + 1);
                r->col.assign(S.h_cols + S.col_off[k], S.h_cols + S.col_off[k] + r->n + 1);
            }
            cells += (uint64_t)r->n * (uint64_t)r->m;
        }
    }
    std::lock_guard<std::mutex> lk(E->mu);
    for (Request *r : S.reqs) r->state = kDone;
    E->stats.cells_done += cells;
    E->stats.completed += S.reqs.size();
    E->in_use -= S.bytes;
    E->stats.inflight_now -= S.reqs.size();
    // reclaim the arena space of the micro-batches completed so far, oldest first
    for (Held &h : E->held)
        if (h.seq == S.seq) h.done = true;
    while (!E->held.empty() && E->held.front().done) {
        E->arena_a.tail = E->held.front().a_end;
        E->arena_b.tail = E->held.front().b_end;
        E->held.pop_front();
    }
    S.bytes = 0;
    S.reqs.clear();
    S.busy = false;
    E->stats.bytes_in_use = E->in_use;
}

// Admit the queue's front requests into slot S while the budget allows (at
// most kMaxBatchPairs pairs and about kMaxBatchCells cells); E->mu held.
void admit(ServeEngine *E, Slot &S) {
    int64_t cells = 0;
    uint64_t a_end = 0, b_end = 0;
    while (!E->queue.empty() && (int32_t)S.reqs.size() < kMaxBatchPairs) {
        Request *r = E->queue.front();
        const int64_t c = r->n * r->m;
        if (!S.reqs.empty() && cells + c > kMaxBatchCells) break;
        if (E->in_use + r->bytes > E->budget) break;  // wait for memory to free up
        E->queue.pop_front();
        r->state = kRunning;
        E->in_use += r->bytes;
        S.bytes += r->bytes;
        S.reqs.push_back(r);
        cells += c;
        a_end = r->a_pos + (uint64_t)r->n;
        b_end = r->b_pos + (uint64_t)r->m;
    }
    if (!S.reqs.empty()) {
        S.seq = E->next_seq++;
        E->held.push_back(Held{S.seq, a_end, b_end, false});
    }
    E->stats.queued_now = E->queue.size();
    E->stats.bytes_in_use = E->in_use;
}

uint64_t ns_since(std::chrono::steady_clock::time_point t0) {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
        .count();
}

// One worker per stream slot: take the next micro-batch from the queue (FIFO
// across the workers), prepare and launch it, wait for it, hand its results
// to the requests.  Host preparation of one slot overlaps the device work of
// the others.
void slot_main(ServeEngine *E, int k) {
    cudaSetDevice(E->ctx->device);
    Slot &S = E->slots[k];
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(E->mu);
            E->cv.wait(lk, [&] {
                return E->stop || (!E->queue.empty() && E->in_use + E->queue.front()->bytes <= E->budget);
            });
            if (E->stop) break;
            admit(E, S);
            if (S.reqs.empty()) continue;
            S.busy = true;
            E->stats.batches_launched += 1;
            E->stats.inflight_now += S.reqs.size();
        }
        E->cv.notify_one();  // more queued work: the next free worker takes it
        auto t0 = std::chrono::steady_clock::now();
        uint64_t stage_ns = 0, batch_ns = 0;
        const int rc = launch_slot(E, S, &stage_ns, &batch_ns);
        uint64_t ns = ns_since(t0);
        if (rc == PACO_OK) cudaEventSynchronize(S.done);
        t0 = std::chrono::steady_clock::now();
        complete_slot(E, S, rc);
        const uint64_t ns2 = ns_since(t0);
        {
            std::lock_guard<std::mutex> lk(E->mu);
            E->stats.host_launch_ns += ns;
            E->stats.host_complete_ns += ns2;
            E->stats.host_stage_ns += stage_ns;
            E->stats.host_batch_ns += batch_ns;
        }
        E->cv.notify_all();  // budget freed: another worker may admit
    }
}

// Copy a request's strings into the arenas and queue it (the caller holds
// sub_mu, so heads move in ticket order; the tails are read under mu).
// PACO_EBUSY when an arena, the queue or the budget cannot take it.
int enqueue(ServeEngine *E, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, bool want, uint64_t *ticket) {
    const size_t bytes = request_bytes(n, m, want);
    if (bytes > E->budget || (size_t)n > E->arena_a.cap || (size_t)m > E->arena_b.cap) return PACO_EBUSY;
    Arena ta, tb;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        if (E->queue.size() >= kMaxQueued) return PACO_EBUSY;
        ta = E->arena_a;
        tb = E->arena_b;
    }
    auto r = std::make_unique<Request>();
    if (!ta.reserve(n, &r->a_pos) || !tb.reserve(m, &r->b_pos)) return PACO_EBUSY;
    // the reserved bytes lie past every admitted request's, so no reader
    // touches them until this request is queued
    if (n) std::memcpy(ta.at(r->a_pos), a, (size_t)n);
    if (m) std::memcpy(tb.at(r->b_pos), b, (size_t)m);
    r->n = n;
    r->m = m;
    r->want = want;
    r->bytes = bytes;
    std::lock_guard<std::mutex> lk(E->mu);
    E->arena_a.head = ta.head;
    E->arena_b.head = tb.head;
    r->ticket = E->next_ticket++;
    *ticket = r->ticket;
    E->queue.push_back(r.get());
    E->table.push_back(std::move(r));
    E->stats.submitted += 1;
    E->stats.queued_now = E->queue.size();
    return PACO_OK;
}

// Queue requests k0 .. k1 - 1 of a concatenated submission (the caller holds
// sub_mu): reserve arena space for as many as fit, copy their strings (in
// parallel when there are many bytes), then publish them in ticket order in
// one critical section.  Returns how many were queued; *rc = PACO_EBUSY when
// an arena, the queue or the budget stopped it early.
int64_t enqueue_group(ServeEngine *E, const uint8_t *a_cat, const int64_t *a_off, const uint8_t *b_cat,
                      const int64_t *b_off, int64_t k0, int64_t k1, uint64_t *tickets, int *rc) {
    Arena ta, tb;
    size_t queued = 0;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        ta = E->arena_a;
        tb = E->arena_b;
        queued = E->queue.size();
    }
    std::vector<std::unique_ptr<Request>> reqs;
    reqs.reserve((size_t)(k1 - k0));
    std::vector<CopyPiece> pieces;
    size_t total = 0;
    auto add = [&](uint8_t *dst, const uint8_t *src, size_t n) {
        for (size_t o = 0; o < n; o += kCopyPiece) pieces.push_back({dst + o, src + o, std::min(kCopyPiece, n - o)});
        total += n;
    };
    for (int64_t k = k0; k < k1; ++k) {
        const int64_t n = a_off[k + 1] - a_off[k], m = b_off[k + 1] - b_off[k];
        const size_t bytes = request_bytes(n, m, false);
        if (bytes > E->budget || (size_t)n > ta.cap || (size_t)m > tb.cap || queued + reqs.size() >= kMaxQueued) {
            *rc = PACO_EBUSY;
            break;
        }
        auto r = std::make_unique<Request>();
        if (!ta.reserve(n, &r->a_pos) || !tb.reserve(m, &r->b_pos)) {
            *rc = PACO_EBUSY;
            break;
        }
        // the reserved bytes lie past every admitted request's, so no reader
        // touches them until the request is queued
        if (n) add(ta.at(r->a_pos), a_cat + a_off[k], (size_t)n);
        if (m) add(tb.at(r->b_pos), b_cat + b_off[k], (size_t)m);
        r->n = n;
        r->m = m;
        r->bytes = bytes;
        reqs.push_back(std::move(r));
    }
    if (reqs.empty()) return 0;
    if (total >= kCopyParallelMin) {
        E->copier.run(pieces);
    } else {
        for (const CopyPiece &c : pieces) std::memcpy(c.dst, c.src, c.n);
    }
    std::lock_guard<std::mutex> lk(E->mu);
    E->arena_a.head = ta.head;
    E->arena_b.head = tb.head;
    int64_t k = k0;
    for (auto &r : reqs) {
        r->ticket = E->next_ticket++;
        tickets[k++] = r->ticket;
        E->queue.push_back(r.get());
        E->table.push_back(std::move(r));
    }
    E->stats.submitted += reqs.size();
    E->stats.queued_now = E->queue.size();
    return (int64_t)reqs.size();
}

}  // namespace

ServeEngine *serve_get(paco_ctx *ctx, int *rc) {
    if (ctx->serve) {
        *rc = ctx->serve->init_status;
        return ctx->serve;
    }
    ServeEngine *E = new (std::nothrow) ServeEngine();
    if (!E) {
        *rc = PACO_ENOMEM;
        return nullptr;
    }
    E->ctx = ctx;
    E->budget = ctx->budget;
    E->stats.bytes_budget = ctx->budget;
    ctx->serve = E;
    if (cudaMallocHost((void **)&E->arena_a.mem, kArenaBytes) != cudaSuccess ||
        cudaMallocHost((void **)&E->arena_b.mem, kArenaBytes) != cudaSuccess) {
        *rc = PACO_ENOMEM;
        E->init_status = PACO_ENOMEM;
        return E;
    }
    E->arena_a.cap = E->arena_b.cap = kArenaBytes;
    for (auto &S : E->slots) {
        if (cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&S.small.ptr, 256) != cudaSuccess || cudaMemset(S.small.ptr, 0, 256) != cudaSuccess ||
            cudaMallocHost((void **)&S.h_err, 64) != cudaSuccess) {
            *rc = PACO_EDEVICE;
            E->init_status = PACO_EDEVICE;
            return E;
        }
        S.small.bytes = 256;
        *S.h_err = 0;
        // the lengths of a full micro-batch, pinned up front (growing pinned
        // memory later would stall the worker for milliseconds)
        if (grow_pinned((void **)&S.h_len, &S.cap_pairs, (size_t)kMaxBatchPairs * 4 + 16) != PACO_OK) {
            *rc = PACO_ENOMEM;
            E->init_status = PACO_ENOMEM;
            return E;
        }
        S.B = batch_state_new((int *)S.small.ptr, (int *)S.small.ptr + 1);
    }
    for (int k = 0; k < kStreams; ++k) E->workers[k] = std::thread(slot_main, E, k);
    E->copier.start();
    *rc = PACO_OK;
    return E;
}

void serve_shutdown(paco_ctx *ctx) {
    ServeEngine *E = ctx->serve;
    if (!E) return;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        E->stop = true;
    }
    E->cv.notify_all();
    for (auto &t : E->workers)
        if (t.joinable()) t.join();
    E->copier.shutdown();
    for (auto &S : E->slots) {
        if (S.stream) cudaStreamSynchronize(S.stream);
        batch_state_free(S.B);
        for (DevBuf *d : {&S.small, &S.a, &S.b, &S.len, &S.rows, &S.cols})
            if (d->ptr) cudaFree(d->ptr);
        for (void *h : {(void *)S.h_len, (void *)S.h_rows, (void *)S.h_cols, (void *)S.h_err})
            if (h) cudaFreeHost(h);
        if (S.done) cudaEventDestroy(S.done);
        if (S.stream) cudaStreamDestroy(S.stream);
    }
    if (E->arena_a.mem) cudaFreeHost(E->arena_a.mem);
    if (E->arena_b.mem) cudaFreeHost(E->arena_b.mem);
    delete E;
    ctx->serve = nullptr;
}

}  // namespace paco

extern "C" {

int paco_lcs_submit(paco_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                    int want_boundaries, uint64_t *ticket) {
    if (!ctx || !ticket || n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL) return PACO_EINVAL;
    if ((n > 0 && !a) || (m > 0 && !b)) return PACO_EINVAL;
    int rc = PACO_OK;
    paco::ServeEngine *E;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        E = paco::serve_get(ctx, &rc);
    }
    if (!E || rc != PACO_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(E->sub_mu);
        rc = paco::enqueue(E, a, n, b, m, want_boundaries != 0, ticket);
    }
    if (rc == PACO_OK) E->cv.notify_one();
    return rc;
}

int paco_lcs_submit_many(paco_ctx *ctx, const uint8_t *a_cat, const int64_t *a_off, const uint8_t *b_cat,
                         const int64_t *b_off, int64_t count, uint64_t *tickets, int64_t *n_submitted) {
    if (n_submitted) *n_submitted = 0;
    if (!ctx || count < 0 || (count > 0 && (!a_off || !b_off || !tickets))) return PACO_EINVAL;
    for (int64_t k = 0; k < count; ++k) {
        const int64_t n = a_off[k + 1] - a_off[k], m = b_off[k + 1] - b_off[k];
        if (n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL) return PACO_EINVAL;
        if ((n > 0 && !a_cat) || (m > 0 && !b_cat)) return PACO_EINVAL;
    }
    int rc = PACO_OK;
    paco::ServeEngine *E;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        E = paco::serve_get(ctx, &rc);
    }
    if (!E || rc != PACO_OK) return rc;
    int64_t taken = 0;
    {
        std::lock_guard<std::mutex> lk(E->sub_mu);
        while (taken < count && rc == PACO_OK) {
            const int64_t k1 = std::min(count, taken + paco::kSubmitGroup);
            const int64_t got = paco::enqueue_group(E, a_cat, a_off, b_cat, b_off, taken, k1, tickets, &rc);
            if (got) E->cv.notify_one();  // let a worker start on a long submission
            const bool partial = taken + got < k1;
            taken += got;
            if (partial) break;
        }
    }
    if (n_submitted) *n_submitted = taken;
    if (taken) E->cv.notify_one();
    return rc;
}

int paco_lcs_poll_many(paco_ctx *ctx, const uint64_t *tickets, int64_t count, int32_t *len, int32_t *status,
                       int64_t *n_done) {
    if (n_done) *n_done = 0;
    if (!ctx || count < 0 || (count > 0 && (!tickets || !len || !status))) return PACO_EINVAL;
    paco::ServeEngine *E = ctx->serve;
    if (!E) {
        for (int64_t k = 0; k < count; ++k) status[k] = PACO_ENOTFOUND;
        return PACO_OK;
    }
    int64_t done = 0;
    std::lock_guard<std::mutex> lk(E->mu);
    for (int64_t k = 0; k < count; ++k) {
        paco::Request *r = E->find(tickets[k]);
        if (!r) {
            status[k] = PACO_ENOTFOUND;
            continue;
        }
        if (r->state != paco::kDone) {
            status[k] = PACO_PENDING;
            continue;
        }
        status[k] = r->status;
        len[k] = r->status == PACO_OK ? r->len : 0;
        E->release(tickets[k]);
        ++done;
    }
    if (n_done) *n_done = done;
    return PACO_OK;
}

int paco_lcs_poll(paco_ctx *ctx, uint64_t ticket, int32_t *len, int32_t *row_out, int32_t *col_out) {
    if (!ctx) return PACO_EINVAL;
    paco::ServeEngine *E = ctx->serve;
    if (!E) return PACO_ENOTFOUND;
    std::lock_guard<std::mutex> lk(E->mu);
    paco::Request *r = E->find(ticket);
    if (!r) return PACO_ENOTFOUND;
    if (r->state != paco::kDone) return PACO_PENDING;
    const int st = r->status;
    if (st == PACO_OK) {
        if (len) *len = r->len;
        if (r->want) {
            if (row_out) std::memcpy(row_out, r->row.data(), r->row.size() * 4);
            if (col_out) std::memcpy(col_out, r->col.data(), r->col.size() * 4);
        }
    }
    E->release(ticket);
    return st;
}

int paco_serve_get_stats(paco_ctx *ctx, paco_serve_stats *out) {
    if (!ctx || !out) return PACO_EINVAL;
    paco::ServeEngine *E = ctx->serve;
    if (!E) {
        std::memset(out, 0, sizeof(*out));
        out->bytes_budget = ctx->budget;
        return PACO_OK;
    }
    std::lock_guard<std::mutex> lk(E->mu);
    *out = E->stats;
    out->queued_now = E->queue.size();
    return PACO_OK;
}

}  // extern "C"
