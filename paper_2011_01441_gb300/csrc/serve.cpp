// Serving: continuous batching of LCS requests under a device-memory budget.
//
// paco_lcs_submit copies a request into the host queue and returns a ticket.
// One worker thread per stream slot (kStreams of them) admits queued
// requests while the budget allows, packs them into a micro-batch and
// launches it (the batch engine, one persistent launch) on its slot's
// stream, so micro-batches overlap on the device and their host preparation
// runs in parallel; when a micro-batch's completion event fires its results
// are copied into the requests and their budget is released.  paco_lcs_poll
// returns PACO_PENDING until then.
#include "../../include/paco_lcs.h"
#include "ctx.hpp"
#include "paco_internal.hpp"

#include <cuda_runtime.h>

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

constexpr int kStreams = 4;
constexpr size_t kMaxQueued = 1u << 20;
constexpr int32_t kMaxBatchPairs = 8192;
// Up to ~0.5 ms of device work per micro-batch at the batch kernel's rate:
// small enough for four to overlap, large enough to amortise each
// micro-batch's host work (layout, copies, launches).
constexpr int64_t kMaxBatchCells = 20000000000LL;

enum ReqState { kQueued, kRunning, kDone };

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> a, b;
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

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    BatchState *B = nullptr;
    DevBuf small;             // ticket + error word
    DevBuf a, b, len, rows, cols;
    // pinned staging
    uint8_t *h_a = nullptr, *h_b = nullptr;
    int32_t *h_len = nullptr, *h_rows = nullptr, *h_cols = nullptr;
    int *h_err = nullptr;
    size_t cap_a = 0, cap_b = 0, cap_rows = 0, cap_cols = 0, cap_pairs = 0;
    std::vector<Request *> reqs;
    std::vector<int64_t> a_off, b_off, row_off, col_off;
    bool busy = false;
    size_t bytes = 0;
};

}  // namespace

struct ServeEngine {
    paco_ctx *ctx = nullptr;
    std::mutex mu;
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
    size_t budget = 0, in_use = 0;
    bool stop = false;
    std::thread workers[kStreams];
    Slot slots[kStreams];
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

int grow_dev(DevBuf &d, size_t need) {
    if (d.bytes >= need) return PACO_OK;
    if (d.ptr) cudaFree(d.ptr);
    d.ptr = nullptr;
    d.bytes = 0;
    size_t want = need < 4096 ? 4096 : need * 2;
    if (cudaMalloc(&d.ptr, want) != cudaSuccess) return PACO_ENOMEM;
    d.bytes = want;
    return PACO_OK;
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
        S.a_off[(size_t)k + 1] = S.a_off[(size_t)k] + (int64_t)r->a.size();
        S.b_off[(size_t)k + 1] = S.b_off[(size_t)k] + (int64_t)r->b.size();
        S.row_off[(size_t)k] = rows_tot;
        S.col_off[(size_t)k] = cols_tot;
        rows_tot += (int64_t)r->b.size() + 1;
        cols_tot += (int64_t)r->a.size() + 1;
        any_want |= r->want;
    }
    const size_t na = (size_t)S.a_off[(size_t)np], nb = (size_t)S.b_off[(size_t)np];
    size_t cap;
    cap = S.cap_a;
    if (grow_pinned((void **)&S.h_a, &cap, na + 16) != PACO_OK) return PACO_ENOMEM;
    S.cap_a = cap;
    cap = S.cap_b;
    if (grow_pinned((void **)&S.h_b, &cap, nb + 16) != PACO_OK) return PACO_ENOMEM;
    S.cap_b = cap;
    cap = S.cap_pairs;
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
    for (int32_t k = 0; k < np; ++k) {
        Request *r = S.reqs[(size_t)k];
        if (!r->a.empty()) std::memcpy(S.h_a + S.a_off[(size_t)k], r->a.data(), r->a.size());
        if (!r->b.empty()) std::memcpy(S.h_b + S.b_off[(size_t)k], r->b.data(), r->b.size());
    }
    if (grow_dev(S.a, na + 16) != PACO_OK || grow_dev(S.b, nb + 16) != PACO_OK ||
        grow_dev(S.len, (size_t)np * 4 + 16) != PACO_OK)
        return PACO_ENOMEM;
    if (any_want && (grow_dev(S.rows, (size_t)rows_tot * 4 + 16) != PACO_OK ||
                     grow_dev(S.cols, (size_t)cols_tot * 4 + 16) != PACO_OK))
        return PACO_ENOMEM;
    cudaError_t e = cudaSuccess;
    if (na) e = cudaMemcpyAsync(S.a.ptr, S.h_a, na, cudaMemcpyHostToDevice, S.stream);
    if (e == cudaSuccess && nb) e = cudaMemcpyAsync(S.b.ptr, S.h_b, nb, cudaMemcpyHostToDevice, S.stream);
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
    // their results are filled in and their strings freed without the engine
    // lock (which the submitters and pollers need).
    uint64_t cells = 0;
    for (size_t k = 0; k < S.reqs.size(); ++k) {
        Request *r = S.reqs[k];
        r->status = launch_rc != PACO_OK ? launch_rc : dev_err;
        if (r->status == PACO_OK) {
            r->len = S.h_len[k];
            if (r->want) {
                r->row.assign(S.h_rows + S.row_off[k], S.h_rows + S.row_off[k] + r->b.size() + 1);
                r->col.assign(S.h_cols + S.col_off[k], S.h_cols + S.col_off[k] + r->a.size() + 1);
            }
            cells += (uint64_t)r->a.size() * r->b.size();
        }
        std::vector<uint8_t>().swap(r->a);
        std::vector<uint8_t>().swap(r->b);
    }
    std::lock_guard<std::mutex> lk(E->mu);
    for (Request *r : S.reqs) r->state = kDone;
    E->stats.cells_done += cells;
    E->stats.completed += S.reqs.size();
    E->in_use -= S.bytes;
    E->stats.inflight_now -= S.reqs.size();
    S.bytes = 0;
    S.reqs.clear();
    S.busy = false;
    E->stats.bytes_in_use = E->in_use;
}

// Admit the queue's front requests into slot S while the budget allows (at
// most kMaxBatchPairs pairs and about kMaxBatchCells cells); E->mu held.
void admit(ServeEngine *E, Slot &S) {
    int64_t cells = 0;
    while (!E->queue.empty() && (int32_t)S.reqs.size() < kMaxBatchPairs) {
        Request *r = E->queue.front();
        const int64_t c = (int64_t)r->a.size() * (int64_t)r->b.size();
        if (!S.reqs.empty() && cells + c > kMaxBatchCells) break;
        if (E->in_use + r->bytes > E->budget) break;  // wait for memory to free up
        E->queue.pop_front();
        r->state = kRunning;
        E->in_use += r->bytes;
        S.bytes += r->bytes;
        S.reqs.push_back(r);
        cells += c;
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
    for (auto &S : E->slots) {
        if (cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&S.small.ptr, 256) != cudaSuccess || cudaMemset(S.small.ptr, 0, 256) != cudaSuccess ||
            cudaMallocHost((void **)&S.h_err, 64) != cudaSuccess) {
            *rc = PACO_EDEVICE;
            E->init_status = PACO_EDEVICE;
            ctx->serve = E;
            return E;
        }
        S.small.bytes = 256;
        *S.h_err = 0;
        S.B = batch_state_new((int *)S.small.ptr, (int *)S.small.ptr + 1);
    }
    ctx->serve = E;
    for (int k = 0; k < kStreams; ++k) E->workers[k] = std::thread(slot_main, E, k);
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
    for (auto &S : E->slots) {
        if (S.stream) cudaStreamSynchronize(S.stream);
        batch_state_free(S.B);
        for (DevBuf *d : {&S.small, &S.a, &S.b, &S.len, &S.rows, &S.cols})
            if (d->ptr) cudaFree(d->ptr);
        for (void *h : {(void *)S.h_a, (void *)S.h_b, (void *)S.h_len, (void *)S.h_rows, (void *)S.h_cols,
                        (void *)S.h_err})
            if (h) cudaFreeHost(h);
        if (S.done) cudaEventDestroy(S.done);
        if (S.stream) cudaStreamDestroy(S.stream);
    }
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
    const size_t bytes = paco::request_bytes(n, m, want_boundaries != 0);
    if (bytes > E->budget) return PACO_EBUSY;
    auto r = std::make_unique<paco::Request>();
    r->a.assign(a, a + n);
    r->b.assign(b, b + m);
    r->want = want_boundaries != 0;
    r->bytes = bytes;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        if (E->queue.size() >= paco::kMaxQueued) return PACO_EBUSY;
        r->ticket = E->next_ticket++;
        *ticket = r->ticket;
        E->queue.push_back(r.get());
        E->table.push_back(std::move(r));
        E->stats.submitted += 1;
        E->stats.queued_now = E->queue.size();
    }
    E->cv.notify_one();
    return PACO_OK;
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
    // copy the strings outside the engine lock
    std::vector<std::unique_ptr<paco::Request>> rs;
    rs.reserve((size_t)count);
    for (int64_t k = 0; k < count; ++k) {
        const int64_t n = a_off[k + 1] - a_off[k], m = b_off[k + 1] - b_off[k];
        auto r = std::make_unique<paco::Request>();
        r->a.assign(a_cat + a_off[k], a_cat + a_off[k] + n);
        r->b.assign(b_cat + b_off[k], b_cat + b_off[k] + m);
        r->want = false;
        r->bytes = paco::request_bytes(n, m, false);
        rs.push_back(std::move(r));
    }
    int64_t taken = 0;
    rc = PACO_OK;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        for (auto &r : rs) {
            if (r->bytes > E->budget || E->queue.size() >= paco::kMaxQueued) {
                rc = PACO_EBUSY;
                break;
            }
            r->ticket = E->next_ticket++;
            tickets[taken++] = r->ticket;
            E->queue.push_back(r.get());
            E->table.push_back(std::move(r));
            E->stats.submitted += 1;
        }
        E->stats.queued_now = E->queue.size();
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
