// Serving: continuous batching of LCS requests under a device-memory budget.
//
// paco_lcs_submit copies a request into the host queue and returns a ticket.
// A worker thread admits queued requests while the budget allows, packs the
// admitted ones into a micro-batch and launches it (the batch engine, one
// persistent launch) on one of kStreams streams, so micro-batches overlap on
// the device; when a micro-batch's completion event fires its results are
// copied into the requests and their budget is released.  paco_lcs_poll
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
#include <unordered_map>
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
    std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
    uint64_t next_ticket = 1;
    size_t budget = 0, in_use = 0;
    bool stop = false;
    std::thread worker;
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
int launch_slot(ServeEngine *E, Slot &S) {
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
    int rc = run_batch(E->ctx, S.B, (const uint8_t *)S.a.ptr, S.a_off.data(), (const uint8_t *)S.b.ptr,
                       S.b_off.data(), np, (int32_t *)S.len.ptr, any_want ? (int32_t *)S.rows.ptr : nullptr,
                       S.row_off.data(), any_want ? (int32_t *)S.cols.ptr : nullptr, S.col_off.data(), S.stream,
                       false, 0, E->ctx->opt_alphabet);
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
    std::lock_guard<std::mutex> lk(E->mu);
    for (size_t k = 0; k < S.reqs.size(); ++k) {
        Request *r = S.reqs[k];
        r->status = launch_rc != PACO_OK ? launch_rc : dev_err;
        if (r->status == PACO_OK) {
            r->len = S.h_len[k];
            if (r->want) {
                r->row.assign(S.h_rows + S.row_off[k], S.h_rows + S.row_off[k] + r->b.size() + 1);
                r->col.assign(S.h_cols + S.col_off[k], S.h_cols + S.col_off[k] + r->a.size() + 1);
            }
            E->stats.cells_done += (uint64_t)r->a.size() * r->b.size();
        }
        r->state = kDone;
        r->a.clear();
        r->a.shrink_to_fit();
        r->b.clear();
        r->b.shrink_to_fit();
        E->stats.completed += 1;
    }
    E->in_use -= S.bytes;
    S.bytes = 0;
    S.reqs.clear();
    S.busy = false;
    E->stats.inflight_now = 0;
    for (auto &sl : E->slots) E->stats.inflight_now += sl.reqs.size();
    E->stats.bytes_in_use = E->in_use;
}

void worker_main(ServeEngine *E) {
    cudaSetDevice(E->ctx->device);
    for (;;) {
        // completions
        for (auto &S : E->slots) {
            if (S.busy && cudaEventQuery(S.done) == cudaSuccess) {
                const auto t0 = std::chrono::steady_clock::now();
                complete_slot(E, S, PACO_OK);
                const uint64_t ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                                        std::chrono::steady_clock::now() - t0).count();
                std::lock_guard<std::mutex> lk(E->mu);
                E->stats.host_complete_ns += ns;
            }
        }
        // admission: fill one free slot from the queue
        Slot *free_slot = nullptr;
        {
            std::unique_lock<std::mutex> lk(E->mu);
            if (E->stop) break;
            for (auto &S : E->slots)
                if (!S.busy) {
                    free_slot = &S;
                    break;
                }
            if (free_slot && !E->queue.empty()) {
                int64_t cells = 0;
                while (!E->queue.empty() && (int32_t)free_slot->reqs.size() < kMaxBatchPairs) {
                    Request *r = E->queue.front();
                    const int64_t c = (int64_t)r->a.size() * (int64_t)r->b.size();
                    if (!free_slot->reqs.empty() && cells + c > kMaxBatchCells) break;
                    if (E->in_use + r->bytes > E->budget) break;  // wait for memory to free up
                    E->queue.pop_front();
                    r->state = kRunning;
                    E->in_use += r->bytes;
                    free_slot->bytes += r->bytes;
                    free_slot->reqs.push_back(r);
                    cells += c;
                }
                E->stats.queued_now = E->queue.size();
                E->stats.bytes_in_use = E->in_use;
            }
            if (!free_slot || free_slot->reqs.empty()) {
                bool any_busy = false;
                for (auto &S : E->slots) any_busy |= S.busy;
                // nothing to launch: sleep until a submit arrives or a short tick passes
                E->cv.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 500));
                continue;
            }
            free_slot->busy = true;
            E->stats.batches_launched += 1;
        }
        const auto t0 = std::chrono::steady_clock::now();
        const int rc = launch_slot(E, *free_slot);
        const uint64_t ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                                std::chrono::steady_clock::now() - t0).count();
        {
            std::lock_guard<std::mutex> lk(E->mu);
            E->stats.host_launch_ns += ns;
        }
        if (rc != PACO_OK) complete_slot(E, *free_slot, rc);
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
    E->worker = std::thread(worker_main, E);
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
    if (E->worker.joinable()) E->worker.join();
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
        E->all.emplace(r->ticket, std::move(r));
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
            E->all.emplace(r->ticket, std::move(r));
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
        auto it = E->all.find(tickets[k]);
        if (it == E->all.end()) {
            status[k] = PACO_ENOTFOUND;
            continue;
        }
        paco::Request *r = it->second.get();
        if (r->state != paco::kDone) {
            status[k] = PACO_PENDING;
            continue;
        }
        status[k] = r->status;
        len[k] = r->status == PACO_OK ? r->len : 0;
        E->all.erase(it);
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
    auto it = E->all.find(ticket);
    if (it == E->all.end()) return PACO_ENOTFOUND;
    paco::Request *r = it->second.get();
    if (r->state != paco::kDone) return PACO_PENDING;
    const int st = r->status;
    if (st == PACO_OK) {
        if (len) *len = r->len;
        if (r->want) {
            if (row_out) std::memcpy(row_out, r->row.data(), r->row.size() * 4);
            if (col_out) std::memcpy(col_out, r->col.data(), r->col.size() * 4);
        }
    }
    E->all.erase(it);
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
