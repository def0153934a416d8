// paco_lcs_boundaries_static: the single-pair path without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they need an
// LCS: code that runs as a plugin or callback inside another framework that
// owns every device allocation through its own pool (and may not be
// re-entered), or a latency-critical loop where cudaMalloc/cudaFree would
// synchronise the whole device.  This entry point serves them: the caller
// passes device inputs and outputs only, and all scratch the strip pipeline
// needs (the tagged carry rows, the ticket and error words) lives in one
// file-scope __device__ array of fixed
// size that every GPU loading this library keeps until the process exits.
//
// The array is shared by all calls on a device and keeps the previous call's
// contents, so each call clears the words that must start at zero.  Calls
// that overlap on the GPU (two streams, or two host threads) race on it;
// serialise them.
#include "../../include/paco_lcs.h"
#include "paco_internal.hpp"
#include "plan.hpp"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>

namespace paco {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int g_sms[kMaxDevices] = {};  // SM count per device, read once
std::atomic<uint32_t> g_epoch{0x40000000u};

// Set-up, with the device current: resolve the array's device address (the
// host-side name is only a stand-in for it).  The lookup allocates nothing
// and is repeated on every call, so a context that was torn down and made
// again on the device (cudaDeviceReset) gets the new address; only the
// first lookup on a device loads the module, which is why the first call
// should come before any stream capture.
int device_scratch(int dev, void **ptr, int *sms) {
    if (dev < 0 || dev >= kMaxDevices) return PACO_EINVAL;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return PACO_EDEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sms[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            return PACO_EDEVICE;
        g_sms[dev] = n;
    }
    *ptr = p;
    *sms = g_sms[dev];
    return PACO_OK;
}

// A device-side failure (a bounded wait that timed out) replaces L by its
// negative status, so the caller sees it in d_len.
__global__ void k_error_to_len(const int *err, int32_t *len) {
    if (*err != 0) *len = *err;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace paco

extern "C" int paco_lcs_boundaries_static(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                                          int32_t *d_bottom_row, int32_t *d_right_col, int32_t *d_len,
                                          void *stream) {
    using namespace paco;
    if (n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL) return PACO_EINVAL;
    if ((n > 0 && !a) || (m > 0 && !b)) return PACO_EINVAL;
    if (!d_len) return PACO_EINVAL;  // the only place a device-side error can be reported
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PACO_EDEVICE;
    void *base = nullptr;
    int sms = 0;
    int rc = device_scratch(dev, &base, &sms);
    if (rc != PACO_OK) return rc;
    unsigned char *scr = (unsigned char *)base;
    int *small = (int *)scr;  // [0] strip ticket, [1] exit count, [2] error word
    int *err = small + 2;
    size_t used = 256;
    cudaError_t e = cudaMemsetAsync(small, 0, 4 * sizeof(int), st);
    if (e != cudaSuccess) return PACO_EDEVICE;
    if (n == 0 || m == 0) {
        e = launch_degenerate(nullptr, nullptr, n, m, d_bottom_row, d_right_col, d_len, err, st);
        return e == cudaSuccess ? PACO_OK : PACO_EDEVICE;
    }

    PairPlanOptions o;
    o.max_warps = pair_max_warps(1);
    o.max_warps_wpl2 = pair_max_warps(2);
    PairPlan pl;
    if (!plan_pair(n, m, sms, o, pl)) return PACO_EINVAL;
    o.resident = sms * std::max(1, pair_occupancy(pl.C, pl.W, pl.wpl));
    if (!plan_pair(n, m, sms, o, pl)) return PACO_EINVAL;
    const int occ = std::max(1, pair_occupancy(pl.C, pl.W, pl.wpl));
    const int64_t L = pl.L, S = pl.S;
    const int64_t nwords = (S + 31) / 32, hstride = (nwords + 1) & ~(int64_t)1;
    const size_t off_hbuf = used;
    used = align_up(used + (size_t)(pl.nstrips + 1) * hstride * 8 + 16);
    if (used > kStaticScratchBytes) return PACO_EINVAL;  // table too large for the fixed scratch

    uint32_t epoch = g_epoch.fetch_add(1) + 1;
    if (epoch == 0 || epoch == 0x80000000u) epoch = g_epoch.fetch_add(1) + 1;
    const bool tr = pl.transpose;
    PairArgs P;
    P.a = tr ? b : a;
    P.b = tr ? a : b;
    P.L = L;
    P.S = S;
    P.nwords = (int32_t)nwords;
    P.hstride = hstride;
    P.granules = (L + 31 * pl.wpl - 1) / (31 * pl.wpl);
    P.uniform_rows = 0;
    P.nstrips = pl.nstrips;
    P.top = nullptr;
    P.left = nullptr;
    P.bottom = tr ? d_right_col : d_bottom_row;
    P.right = tr ? d_bottom_row : d_right_col;
    P.len = d_len;
    P.hbuf = (uint64_t *)(scr + off_hbuf);
    P.ctl = small;
    P.err = err;
    P.epoch = epoch;
    P.wait_limit_ns = 2000000000LL;
    P.stall_strip = -1;
    const int grid = std::min(pl.nstrips, sms * occ);
    e = launch_pair_bp(P, pl.C, pl.W, pl.wpl, grid, st);
    if (e != cudaSuccess) return PACO_EDEVICE;
    k_error_to_len<<<1, 1, 0, st>>>(err, d_len);
    return cudaGetLastError() == cudaSuccess ? PACO_OK : PACO_EDEVICE;
}
