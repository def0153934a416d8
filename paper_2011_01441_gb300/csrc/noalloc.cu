// paco_lcs_boundaries_static: the single-pair path without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they need an
// LCS: code that runs as a plugin or callback inside another framework that
// owns every device allocation through its own pool (and may not be
// re-entered), or a latency-critical loop where cudaMalloc/cudaFree would
// synchronise the whole device.  This entry point serves them: the caller
// passes device inputs and outputs only, and all scratch the strip pipeline
// needs (boundary step bits, tagged carry rows, the ticket and error
// words) lives in one file-scope __device__ array of fixed
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
void *g_scratch[kMaxDevices] = {};  // device address of g_static_scratch, per device
int g_sms[kMaxDevices] = {};
std::atomic<uint32_t> g_epoch{0x40000000u};

// Set-up, once per device with that device current: resolve the array's
// device address (the host-side name is only a stand-in for it).
int device_scratch(int dev, void **ptr, int *sms) {
    if (dev < 0 || dev >= kMaxDevices) return PACO_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return PACO_EDEVICE;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PACO_EDEVICE;
        g_scratch[dev] = p;
        g_sms[dev] = n;
    }
    *ptr = g_scratch[dev];
    *sms = g_sms[dev];
    return PACO_OK;
}

__global__ void k_error_to_len(const int *err, int32_t *len) {
    if (*err != 0 && len) *len = *err;
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
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PACO_EDEVICE;
    void *base = nullptr;
    int sms = 0;
    int rc = device_scratch(dev, &base, &sms);
    if (rc != PACO_OK) return rc;
    unsigned char *scr = (unsigned char *)base;
    int *small = (int *)scr;  // [0] ticket, [1] error word
    size_t used = 256;
    cudaError_t e = cudaMemsetAsync(small, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return PACO_EDEVICE;
    if (n == 0 || m == 0) {
        e = launch_degenerate(nullptr, nullptr, n, m, d_bottom_row, d_right_col, d_len, small + 1, st);
        return e == cudaSuccess ? PACO_OK : PACO_EDEVICE;
    }

    PairPlanOptions o;
    o.max_warps = pair_max_warps(1);
    PairPlan pl;
    if (!plan_pair(n, m, sms, o, pl)) return PACO_EINVAL;
    o.resident = sms * std::max(1, pair_occupancy(pl.C, pl.W, pl.wpl));
    if (!plan_pair(n, m, sms, o, pl)) return PACO_EINVAL;
    const int occ = std::max(1, pair_occupancy(pl.C, pl.W, pl.wpl));
    const int64_t L = pl.L, S = pl.S;
    const int64_t nwords = (S + 31) / 32, hstride = (nwords + 1) & ~(int64_t)1;
    const int64_t lwords = (L + 31) / 32, rwords = (L + 30) / 31;
    const int64_t nblocks = ((std::max(L, S) + 30) / 31 + 1023) / 1024 + 1;
    const size_t off_hbuf = used;
    used = align_up(used + (size_t)(pl.nstrips + 1) * hstride * 8 + 16);
    const size_t off_lbits = used;
    used = align_up(used + (size_t)lwords * 4 + 16);
    const size_t off_rbits = used;
    used = align_up(used + (size_t)rwords * 4 + 16);
    const size_t off_sums = used;
    used = align_up(used + (size_t)nblocks * 8 * 2);
    if (used > kStaticScratchBytes) return PACO_EINVAL;  // table too large for the fixed scratch

    uint32_t epoch = g_epoch.fetch_add(1) + 1;
    if (epoch == 0 || epoch == 0x80000000u) epoch = g_epoch.fetch_add(1) + 1;
    const bool tr = pl.transpose;
    const uint8_t *ka = tr ? b : a, *kb = tr ? a : b;
    int32_t *kbottom = tr ? d_right_col : d_bottom_row;
    int32_t *kright = tr ? d_bottom_row : d_right_col;
    uint64_t *hbuf = (uint64_t *)(scr + off_hbuf);
    e = launch_boundary_bits(nullptr, L, (uint32_t *)(scr + off_lbits), nullptr, epoch, nullptr, small + 1, st);
    if (e == cudaSuccess) e = launch_boundary_bits(nullptr, S, nullptr, hbuf, epoch, nullptr, small + 1, st);
    if (e != cudaSuccess) return PACO_EDEVICE;

    PairArgs P;
    P.a = ka;
    P.b = kb;
    P.L = L;
    P.S = S;
    P.nwords = nwords;
    P.hstride = hstride;
    P.strip_row0 = nullptr;
    P.granules = (L + 31 * pl.wpl - 1) / (31 * pl.wpl);
    P.nstrips = pl.nstrips;
    P.sigma = kMaxSigma;
    P.left_bits = (const uint32_t *)(scr + off_lbits);
    P.right_bits = (uint32_t *)(scr + off_rbits);
    P.hbuf = hbuf;
    P.ticket = small;
    P.err = small + 1;
    P.epoch = epoch;
    P.wait_limit_ns = 2000000000LL;
    P.stall_strip = -1;
    const int grid = std::min(pl.nstrips, sms * occ);
    e = launch_pair_bp(P, pl.C, pl.W, pl.wpl, grid, st);
    if (e != cudaSuccess) return PACO_EDEVICE;
    PrefixScratch s1{(int64_t *)(scr + off_sums), nblocks};
    e = launch_bits_prefix(nullptr, hbuf + (size_t)pl.nstrips * hstride, S, 32, nullptr, 0, kbottom, d_len, s1,
                           st);
    if (e == cudaSuccess && kright) {
        PrefixScratch s2{(int64_t *)(scr + off_sums) + nblocks, nblocks};
        e = launch_bits_prefix((const uint32_t *)(scr + off_rbits), nullptr, L, 31, nullptr, 0, kright, nullptr,
                               s2, st);
    }
    if (e != cudaSuccess) return PACO_EDEVICE;
    k_error_to_len<<<1, 1, 0, st>>>(small + 1, d_len);
    return cudaGetLastError() == cudaSuccess ? PACO_OK : PACO_EDEVICE;
}
