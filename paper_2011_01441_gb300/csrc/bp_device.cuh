// Device helpers shared by the single-pair and batch kernels: relaxed
// global accesses, bounded polls, and the bit-parallel column step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "paco_internal.hpp"

namespace paco {
namespace dev {

constexpr uint32_t kFull = 0xffffffffu;

static __device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ int ld_relaxed_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
static __device__ __forceinline__ void raise_error(int *err, int code) { atomicCAS(err, 0, code); }

constexpr size_t kTableBytes = (size_t)kMaxSigma * 32 * sizeof(uint32_t);  // per warp

// One lane polls a global tagged word until its tag is `want`.  Bounded: on
// timeout or a raised error `ok` turns false (the caller ends the strip).
static __device__ __noinline__ uint64_t poll_global_lane(const uint64_t *p, uint32_t want, int *err,
                                                  long long limit, bool &ok) {
    uint64_t v = ld_relaxed_u64(p);
    if ((uint32_t)(v >> 32) == want) return v;
    const uint64_t t0 = global_ns();
    for (int spin = 0;; ++spin) {
        if (spin > 16) __nanosleep(32);
        v = ld_relaxed_u64(p);
        if ((uint32_t)(v >> 32) == want) return v;
        if (ld_relaxed_i32(err) != 0) {
            ok = false;
            return v;
        }
        if ((long long)(global_ns() - t0) > limit) {
            raise_error(err, kEtimeout);
            ok = false;
            return v;
        }
    }
}

// Lane 31 waits until the next warp has consumed ring word `need - 1`.
static __device__ __noinline__ bool wait_consumed(volatile int *cons, int need, int *err, long long limit) {
    if (*cons >= need) return true;
    const uint64_t t0 = global_ns();
    while (*cons < need) {
        if (ld_relaxed_i32(err) != 0) return false;
        if ((long long)(global_ns() - t0) > limit) {
            raise_error(err, kEtimeout);
            return false;
        }
    }
    return true;
}

constexpr int kLaneRows = 31;

// Shared-memory load at a 32-bit shared address.
static __device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// One column of Eq. (1) on a lane's 31 rows (bits 0..30), state (S, Y) with
// V = S | Y and bit 31 of V held at 1.  Then bit 31 of V + X + c is
// 1 + 0 + (carry out of row 30), so the carry
// flag of the 32-bit add is the lane's carry out; it is shifted straight
// into cw by a second add-with-carry, and V' = S' | Y' keeps bit 31 set
// through Y' = (S | Y) & ~M (M has no bit 31).
//   V = S | Y, X = (S|Y) & M, Y' = (S|Y) & ~M                  (three LOP3)
//   CC = top bit of sr; S' = V + X + CC, CC = carry out; cw = 2 cw + CC
static __device__ __forceinline__ void column31c(uint32_t &S, uint32_t &Y, uint32_t &sr, uint32_t &cw,
                                          uint32_t M) {
    uint32_t V, X, Yn;
    asm("lop3.b32 %0, %1, %2, 0, 0xFC;" : "=r"(V) : "r"(S), "r"(Y));
    asm("lop3.b32 %0, %1, %2, %3, 0xA8;" : "=r"(X) : "r"(S), "r"(Y), "r"(M));
    asm("lop3.b32 %0, %1, %2, %3, 0x54;" : "=r"(Yn) : "r"(S), "r"(Y), "r"(M));
    asm("{\n\t"
        "add.cc.u32 %0, %0, %0;\n\t"
        "addc.cc.u32 %1, %3, %4;\n\t"
        "addc.u32 %2, %2, %2;\n\t"
        "}"
        : "+r"(sr), "=r"(S), "+r"(cw)
        : "r"(V), "r"(X));
    Y = Yn;
}

// Predicated stores (no branch, so no divergence for a one-lane store).
static __device__ __forceinline__ void st_relaxed_u64_if(bool p, uint64_t *ptr, uint64_t v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.relaxed.gpu.global.u64 [%1], %2;\n\t}"
                 ::"r"((uint32_t)p), "l"(ptr), "l"(v));
}
static __device__ __forceinline__ void st_volatile_shared_u64_if(bool p, uint32_t addr, uint64_t v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.volatile.shared.u64 [%1], %2;\n\t}"
                 ::"r"((uint32_t)p), "r"(addr), "l"(v));
}

// The column on V itself (bit 31 held at 1, rows in bits 0..30): two LOP3
// and three adds, the fewest ALU issue slots of the forms here (the single
// pair, bound by one lane's dependency chain, uses column31c instead).
//   CC = top bit of sr; X = V & M; A = V + X + CC, CC = carry out;
//   cw = 2 cw + CC; V' = A | (V & ~M)
static __device__ __forceinline__ void column31v(uint32_t &V, uint32_t &sr, uint32_t &cw, uint32_t M) {
    asm("{\n\t.reg .u32 x, a;\n\t"
        "add.cc.u32 %0, %0, %0;\n\t"
        "and.b32 x, %1, %3;\n\t"
        "addc.cc.u32 a, %1, x;\n\t"
        "addc.u32 %2, %2, %2;\n\t"
        "lop3.b32 %1, a, %1, %3, 0xF4;\n\t"
        "}"
        : "+r"(sr), "+r"(V), "+r"(cw)
        : "r"(M));
}

// Plain (weak) 64-bit shared-memory load and predicated store of a tagged
// word (tag in the high half, data in the low half).  One aligned 64-bit
// access is a single transaction, so a reader sees either the old word or the
// new one, and the tag tells which: the steady state needs no strong access
// (a volatile or relaxed one costs the warp a few hundred cycles in this
// loop); only the wait loops that run when a tag is stale read strongly.
static __device__ __forceinline__ uint64_t lds_u64(uint32_t addr) {
    uint64_t v;
    asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}
static __device__ __forceinline__ void sts_u64_if(bool p, uint32_t addr, uint64_t v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.shared.u64 [%1], %2;\n\t}"
                 ::"r"((uint32_t)p), "r"(addr), "l"(v));
}

static __device__ __forceinline__ int ld_acquire_shared(uint32_t addr) {
    int v;
    asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
static __device__ __forceinline__ void st_release_shared(uint32_t addr, int v) {
    asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// An acquire load that only some iterations take: with p false the register
// keeps its value (predicated, no branch).
static __device__ __forceinline__ void ld_acquire_shared_if(bool p, uint32_t addr, int &v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t@q ld.acquire.cta.shared.s32 %0, [%2];\n\t}"
                 : "+r"(v) : "r"((uint32_t)p), "r"(addr) : "memory");
}
// The same, predicated (no branch around a one-lane store).
static __device__ __forceinline__ void st_release_shared_if(bool p, uint32_t addr, int v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.release.cta.shared.s32 [%1], %2;\n\t}"
                 ::"r"((uint32_t)p), "r"(addr), "r"(v) : "memory");
}
}  // namespace dev
}  // namespace paco
