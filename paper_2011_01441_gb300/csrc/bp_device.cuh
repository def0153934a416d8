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
static __device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
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

// One lane waits for slot (u mod kRing) of a shared ring to carry tag u+1.
static __device__ __noinline__ uint32_t poll_ring_lane(const uint64_t *ring, int64_t u, int *err, long long limit,
                                                bool &ok) {
    const volatile uint64_t *slot = ring + (u % kRing);
    const uint32_t want = (uint32_t)(u + 1);
    uint64_t v = *slot;
    if ((uint32_t)(v >> 32) == want) return (uint32_t)v;
    const uint64_t t0 = global_ns();
    for (;;) {
        v = *slot;
        if ((uint32_t)(v >> 32) == want) return (uint32_t)v;
        if (ld_relaxed_i32(err) != 0) {
            ok = false;
            return 0;
        }
        if ((long long)(global_ns() - t0) > limit) {
            raise_error(err, kEtimeout);
            ok = false;
            return 0;
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

constexpr uint32_t kK31 = 0x7fffffffu;  // the 31 row bits of a lane word
constexpr int kLaneRows = 31;

static __device__ __forceinline__ uint4 ldg_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

// Shared-memory load at a 32-bit shared address.
static __device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// One column of Eq. (1) on a lane's 31 rows, state (S, Y) with V = (S|Y) & K31.
//   V = (S|Y) & K31, X = (S|Y) & M, Y' = (S|Y) & ~M        (three LOP3, one level)
//   S' = V + X + c, with c the top bit of the shift register sr (add.cc)
// V and X are below 2^31, so bit 31 of S' is the carry out of the lane's
// bottom row; bit 31 of S and Y is never read (V and X mask it), and the
// carry is shifted into cw (MSB first).
static __device__ __forceinline__ void column31(uint32_t &S, uint32_t &Y, uint32_t &sr, uint32_t &cw,
                                         uint32_t M) {
    uint32_t V, X, Yn, A;
    asm("lop3.b32 %0, %1, %2, %3, 0xA8;" : "=r"(V) : "r"(S), "r"(Y), "r"(kK31));
    asm("lop3.b32 %0, %1, %2, %3, 0xA8;" : "=r"(X) : "r"(S), "r"(Y), "r"(M));
    asm("lop3.b32 %0, %1, %2, %3, 0x54;" : "=r"(Yn) : "r"(S), "r"(Y), "r"(M));
    asm("{\n\t"
        "add.cc.u32 %0, %0, %0;\n\t"
        "addc.u32 %1, %2, %3;\n\t"
        "}"
        : "+r"(sr), "=r"(A)
        : "r"(V), "r"(X));
    S = A;
    Y = Yn;
    cw = __funnelshift_l(A, cw, 1);
}

// The same column with bit 31 of S | Y held at 1 (rows live in bits 0..30).
// Then bit 31 of V + X + c is 1 + 0 + (carry out of row 30), so the carry
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

static __device__ __forceinline__ int ld_acquire_shared(uint32_t addr) {
    int v;
    asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
static __device__ __forceinline__ void st_release_shared(uint32_t addr, int v) {
    asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
static __device__ __forceinline__ int ld_volatile_shared(uint32_t addr) {
    int v;
    asm volatile("ld.volatile.shared.s32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// The 32 column offsets [col0, col0 + 32) of a lane's word; columns outside
// [0, S) read as 0 (their steps are inactive).
static __device__ __forceinline__ uint2 ldg_v2(const void *p) {
    uint2 v;
    asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

// The 32 column offsets [col0, col0 + 32) of a lane's word; columns outside
// [0, S) read as 0 (their steps are inactive).  A 4-column block is read with
// one 16-byte load only when its address is 16-byte aligned, with two 8-byte
// loads when 8-byte aligned, otherwise element by element.
static __device__ __forceinline__ void load_window(const uint32_t *boff, int64_t col0, int64_t S,
                                                   uint32_t (&w)[32]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int64_t c = col0 + 4 * k;
        const uintptr_t addr = reinterpret_cast<uintptr_t>(boff + c);
        if (c >= 0 && c + 4 <= S && (addr & 15) == 0) {
            const uint4 v = ldg_v4(boff + c);
            w[4 * k] = v.x;
            w[4 * k + 1] = v.y;
            w[4 * k + 2] = v.z;
            w[4 * k + 3] = v.w;
        } else if (c >= 0 && c + 4 <= S && (addr & 7) == 0) {
            const uint2 v0 = ldg_v2(boff + c);
            const uint2 v1 = ldg_v2(boff + c + 2);
            w[4 * k] = v0.x;
            w[4 * k + 1] = v0.y;
            w[4 * k + 2] = v1.x;
            w[4 * k + 3] = v1.y;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) w[4 * k + e] = (c + e >= 0 && c + e < S) ? __ldg(boff + c + e) : 0u;
        }
    }
}

}  // namespace dev
}  // namespace paco
