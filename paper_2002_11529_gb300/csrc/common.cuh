// Device helpers shared by the UT decoding and Compass kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ut_compass.h"

namespace utc {

// ---------------------------------------------------------------------------
// Status word: one u64 per context, lowered with atomicMin so that the error
// with the smallest (a, b) wins whatever the scheduling order.
//   key = a[32 bits] | b[24 bits] | (-code)[8 bits]; a/b = -1 -> all ones.
// UINT64_MAX means "no error".
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long err_key(int code, long long a, long long b) {
    const unsigned long long ka = a < 0 ? 0xFFFFFFFFull : (unsigned long long)(a & 0xFFFFFFFFll);
    const unsigned long long kb = b < 0 ? 0xFFFFFFull : (unsigned long long)(b & 0xFFFFFFll);
    return (ka << 32) | (kb << 8) | (unsigned long long)((-code) & 0xFF);
}

__device__ __forceinline__ void report(unsigned long long* status, int code, long long a, long long b) {
    atomicMin(status, err_key(code, a, b));
}

// ---------------------------------------------------------------------------
// Bounds-checked accesses.  In a build with -DUT_CHECKED every access made
// through these helpers compares its index with the array's extent first; a
// violation records UT_ERR_BOUNDS at (-1, site) in the status word and the
// access is skipped (a load yields zero) -- no trap, no fault.  Sites are
// numbered per file (decode 1xx, Compass 2xx, group search 3xx, persistent
// kernel 4xx, consolidation 5xx, alignment 6xx).  Without UT_CHECKED the
// helpers are the plain access and the extents are never computed.
// ---------------------------------------------------------------------------
#ifdef UT_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

__device__ __forceinline__ bool chk(bool ok, unsigned long long* status, int site) {
    if constexpr (kChecked) {
        if (!ok) report(status, UT_ERR_BOUNDS, -1, site);
        return ok;
    }
    return true;
}

template <class T>
__device__ __forceinline__ T ld_chk(const T* p, long long i, long long n, unsigned long long* status, int site) {
    if constexpr (kChecked) {
        if (i < 0 || i >= n) {
            report(status, UT_ERR_BOUNDS, -1, site);
            return T();
        }
    }
    return p[i];
}

template <class T>
__device__ __forceinline__ void st_chk(T* p, long long i, long long n, T v, unsigned long long* status, int site) {
    if constexpr (kChecked) {
        if (i < 0 || i >= n) {
            report(status, UT_ERR_BOUNDS, -1, site);
            return;
        }
    }
    p[i] = v;
}

// Default upper bound on the polls of a device-side wait (~0.5 s with the
// back-off below); past it the kernel records UT_ERR_TIMEOUT and moves on.
// A context can lower it (ut_ctx_set_wait_limit).
constexpr long long kSpinLimit = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------------------
// mbarrier + bulk (TMA) copy global -> shared.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders earlier generic-proxy accesses to shared memory before later
// async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; returns false if `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_volatile_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Half-strip key of a 16-bit hit word: 2*strip + frac.
__device__ __forceinline__ uint32_t half_strip(uint32_t w) { return 2u * (w & 0x3FFu) + ((w >> 10) & 1u); }

// Largest b in [0, n) with off[b] <= i (off non-decreasing, off[0] <= i).
__device__ __forceinline__ int find_bank(const uint32_t* off, int n, uint32_t i) {
    int lo = 0, hi = n;  // invariant: off[lo] <= i, answer < hi
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace utc

// Opaque context behind ut_ctx*.
struct ut_ctx {
    ut_geometry geom;
    unsigned long long* d_status;
    unsigned long long* h_status;  // pinned
    int device;
    int num_sms;
    int smem_optin;  // largest dynamic shared memory a block may opt in to
    // kick map (ut_ctx_set_kick_map): nx = 0 when none
    float* d_kmap;
    int kmap_nx, kmap_ny;
    float kmap_tx_max, kmap_ty_max, kmap_max;
    long long wait_limit;   // polls of a bounded device wait (ut_ctx_set_wait_limit)
    unsigned first_ticket;  // first work ticket of the decodes (ut_ctx_set_first_ticket)
};

namespace utc {
inline int check_cuda(cudaError_t e) { return e == cudaSuccess ? UT_OK : UT_ERR_CUDA; }
}  // namespace utc
