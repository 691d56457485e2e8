// common.cuh -- device-side helpers shared by the stencil kernels (sm_103a).
//
// Layout, element traits, TMA (cp.async.bulk.tensor) and mbarrier wrappers in inline PTX,
// bounded waits that report expiry through a per-plan error word instead of hanging.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace stn {

// Radius of the 6th-order central differences (Sec. 3.3).
constexpr int R6 = 3;

// Geometry of one padded field (augmented array f^ of Eq. 2), in elements.
struct Geom {
    int64_t n[3];    // interior extents (1 on unused axes)
    int64_t off[3];  // interior origin in padded coordinates
    int64_t pad[3];  // padded extents; pad[0] is the row pitch
    __host__ __device__ int64_t idx(int64_t i, int64_t j, int64_t k) const {
        return (off[0] + i) + pad[0] * ((off[1] + j) + pad[1] * (off[2] + k));
    }
    __host__ __device__ int64_t plane() const { return pad[0] * pad[1]; }
};

// Error word bits written by kernels (read and cleared by the host at sync points).
enum : unsigned { ERR_TIMEOUT = 1u };

// ---------------------------------------------------------------- element traits

template <typename S> struct Elem;
template <> struct Elem<double> {
    static constexpr CUtensorMapDataType tma = CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
};
template <> struct Elem<float> {
    static constexpr CUtensorMapDataType tma = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <> struct Elem<__nv_bfloat16> {
    static constexpr CUtensorMapDataType tma = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};

template <typename C, typename S> __device__ __forceinline__ C to_c(S v) { return (C)v; }
template <> __device__ __forceinline__ float to_c<float, __nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}
template <typename S, typename C> __device__ __forceinline__ S to_s(C v) { return (S)v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_s<__nv_bfloat16, float>(float v) {
    return __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of phase `parity` (mbarrier.test_wait never suspends the thread).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` for at most `limit_ns` nanoseconds.  Returns false if
// the wait expired (the caller then records ERR_TIMEOUT and leaves the kernel cleanly).
// Two independent bounds: the global nanosecond timer and the SM cycle counter (3 cycles per
// nanosecond of limit, i.e. at least the limit at clocks up to 3 GHz), whichever trips first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    const long long c0 = clock64();
    const long long climit = (long long)(3 * limit_ns);
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && (global_ns() - t0 > limit_ns || clock64() - c0 > climit)) return false;
    }
}

// Programmatic dependent launch.  A kernel launched with programmatic stream serialization
// lets the next such kernel in the stream start its preamble (barrier set-up, descriptor
// prefetch) early; every thread then waits until the previous kernel has completed and its
// memory operations are visible before it touches global memory.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// 3D tiled TMA load of one box into shared memory, completion signalled on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// 1D bulk copy of `bytes` (a multiple of 16) from global to shared memory, both addresses
// 16-byte aligned, completion signalled on `bar`.
__device__ __forceinline__ void bulk_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before its later
// async-proxy (bulk copy) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------- periodic images

// Store v at interior cell (i, j, k) and, when `images`, at every periodic image of that
// cell that falls inside the halo of width r (Eq. 2 with periodic beta), so the output
// array is a complete augmented array without a separate halo pass.
template <typename S>
__device__ __forceinline__ void store_with_images(S *__restrict__ f, const Geom &g, int r,
                                                  bool images, int64_t i, int64_t j, int64_t k,
                                                  S v) {
    f[g.idx(i, j, k)] = v;
    if (!images) return;
    int64_t xs[2] = {i, i}, ys[2] = {j, j}, zs[2] = {k, k};
    int nxs = 1, nys = 1, nzs = 1;
    if (i < r) xs[nxs++] = i + g.n[0];
    else if (i >= g.n[0] - r) xs[nxs++] = i - g.n[0];
    if (g.n[1] > 1) {
        if (j < r) ys[nys++] = j + g.n[1];
        else if (j >= g.n[1] - r) ys[nys++] = j - g.n[1];
    }
    if (g.n[2] > 1) {
        if (k < r) zs[nzs++] = k + g.n[2];
        else if (k >= g.n[2] - r) zs[nzs++] = k - g.n[2];
    }
    for (int c = 0; c < nzs; ++c)
        for (int b = 0; b < nys; ++b)
            for (int a = 0; a < nxs; ++a)
                if (a | b | c) f[g.idx(xs[a], ys[b], zs[c])] = v;
}

}  // namespace stn
