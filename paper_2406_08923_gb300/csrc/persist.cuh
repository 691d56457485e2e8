// persist.cuh -- persistent multi-step schedule of the streaming 3D heat kernels (Sec. 3.2,
// Eqs. 4-7 advanced nsteps times in one launch).
//
// One cooperative launch runs every forward-Euler step of a stencil_step call.  The work
// units are the (x tile, y tile, z chunk) boxes of the one-launch-per-step schedule; CTA b
// takes units b, b + G, b + 2G, ... (G CTAs) in every step, in that order.  No grid-wide
// barrier separates the steps.  Before a unit of step s loads its input, the units that wrote
// the cells it reads in step s-1 must have published step s-1: the owners of the R cells
// beyond each of its six faces, with periodic wrap (the star stencil reads nothing else; the
// periodic images a unit stores are read only by the face neighbours across the boundary).
// The same wait covers the write-after-read hazard of the ping-pong buffers: step s writes
// the buffer that the neighbours read in step s-1, and they finished reading it before they
// published s-1.  Dependencies always point to the previous step, so with every CTA resident
// (the cooperative launch guarantees it) every wait is eventually satisfied.
//
// Sync words (64-bit, device memory owned by the plan, zeroed once when allocated):
//   [0] epoch: steps run by earlier launches on these words.  Unit flags are set to
//       epoch + s + 1 once step s of the unit is stored, so flags left by earlier launches are
//       always below the current targets and the words never need clearing;
//   [1] number of CTAs that have left the current launch (the last one advances the epoch);
//   [2] abort tag: epoch + 1 once some CTA gave up, so the others stop waiting at once;
//   [3 + u] flag of unit u.
// Every wait is bounded: on expiry the CTA records ERR_TIMEOUT, raises the abort tag and
// leaves the kernel.
//
// Memory ordering.  Outputs are written with generic stores and read in the next step by TMA
// (the async proxy), possibly on another SM: every writer thread fences its stores toward the
// async proxy, the CTA synchronises, and one thread publishes the flag with a GPU-scope
// release after a GPU-scope fence.  The reader acquires the flag, synchronises its CTA, and
// the thread that issues the TMA loads fences toward the async proxy before issuing them.
#pragma once

#include "common.cuh"

namespace stn {

// Invalidates a completed mbarrier so that its word can be initialised again.
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Orders this thread's earlier generic-proxy global-memory accesses against later async-proxy
// (TMA) accesses of global memory, in either direction.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// 64-bit release store / acquire and relaxed loads at GPU scope (inter-CTA flags).
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

constexpr int PERSIST_HDR = 3;                             // sync words before the unit flags
constexpr unsigned long long PERSIST_WAIT_NS = 1000000000ull;  // 1 s per wait

// Unit decomposition of one launch: tiles per axis and tile length per axis (cells).
struct PersistGrid {
    int nt[3];
    int tl[3];
    __host__ __device__ int units() const { return nt[0] * nt[1] * nt[2]; }
};

// Waits until every face neighbour of unit (t0, t1, t2) has published `target` or later.
// Called by all threads of the CTA; returns false (uniformly) if a wait expired or the abort
// tag was raised.
template <int R>
__device__ __forceinline__ bool wait_face_neighbours(const unsigned long long *sync, const PersistGrid &pg,
                                                     const Geom &g, int t0, int t1, int t2,
                                                     unsigned long long target, unsigned long long abort_tag) {
    bool fail = false;
    if (threadIdx.x < 6 * R) {
        // thread -> (axis, side, distance k = 1..R of the cell beyond that face)
        const int ax = threadIdx.x / (2 * R), side = (threadIdx.x / R) & 1, k = threadIdx.x % R + 1;
        const int n = (int)(ax == 0 ? g.n[0] : ax == 1 ? g.n[1] : g.n[2]);
        const int L = ax == 0 ? pg.tl[0] : ax == 1 ? pg.tl[1] : pg.tl[2];
        const int t = ax == 0 ? t0 : ax == 1 ? t1 : t2;
        const int lo = t * L, hi = min(n, lo + L);
        int cell = side ? hi - 1 + k : lo - k;
        cell = ((cell % n) + n) % n;
        const int o = cell / L;
        if (o != t) {
            const int q0 = ax == 0 ? o : t0, q1 = ax == 1 ? o : t1, q2 = ax == 2 ? o : t2;
            const unsigned long long *fl = sync + PERSIST_HDR + q0 + pg.nt[0] * (q1 + pg.nt[1] * q2);
            if ((long long)(ld_acquire_u64(fl) - target) < 0) {
                const uint64_t ns0 = global_ns();
                const long long c0 = clock64();
                for (uint32_t it = 0;; ++it) {
                    __nanosleep(64);
                    if ((long long)(ld_acquire_u64(fl) - target) >= 0) break;
                    if ((it & 15u) == 15u &&
                        (ld_relaxed_u64(sync + 2) == abort_tag || global_ns() - ns0 > PERSIST_WAIT_NS ||
                         clock64() - c0 > (long long)(3 * PERSIST_WAIT_NS))) {
                        fail = true;
                        break;
                    }
                }
            }
        }
    }
    return !__syncthreads_or(fail);
}

// Publishes step `s` of unit `u` (thread 0, after the CTA synchronised on the stores).
__device__ __forceinline__ void publish_unit(unsigned long long *sync, int u, unsigned long long value) {
    __threadfence();
    st_release_u64(sync + PERSIST_HDR + u, value);
}

// Leaves the launch (thread 0): raises the abort tag if this CTA gave up, and the last CTA
// out advances the epoch by the launch's steps for the next launch on these words.
__device__ __forceinline__ void persist_exit(unsigned long long *sync, unsigned long long base, int nsteps,
                                             bool failed) {
    if (failed) st_release_u64(sync + 2, base + 1);
    __threadfence();
    const unsigned long long left = atomicAdd(sync + 1, 1ull);
    if (left == (unsigned long long)gridDim.x - 1) {
        sync[1] = 0;
        st_release_u64(sync, base + (unsigned long long)nsteps);
    }
}

}  // namespace stn
