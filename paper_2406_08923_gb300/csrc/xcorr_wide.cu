// xcorr_wide.cu -- 1D stencils of large radius: the cross-correlation of Eq. 3 for radius
// 5..1024 in FP64 and 33..1024 in FP32 (the radius sweep of Sec. 5.2, Fig. 8; FP32 up to radius
// 32 runs the temporally blocked kernel of xcorr.cu) and the max filter
// f'_i = max_{j=-r..r} f^_{i+j} (the nonlinear stencil of Sec. 2.1) for radius 0..1024.
//
// Cross-correlation.  At large radius the work is 2r+1 multiply-adds per output, so the kernel
// is built for FMA throughput: a CTA stages its chunk of outputs plus a halo of r cells per side
// and the 2r+1 weights in shared memory; each thread computes V consecutive outputs, and for
// every block of V weights loads the 2V-1 cells those outputs need into registers once and
// performs V x V multiply-adds from registers (one shared load per ~5 FMAs at V = 15).  V is
// odd so that lanes, V cells apart, fall on distinct shared-memory banks, and chosen per radius
// (wide_block).  Each output adds its terms in the order j = -r .. r.
//
// Max filter.  A direct window maximum costs 2r+1 comparisons per output.  Instead the chunk
// (+ halo) is reduced by doubling in shared memory: after step k every cell holds the maximum
// of the 2^k cells starting at it; with 2^K <= 2r+1 < 2^(K+1), the window [i-r, i+r] is the union
// of the two 2^K-cell runs starting at i-r and at i+r+1-2^K.  That is K + 1 <= 12 passes at
// r = 1024 instead of 2049 comparisons, and the maximum is exact in any order, so the result is
// bit-identical to the plain definition.  FP64 values are compared as order-preserving integer
// keys (see MaxKey).
//
// Both write the periodic images of the output's ends into its halo (Eq. 2) when asked.
#include <algorithm>

#include "internal.h"

namespace stn {
namespace {

constexpr int WT = 256;                // threads per CTA
constexpr int MF_CHUNK = 4096;         // max-filter outputs per CTA

// Stage cells [c0 - r, c0 - r + len) of the (padded, interior at `inx`) array into s[0, len):
// periodic wrap, or the caller's halo (cells -r .. n+r-1; anything beyond reads 0).  When the
// body [c0, c0 + body) lies inside the interior it is read with 16-byte vector loads (c0 and
// the interior origin are 16-byte aligned), the 2r halo cells with scalar loads.
template <typename T> struct V16;
template <> struct V16<float> { using type = float4; };
template <> struct V16<double> { using type = double2; };
template <> struct V16<int32_t> { using type = int4; };

template <typename T>
__device__ __forceinline__ void stage(const T *__restrict__ inx, int64_t n, int64_t c0, int r, int len, int body,
                                      int periodic, T *s) {
    constexpr int L = 16 / (int)sizeof(T);
    using VT = typename V16<T>::type;
    const int64_t g0 = c0 - r;
    auto cell = [&](int64_t gi) -> T {
        if (gi >= 0 && gi < n) return inx[gi];
        if (periodic) {
            gi %= n;
            if (gi < 0) gi += n;
            return inx[gi];
        }
        return (gi >= -r && gi < n + r) ? inx[gi] : T(0);
    };
    if (c0 + body <= n && body % L == 0) {
        const VT *src = reinterpret_cast<const VT *>(inx + c0);
        for (int v = threadIdx.x; v < body / L; v += blockDim.x) {
            const VT x = src[v];
            const T *e = reinterpret_cast<const T *>(&x);
#pragma unroll
            for (int u = 0; u < L; ++u) s[r + v * L + u] = e[u];
        }
        for (int e = threadIdx.x; e < len - body; e += blockDim.x) {  // r cells before, the rest after
            const int q = e < r ? e : body + e;
            s[q] = cell(g0 + q);
        }
    } else {
        for (int e = threadIdx.x; e < len; e += blockDim.x) s[e] = cell(g0 + e);
    }
}

// Store output p (interior index) and, when `images`, its periodic image in the halo.
template <typename T>
__device__ __forceinline__ void put1(T *outx, int64_t n, int r, int images, int64_t p, T v) {
    outx[p] = v;
    if (images) {
        if (p < r) outx[p + n] = v;
        if (p >= n - r) outx[p - n] = v;
    }
}

// Shared-memory layout of one staging buffer of the wide cross-correlation: the chunk's cells
// c0 - r .. c0 + CH + r - 1 start at element `lead` = rr - r, where rr is r rounded up to whole
// 16-byte groups, so that a bulk copy of cells c0 - rr .. c0 + CH + rr - 1 lands at element 0.
// Past the span come zeros for the padded weight blocks.
template <typename T, int V_> struct WideBuf {
    static constexpr int V = V_, CH = WT * V, L = 16 / (int)sizeof(T);
    static __host__ __device__ int rr(int r) { return (r + L - 1) / L * L; }
    static __host__ __device__ int nwp(int r) { return (2 * r + 1 + V - 1) / V * V; }
    // elements per buffer (a multiple of L, so every buffer starts 16-byte aligned)
    static __host__ __device__ int elems(int r) { return (2 * rr(r) + CH + nwp(r) + V + L - 1) / L * L; }
    static __host__ __device__ int wlen(int r) { return (nwp(r) + L - 1) / L * L; }
};

// The chunk's staging can use one bulk copy when its whole aligned span lies in the interior
// (the edge chunks wrap or read the caller's halo through `stage`).
__device__ __forceinline__ bool wide_bulk_ok(int64_t c0, int64_t n, int ch, int rr) {
    return c0 - rr >= 0 && c0 + ch + rr <= n;
}

constexpr int MAX_NBUF = 3;

// Bulk-copy pipeline over the chunks of a persistent CTA.  The CTA's k-th chunk (global chunk
// blockIdx.x + k gridDim.x) is staged in buffer k % nbuf, and copies run nbuf - 1 chunks ahead:
// thread 0 issues one cp.async.bulk per chunk, completion on the buffer's mbarrier.  The state
// (bit b of `phase`: parity of buffer b's next completion; bit b of `inflight`: a copy into
// buffer b is outstanding) is kept identically by every thread.
template <typename T> struct ChunkPipe {
    uint64_t *full;
    T *buf0;
    int be, ch, rr, nbuf;
    const T *inx;
    int64_t n, nchunks;
    uint32_t bytes, phase, inflight;

    __device__ bool bulk_ok(int64_t c) const { return c < nchunks && wide_bulk_ok(c * ch, n, ch, rr); }
    __device__ T *buf(int b) const { return buf0 + (size_t)b * be; }
    // chunk c into buffer b (a no-op for chunks that are staged by `stage` instead)
    __device__ void issue(int64_t c, int b) {
        if (!bulk_ok(c)) return;
        if (threadIdx.x == 0) {
            fence_proxy_async();
            mbar_arrive_expect_tx(&full[b], bytes);
            bulk_load_1d(buf(b), inx + c * ch - rr, bytes, &full[b]);
        }
        inflight |= 1u << b;
    }
    // Wait for buffer b's copy if one is outstanding; `*bulk` says whether there was one.
    // Returns false if the bounded wait expired.
    __device__ bool wait(int b, bool *bulk) {
        *bulk = (inflight >> b) & 1u;
        if (!*bulk) return true;
        if (!mbar_wait_bounded(&full[b], (phase >> b) & 1u)) return false;
        phase ^= 1u << b;
        inflight &= ~(1u << b);
        return true;
    }
    // thread 0, after a timeout: wait (bounded) for copies still in flight before the CTA exits
    __device__ void drain() {
        for (int b = 0; b < nbuf; ++b)
            if ((inflight >> b) & 1u) (void)mbar_wait_bounded(&full[b], (phase >> b) & 1u, 100000000ull);
    }
};

// Persistent kernel: CTA b handles chunks b, b + G, b + 2G, ... (G = gridDim.x) with two
// staging buffers.  While it computes chunk k, the bulk copy of chunk k + 1 (issued by thread 0,
// completion on one mbarrier per buffer) is in flight, so the load latency of a chunk overlaps
// the previous chunk's multiply-adds and stores.  Bounded waits: on expiry the CTA records
// ERR_TIMEOUT, waits (bounded) for its copy in flight and returns.
template <typename T, int V_>
__global__ void __launch_bounds__(WT)
xcorr_wide_kernel(const T *__restrict__ in, T *__restrict__ out, Geom geo, const T *__restrict__ wg, int r,
                  int periodic, int images, int nbuf, unsigned *err) {
    using B = WideBuf<T, V_>;
    constexpr int V = B::V, CH = B::CH, L = B::L;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[MAX_NBUF];
    const int nw = 2 * r + 1, nwp = B::nwp(r), rr = B::rr(r), lead = rr - r, be = B::elems(r);
    T *ws = reinterpret_cast<T *>(smem_raw);
    const int64_t n = geo.n[0];
    T *outx = out + geo.off[0];
    ChunkPipe<T> pp{full, ws + B::wlen(r), be, CH, rr, nbuf, in + geo.off[0], n, (n + CH - 1) / CH,
                    (uint32_t)((CH + 2 * rr) * sizeof(T)), 0u, 0u};

    if (threadIdx.x == 0) {
        for (int b = 0; b < nbuf; ++b) mbar_init(&full[b], 1);
        mbar_fence_init();
    }
    for (int j = threadIdx.x; j < nwp; j += WT) ws[j] = j < nw ? wg[j] : T(0);
    for (int e = threadIdx.x; e < nbuf * be; e += WT) pp.buf0[e] = T(0);
    fence_proxy_async();  // the zero fill precedes the bulk copies into the same buffers
    __syncthreads();

    const int64_t G = gridDim.x;
    int64_t c = blockIdx.x;
    for (int j = 0; j < nbuf - 1; ++j) pp.issue(c + j * G, j);
    bool ok = true;
    for (int k = 0; c < pp.nchunks; ++k, c += G) {
        const int b = k % nbuf;
        T *buf = pp.buf(b);
        const int64_t c0 = c * CH;
        // the buffer of chunk k + nbuf - 1 last held chunk k - 1, finished at the loop's barrier
        pp.issue(c + (nbuf - 1) * G, (k + nbuf - 1) % nbuf);
        const int span = CH + 2 * r;
        bool bulk;
        ok = pp.wait(b, &bulk);
        if (ok && bulk) {
            // cells the copy brought past the span (fewer than L) must read as 0
            if (threadIdx.x < rr - r) buf[lead + span + threadIdx.x] = T(0);
        } else if (ok) {
            stage(pp.inx, n, c0, r, span, CH, periodic, buf + lead);
            for (int e = lead + span + threadIdx.x; e < be; e += WT) buf[e] = T(0);
        }
        if (__syncthreads_or(!ok)) break;

        const T *s = buf + lead;
        const int base = threadIdx.x * V;
        T acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = T(0);
        for (int j0 = 0; j0 < nwp; j0 += V) {
            T w[V], x[2 * V - 1];
#pragma unroll
            for (int u = 0; u < V; ++u) w[u] = ws[j0 + u];
#pragma unroll
            for (int q = 0; q < 2 * V - 1; ++q) x[q] = s[base + j0 + q];
#pragma unroll
            for (int u = 0; u < V; ++u)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = fma(w[u], x[v + u], acc[v]);
        }
        // results through shared memory (the staged cells are no longer needed), then
        // coalesced 16-byte stores of the chunk and scalar stores of its periodic images
        __syncthreads();
#pragma unroll
        for (int v = 0; v < V; ++v) buf[base + v] = acc[v];
        __syncthreads();
        using VT = typename V16<T>::type;
        if (c0 + CH <= n) {
            for (int q = threadIdx.x; q < CH / L; q += WT) {
                VT x;
                T *e = reinterpret_cast<T *>(&x);
#pragma unroll
                for (int u = 0; u < L; ++u) e[u] = buf[q * L + u];
                reinterpret_cast<VT *>(outx + c0)[q] = x;
            }
        } else {
            for (int q = threadIdx.x; q < CH && c0 + q < n; q += WT) outx[c0 + q] = buf[q];
        }
        if (images && (c0 < r || c0 + CH > n - r))
            for (int q = threadIdx.x; q < CH; q += WT) {
                const int64_t p = c0 + q;
                if (p >= n) break;
                if (p < r) outx[p + n] = buf[q];
                if (p >= n - r) outx[p - n] = buf[q];
            }
        // buffer b is refilled (chunk k + nbuf) only after every thread is done with it
        fence_proxy_async();
        __syncthreads();
    }
    if (!ok && threadIdx.x == 0) {
        atomicOr(err, ERR_TIMEOUT);
        pp.drain();
    }
}

template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return b > a ? b : a; }

// FP64 comparisons run on GB300's FP64 pipe (1/64 of the FP32 rate), so the FP64 max filter
// compares order-preserving 64-bit integer keys instead: negative values have all bits flipped,
// the others the sign bit set, which orders finite doubles like their values.
template <typename T> struct MaxKey {  // identity for int32 and FP32
    using K = T;
    static __device__ __forceinline__ K to(T v) { return v; }
    static __device__ __forceinline__ T from(K k) { return k; }
};
template <> struct MaxKey<double> {
    using K = unsigned long long;
    static __device__ __forceinline__ K to(double v) {
        const K b = (K)__double_as_longlong(v);
        return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    }
    static __device__ __forceinline__ double from(K k) {
        return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
    }
};

// Max filter, persistent like the cross-correlation: two staging buffers (chunk k + 1 arrives by
// bulk copy while chunk k is reduced) and one work buffer for the doubling passes, which
// ping-pong between the chunk's staging buffer and the work buffer.
template <typename T> struct MaxBuf {
    static constexpr int L = 16 / (int)sizeof(T);
    static __host__ __device__ int rr(int r) { return (r + L - 1) / L * L; }
    static __host__ __device__ int elems(int r) { return (MF_CHUNK + 2 * rr(r) + L - 1) / L * L; }
};

template <typename T>
__global__ void __launch_bounds__(WT)
maxfilter_kernel(const T *__restrict__ in, T *__restrict__ out, Geom geo, int r, int periodic, int images,
                 int nbuf, unsigned *err) {
    using MK = MaxKey<T>;
    using K = typename MK::K;
    static_assert(sizeof(K) == sizeof(T), "keys are converted in place");
    using B = MaxBuf<T>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[MAX_NBUF];
    const int span = MF_CHUNK + 2 * r, rr = B::rr(r), lead = rr - r, be = B::elems(r);
    const int64_t n = geo.n[0];
    T *outx = out + geo.off[0];
    // buffers 0 .. nbuf-1 stage chunks; buffer nbuf is the work buffer of the doubling passes
    ChunkPipe<T> pp{full, reinterpret_cast<T *>(smem_raw), be, MF_CHUNK, rr, nbuf, in + geo.off[0], n,
                    (n + MF_CHUNK - 1) / MF_CHUNK, (uint32_t)((MF_CHUNK + 2 * rr) * sizeof(T)), 0u, 0u};
    const int w = 2 * r + 1;

    if (threadIdx.x == 0) {
        for (int b = 0; b < nbuf; ++b) mbar_init(&full[b], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int64_t G = gridDim.x;
    int64_t c = blockIdx.x;
    for (int j = 0; j < nbuf - 1; ++j) pp.issue(c + j * G, j);
    bool ok = true;
    for (int k = 0; c < pp.nchunks; ++k, c += G) {
        const int b = k % nbuf;
        T *st = pp.buf(b) + lead;
        const int64_t c0 = c * MF_CHUNK;
        pp.issue(c + (nbuf - 1) * G, (k + nbuf - 1) % nbuf);
        bool bulk;
        ok = pp.wait(b, &bulk);
        if (ok && !bulk) stage(pp.inx, n, c0, r, span, MF_CHUNK, periodic, st);
        if (__syncthreads_or(!ok)) break;
        K *a = reinterpret_cast<K *>(st);
        K *bw = reinterpret_cast<K *>(pp.buf(nbuf) + lead);
        for (int i = threadIdx.x; i < span; i += WT) a[i] = MK::to(st[i]);  // same size: in place
        __syncthreads();
        int len = 1;  // a[i] = max of the `len` cells starting at i, for i <= span - len
        while (2 * len <= w) {
            for (int i = threadIdx.x; i <= span - 2 * len; i += WT) bw[i] = tmax(a[i], a[i + len]);
            __syncthreads();
            K *t = a;
            a = bw;
            bw = t;
            len *= 2;
        }
        for (int i = threadIdx.x; i < MF_CHUNK; i += WT) {
            const int64_t p = c0 + i;
            if (p < n) put1(outx, n, r, images, p, MK::from(tmax(a[i], a[i + w - len])));
        }
        fence_proxy_async();
        __syncthreads();
    }
    if (!ok && threadIdx.x == 0) {
        atomicOr(err, ERR_TIMEOUT);
        pp.drain();
    }
}

// Pipeline depth of the max filter.  Its doubling passes are bound by shared memory, and
// measured depths 1-3 at radius 8..1024 (FP32 and FP64) favour occupancy over prefetch: one
// staging buffer (the chunk's own copy, then its passes), except at radius 0, a plain copy,
// where prefetching the next chunk wins.
inline int maxf_nbuf(int r) { return r == 0 ? 2 : 1; }

template <typename T, int V>
cudaError_t run_wide(const void *in, void *out, const Geom &g, const void *wdev, int r, bool periodic, bool images,
                     unsigned *err, cudaStream_t s) {
    using B = WideBuf<T, V>;
    auto k = xcorr_wide_kernel<T, V>;
    // two staging buffers (prefetch) unless the second one costs resident CTAs; the choice
    // and the occupancy are computed once per radius
    static int choice[1025][2];  // {nbuf, resident CTAs per SM}, 0 = not yet computed
    if (!choice[r][0]) {
        int nbuf = 0, occ = 0;
        for (int nb = 2; nb >= 1; --nb) {
            const size_t sm = sizeof(T) * ((size_t)B::wlen(r) + (size_t)nb * B::elems(r));
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            int o = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, WT, sm);
            if (e != cudaSuccess) return e;
            if (nbuf == 0 || o > occ) {
                nbuf = nb;
                occ = o;
            }
        }
        choice[r][1] = occ;
        choice[r][0] = nbuf;
    }
    const int nbuf = choice[r][0], occ = choice[r][1];
    const size_t smem = sizeof(T) * ((size_t)B::wlen(r) + (size_t)nbuf * B::elems(r));
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long chunks = (long)((g.n[0] + B::CH - 1) / B::CH);
    const unsigned blocks = (unsigned)std::max(1L, std::min(chunks, (long)std::max(occ, 1) * device_sms()));
    k<<<blocks, WT, smem, s>>>(static_cast<const T *>(in), static_cast<T *>(out), g, static_cast<const T *>(wdev), r,
                               periodic ? 1 : 0, images ? 1 : 0, nbuf, err);
    return cudaGetLastError();
}

// Outputs per thread V (= weights per register block): the 2r+1 weights are padded to whole
// blocks of V, so V is chosen per radius from a few compiled sizes (all odd: lanes V cells
// apart fall on distinct banks).  A block costs V^2 multiply-adds, about 3V shared loads and
// some address arithmetic for V outputs.  FP32 is issue-bound: the cost per output is blocks
// x (V + 6), the 6 fitted to radius sweeps on GB300 (at r = 64 and 128, V = 15 beats V = 13
// although it pads more).  FP64 is bound by the FP64 pipe, where a shared load weighs about a
// tenth of a multiply-add: blocks x (V + 0.3), in tenths.  Ties go to the larger V.
template <typename T> int wide_block(int r, const int *vs, int nv) {
    const int nw = 2 * r + 1;
    int best = vs[0];
    long best_cost = -1;
    for (int i = 0; i < nv; ++i) {
        const int v = vs[i], blocks = (nw + v - 1) / v;
        const long cost = sizeof(T) == 8 ? (long)blocks * (10 * v + 3) : (long)blocks * (v + 6);
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && v > best)) {
            best = v;
            best_cost = cost;
        }
    }
    return best;
}
constexpr int WIDE_V_F32[] = {9, 11, 13, 15};
constexpr int WIDE_V_F64[] = {5, 7, 9};

template <typename T>
cudaError_t run_maxf(const void *in, void *out, const Geom &g, int r, bool periodic, bool images, unsigned *err,
                     cudaStream_t s) {
    const int nbuf = maxf_nbuf(r);
    const size_t smem = (size_t)(nbuf + 1) * sizeof(T) * (size_t)MaxBuf<T>::elems(r);
    auto k = maxfilter_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, WT, smem);
    if (e != cudaSuccess) return e;
    const long chunks = (long)((g.n[0] + MF_CHUNK - 1) / MF_CHUNK);
    const unsigned blocks = (unsigned)std::max(1L, std::min(chunks, (long)std::max(occ, 1) * device_sms()));
    k<<<blocks, WT, smem, s>>>(static_cast<const T *>(in), static_cast<T *>(out), g, r, periodic ? 1 : 0,
                               images ? 1 : 0, nbuf, err);
    return cudaGetLastError();
}

}  // namespace

int xcorr_wide_max_radius() { return 1024; }

cudaError_t launch_xcorr_wide(int dtype, int r, const void *in, void *out, const Geom &g, const void *wdev,
                              bool periodic, bool images, unsigned *err, cudaStream_t s) {
    if (r < 0 || r > xcorr_wide_max_radius()) return cudaErrorInvalidValue;
    if (dtype == 1) {
        switch (wide_block<double>(r, WIDE_V_F64, 3)) {
        case 5: return run_wide<double, 5>(in, out, g, wdev, r, periodic, images, err, s);
        case 9: return run_wide<double, 9>(in, out, g, wdev, r, periodic, images, err, s);
        default: return run_wide<double, 7>(in, out, g, wdev, r, periodic, images, err, s);
        }
    }
    if (dtype == 2) {
        switch (wide_block<float>(r, WIDE_V_F32, 4)) {
        case 9: return run_wide<float, 9>(in, out, g, wdev, r, periodic, images, err, s);
        case 11: return run_wide<float, 11>(in, out, g, wdev, r, periodic, images, err, s);
        case 13: return run_wide<float, 13>(in, out, g, wdev, r, periodic, images, err, s);
        default: return run_wide<float, 15>(in, out, g, wdev, r, periodic, images, err, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_maxfilter(int dtype, int r, const void *in, void *out, const Geom &g, bool periodic, bool images,
                             unsigned *err, cudaStream_t s) {
    if (r < 0 || r > xcorr_wide_max_radius()) return cudaErrorInvalidValue;
    switch (dtype) {
    case 0: return run_maxf<int32_t>(in, out, g, r, periodic, images, err, s);
    case 1: return run_maxf<double>(in, out, g, r, periodic, images, err, s);
    case 2: return run_maxf<float>(in, out, g, r, periodic, images, err, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace stn
