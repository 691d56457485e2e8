// xcorr_wide.cu -- 1D stencils of large radius: the cross-correlation of Eq. 3 for radius
// 5..1024 (the radius sweep of Sec. 5.2, Fig. 8) and the max filter f'_i = max_{j=-r..r} f^_{i+j}
// (the nonlinear stencil of Sec. 2.1) for radius 0..1024.
//
// Cross-correlation.  At large radius the work is 2r+1 multiply-adds per output, so the kernel
// is built for FMA throughput: a CTA stages its chunk of outputs plus a halo of r cells per side
// and the 2r+1 weights in shared memory; each thread computes V consecutive outputs, and for
// every block of V weights loads the 2V-1 cells those outputs need into registers once and
// performs V x V multiply-adds from registers (one shared load per ~5 FMAs at V = 15).  V is
// odd so that lanes, V cells apart, fall on distinct shared-memory banks.  Each output adds its
// terms in the order j = -r .. r.
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

template <typename T> struct Wide;
template <> struct Wide<float> { static constexpr int V = 15; };
template <> struct Wide<double> { static constexpr int V = 7; };
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

template <typename T>
__global__ void __launch_bounds__(WT)
xcorr_wide_kernel(const T *__restrict__ in, T *__restrict__ out, Geom geo, const T *__restrict__ wg, int r,
                  int periodic, int images) {
    constexpr int V = Wide<T>::V;
    constexpr int CH = WT * V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nw = 2 * r + 1;
    const int nwp = (nw + V - 1) / V * V;  // weights padded to whole blocks of V (zeros)
    T *ws = reinterpret_cast<T *>(smem_raw);
    T *s = ws + nwp;                       // CH + nwp + V cells (the tail past the span is 0)
    const int64_t n = geo.n[0];
    const int64_t c0 = (int64_t)blockIdx.x * CH;
    const T *inx = in + geo.off[0];
    T *outx = out + geo.off[0];

    for (int j = threadIdx.x; j < nwp; j += WT) ws[j] = j < nw ? wg[j] : T(0);
    const int span = CH + 2 * r;
    stage(inx, n, c0, r, span, CH, periodic, s);
    for (int e = span + threadIdx.x; e < CH + nwp + V; e += WT) s[e] = T(0);
    __syncthreads();

    const int base = threadIdx.x * V;
    T acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = T(0);
    for (int j0 = 0; j0 < nwp; j0 += V) {
        T w[V], x[2 * V - 1];
#pragma unroll
        for (int u = 0; u < V; ++u) w[u] = ws[j0 + u];
#pragma unroll
        for (int k = 0; k < 2 * V - 1; ++k) x[k] = s[base + j0 + k];
#pragma unroll
        for (int u = 0; u < V; ++u)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = fma(w[u], x[v + u], acc[v]);
    }
    // results through shared memory (the staged cells are no longer needed), then coalesced
    // 16-byte stores of the chunk and scalar stores of its periodic images
    __syncthreads();
#pragma unroll
    for (int v = 0; v < V; ++v) s[base + v] = acc[v];
    __syncthreads();
    constexpr int L = 16 / (int)sizeof(T);
    using VT = typename V16<T>::type;
    if (c0 + CH <= n) {
        for (int q = threadIdx.x; q < CH / L; q += WT) {
            VT x;
            T *e = reinterpret_cast<T *>(&x);
#pragma unroll
            for (int u = 0; u < L; ++u) e[u] = s[q * L + u];
            reinterpret_cast<VT *>(outx + c0)[q] = x;
        }
    } else {
        for (int q = threadIdx.x; q < CH && c0 + q < n; q += WT) outx[c0 + q] = s[q];
    }
    if (images)
        for (int q = threadIdx.x; q < CH; q += WT) {
            const int64_t p = c0 + q;
            if (p >= n) break;
            if (p < r) outx[p + n] = s[q];
            if (p >= n - r) outx[p - n] = s[q];
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

template <typename T>
__global__ void __launch_bounds__(WT)
maxfilter_kernel(const T *__restrict__ in, T *__restrict__ out, Geom geo, int r, int periodic, int images) {
    using MK = MaxKey<T>;
    using K = typename MK::K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int span = MF_CHUNK + 2 * r;
    T *st = reinterpret_cast<T *>(smem_raw);
    K *a = reinterpret_cast<K *>(smem_raw);
    K *b = a + span;
    const int64_t n = geo.n[0];
    const int64_t c0 = (int64_t)blockIdx.x * MF_CHUNK;
    const T *inx = in + geo.off[0];
    T *outx = out + geo.off[0];
    stage(inx, n, c0, r, span, MF_CHUNK, periodic, st);
    __syncthreads();
    for (int i = threadIdx.x; i < span; i += WT) a[i] = MK::to(st[i]);  // same size: in place
    __syncthreads();
    const int w = 2 * r + 1;
    int len = 1;  // a[i] = max of the `len` cells starting at i, for i <= span - len
    while (2 * len <= w) {
        for (int i = threadIdx.x; i <= span - 2 * len; i += WT) b[i] = tmax(a[i], a[i + len]);
        __syncthreads();
        K *t = a;
        a = b;
        b = t;
        len *= 2;
    }
    for (int i = threadIdx.x; i < MF_CHUNK; i += WT) {
        const int64_t p = c0 + i;
        if (p < n) put1(outx, n, r, images, p, MK::from(tmax(a[i], a[i + w - len])));
    }
}

template <typename T>
cudaError_t run_wide(const void *in, void *out, const Geom &g, const void *wdev, int r, bool periodic, bool images,
                     cudaStream_t s) {
    constexpr int V = Wide<T>::V;
    const int nwp = (2 * r + 1 + V - 1) / V * V;
    const size_t smem = sizeof(T) * ((size_t)nwp + WT * V + nwp + V);
    auto k = xcorr_wide_kernel<T>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)((g.n[0] + WT * V - 1) / (WT * V));
    k<<<blocks, WT, smem, s>>>(static_cast<const T *>(in), static_cast<T *>(out), g, static_cast<const T *>(wdev), r,
                               periodic ? 1 : 0, images ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_maxf(const void *in, void *out, const Geom &g, int r, bool periodic, bool images, cudaStream_t s) {
    const size_t smem = 2 * sizeof(T) * ((size_t)MF_CHUNK + 2 * r);
    auto k = maxfilter_kernel<T>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)((g.n[0] + MF_CHUNK - 1) / MF_CHUNK);
    k<<<blocks, WT, smem, s>>>(static_cast<const T *>(in), static_cast<T *>(out), g, r, periodic ? 1 : 0,
                               images ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

int xcorr_wide_max_radius() { return 1024; }

cudaError_t launch_xcorr_wide(int dtype, int r, const void *in, void *out, const Geom &g, const void *wdev,
                              bool periodic, bool images, cudaStream_t s) {
    if (r < 0 || r > xcorr_wide_max_radius()) return cudaErrorInvalidValue;
    if (dtype == 1) return run_wide<double>(in, out, g, wdev, r, periodic, images, s);
    if (dtype == 2) return run_wide<float>(in, out, g, wdev, r, periodic, images, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_maxfilter(int dtype, int r, const void *in, void *out, const Geom &g, bool periodic, bool images,
                             cudaStream_t s) {
    if (r < 0 || r > xcorr_wide_max_radius()) return cudaErrorInvalidValue;
    switch (dtype) {
    case 0: return run_maxf<int32_t>(in, out, g, r, periodic, images, s);
    case 1: return run_maxf<double>(in, out, g, r, periodic, images, s);
    case 2: return run_maxf<float>(in, out, g, r, periodic, images, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace stn
