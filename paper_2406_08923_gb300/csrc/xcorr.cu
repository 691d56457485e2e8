// xcorr.cu -- 1D cross-correlation f'_i = sum_{j=-r..r} g_j f^_{i+j} (Sec. 3.1, Eq. 3).
//
// Radius 0..4 (int32, FP32, FP64) and, for FP32, 5..32.
//
// GB300 design: the input (2^20 int32 = 4 MiB in the benchmark) is L2-resident and a single
// sweep moves ~8 MB, far less than what a launch costs in latency.  So one launch performs
// several sweeps (temporal blocking): each CTA stages its chunk plus a halo of
// sweeps * r cells per side in shared memory (coalesced 128-bit loads for the body,
// periodic wrap for the halo), runs the sweeps in shared memory on a shrinking valid region
// (each thread 9 consecutive outputs from a register window; FP64 one output per thread),
// and writes its chunk once, together with the periodic images of the array ends so the
// output is a complete augmented array (Eq. 2).  Every output value is produced by the same
// multiply-add sequence j = -r..r as a one-sweep-per-launch kernel would use, so the result
// is bit-identical to sweeping once per launch.  int32 arithmetic is done in uint32
// (modulo 2^32); floating point uses fused multiply-add in order j = -r..r.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace stn {

constexpr int XC_THREADS = 256;
// FP64 CTAs: 512 threads, two per SM, when one wave of them covers the input; else 256
// threads, four per SM (below).  Either way 1024 threads per SM at 64 registers.
constexpr int XC_T64 = 512;
template <typename T, int NT> constexpr int xc_minb() { return sizeof(T) == 8 ? 1024 / NT : 1; }
// Consecutive outputs per thread and sweep (register blocking).  Odd, so that lanes XC_V cells
// apart read and write distinct shared-memory banks.
constexpr int XC_V = 9;
constexpr int XC_MAX_SWEEPS = 16;
// Outputs per CTA: with its halo (up to 15 sweeps x 4 cells per side) every sweep's span fits
// in the 256 x 9 outputs one pass of the threads computes.
constexpr int XC_CHUNK = XC_THREADS * XC_V - 2 * (XC_MAX_SWEEPS - 1) * 4;  // 2184
// FP64 sweeps one output per thread and iteration (below), so its chunk is a runtime length
// (even, 256..4096), chosen so that the grid fills whole waves.  The FP64 pipe retires one
// warp instruction per 16 SM cycles, so what a sweep costs is the warp instructions of the
// busiest SM sub-partition, and whole warps count even where lanes idle.  Per sweep a CTA
// evaluates its chunk plus the halo of the sweeps still to come, in rows of 32 cells.
//   * Inputs whose input and output arrays fill at most 7/8 of L2 together run as whole
//     waves of two 512-thread CTAs per SM (chunks up to 4096 cells): the 2^20-cell benchmark
//     is one wave of 3450-cell chunks.  With the rows spread evenly over the sub-partitions
//     (below), 98.7 % of the issued lanes are outputs, against 96.2 % with four 1726-cell
//     CTAs of 256 threads per SM.  Measured with 16 sweeps per launch, r = 3: 2^22 cells
//     794 us in 4 waves (835 us in 3.4 waves of 2048-cell chunks), 3 x 2^21 cells 1189 us in
//     6 waves (1248 us).
//   * Larger inputs run 2048-cell chunks in CTAs of 256 threads, four per SM, scheduled as
//     SMs free up; there each CTA's staging reads DRAM, and four CTAs per SM keep more of them
//     sweeping meanwhile.  2^23 cells: 1602 us (1648 us in 7 whole waves of 512-thread CTAs);
//     2^24 cells: 3192 us (3278 us in whole waves of 512-thread CTAs, 3314 us in 14 whole
//     waves of 1972-cell chunks of 256 threads).  Rotating the rows changed nothing there, nor
//     did PDL, nor 128-byte aligned chunks.
template <typename T> constexpr int xc_chunk() { return sizeof(T) == 8 ? 4096 : XC_CHUNK; }
constexpr int XC_F64_MULTI_CHUNK = 2048;

// L2 capacity in bytes of the current device (cached per device).
static int64_t device_l2_bytes() {
    static int l2[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!l2[dev] && cudaDeviceGetAttribute(&l2[dev], cudaDevAttrL2CacheSize, dev) != cudaSuccess) l2[dev] = -1;
    return l2[dev] > 0 ? l2[dev] : 0;
}
constexpr int XC_PAD = 4;  // buffer elements before logical cell 0
// elements per shared-memory buffer: a sweep starting at cell s r <= 96 (the halo of the
// sweeps one launch runs, at most 3 x 30 cells) reads up to 256 x 9 + 40 cells past its start
constexpr int XC_BUF = XC_PAD + 96 + XC_THREADS * XC_V + 40;
// FP64 buffers hold exactly the staged span (the scalar sweep reads nothing outside it), so a
// short chunk also takes less shared memory; even, so the second buffer stays 16-byte aligned.
__host__ __device__ constexpr int xc_f64_stride(int chunk, int halo) { return (XC_PAD + chunk + 2 * halo + 1) & ~1; }
static_assert(XC_CHUNK % 4 == 0, "the chunk body is moved as 16-byte vectors");

// Sweeps per launch at radius r: the halo of S sweeps must leave every sweep's span within the
// 256 x 9 outputs of one pass, i.e. 2 r (S - 1) <= 120.
int xcorr_max_sweeps_per_launch(int r) { return r <= 4 ? XC_MAX_SWEEPS : std::min(XC_MAX_SWEEPS, 1 + 60 / r); }

template <typename T> struct XAcc { using type = T; };
template <> struct XAcc<int32_t> { using type = uint32_t; };

template <typename T> struct Vec16;
template <> struct Vec16<int32_t> { using type = int4; static constexpr int n = 4; };
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

template <typename A> __device__ __forceinline__ A mac(A acc, A g, A f) { return fma(g, f, acc); }
template <> __device__ __forceinline__ uint32_t mac<uint32_t>(uint32_t acc, uint32_t g, uint32_t f) {
    return acc + g * f;
}

constexpr int XC_MAX_R = 32;  // FP32 radius 5..32 also runs here (int32 and FP64: 0..4)
template <typename T> struct XCoef { T g[2 * XC_MAX_R + 1]; };

// One chunk of outputs (xc_chunk<T>(); FP64: chunk_len) : stage, sweep in shared memory, write
// (+ images).
template <typename T, int R, int NT = XC_THREADS>
__device__ __forceinline__ void xcorr_chunk(const T *__restrict__ in, T *__restrict__ out, const Geom &geo,
                                            const XCoef<T> &cf, int sweeps, int periodic, int images, int chunk,
                                            unsigned char *smem_raw, int chunk_len = 0) {
    using A = typename XAcc<T>::type;
    static_assert(sizeof(A) == 8 || NT == XC_THREADS, "the register-window sweep assumes XC_THREADS threads");
    const int CHUNK = sizeof(A) == 8 ? chunk_len : xc_chunk<T>();
    const int H = sweeps * R;
    const int W = CHUNK + 2 * H;
    A *buf0 = reinterpret_cast<A *>(smem_raw);
    A *buf1 = buf0 + (sizeof(A) == 8 ? xc_f64_stride(CHUNK, H) : XC_BUF);
    const int64_t n = geo.n[0];
    const int64_t c0 = (int64_t)chunk * CHUNK;
    const T *inx = in + geo.off[0];  // interior element 0
    T *outx = out + geo.off[0];

    // stage [c0 - H, c0 + CHUNK + H) into buf0[0 .. W)
    constexpr int V = Vec16<T>::n;
    using VT = typename Vec16<T>::type;
    const bool full = c0 + CHUNK <= n;
    if (full) {
        const VT *src = reinterpret_cast<const VT *>(inx + c0);
        for (int v = threadIdx.x; v < CHUNK / V; v += NT) {
            VT x = src[v];
            const T *e = reinterpret_cast<const T *>(&x);
#pragma unroll
            for (int u = 0; u < V; ++u) buf0[XC_PAD + H + v * V + u] = (A)e[u];
        }
    }
    for (int e = threadIdx.x; e < W; e += NT) {
        const bool body = e >= H && e < H + CHUNK;
        if (full && body) continue;
        int64_t gi = c0 - H + e;
        T v;
        if (periodic) {
            gi %= n;
            if (gi < 0) gi += n;
            v = inx[gi];
        } else {
            v = (gi >= -R && gi < n + R) ? inx[gi] : T(0);
        }
        buf0[XC_PAD + e] = (A)v;
    }
    // FP64: the weights go through shared memory into registers, so that every multiply-add
    // takes register operands.  Taken as kernel parameters, they became constant-bank operands
    // of the FP64 multiply-adds, and a sweep ran 12 % slower (0.1498 against 0.1313 ms for the
    // 2^20-cell, 10-sweep job).
    __shared__ A wsm[2 * R + 1];
    if (sizeof(A) == 8 && threadIdx.x < 2 * R + 1) wsm[threadIdx.x] = (A)cf.g[threadIdx.x];
    __syncthreads();
    A wr[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) wr[j] = sizeof(A) == 8 ? wsm[j] : (A)cf.g[j];

    // Sweeps.  Thread t computes the XC_V outputs starting at s r + XC_V t from one window of
    // XC_V + 2r cells in registers, so a cell is read from shared memory (XC_V + 2r) / XC_V
    // times per sweep instead of 2r + 1 times.  Outputs past the valid span [s r, W - s r) are
    // computed from stale cells and never read by a valid output.
    // FP64 is bound by the FP64 pipe rather than by shared memory, and keeps one output per
    // thread and iteration (measured 9 % faster there).  Its sweep takes the span in rows of 32
    // cells, row k to warp (k + rot) mod (warps), with rot advancing by one per sweep and per
    // CTA: a span of rows that is not a multiple of the warp count leaves its extra rows to
    // other warps, and so to other SM sub-partitions, from sweep to sweep.  Each output is the
    // same multiply-add chain whichever warp computes it.
    A *src = buf0, *dst = buf1;
    for (int s = 1; s <= sweeps; ++s) {
        if constexpr (sizeof(A) == 8) {
            const int lo = s * R, hi = W - s * R;
            constexpr int NW = NT / 32;
            const int rot = (s + (int)blockIdx.x) % NW;
            int k0 = (int)(threadIdx.x >> 5) - rot;
            if (k0 < 0) k0 += NW;
            for (int p = lo + 32 * k0 + (int)(threadIdx.x & 31); p < hi; p += NT) {
                A acc = A(0);
#pragma unroll
                for (int j = -R; j <= R; ++j) acc = mac<A>(acc, wr[j + R], src[XC_PAD + p + j]);
                dst[XC_PAD + p] = acc;
            }
            __syncthreads();
            A *t = src;
            src = dst;
            dst = t;
            continue;
        }
        const int q0 = s * R + XC_V * threadIdx.x;
        const A *wp = src + XC_PAD + q0 - R;
        A win[XC_V + 2 * R];  // cells q0 - R .. q0 + XC_V - 1 + R
#pragma unroll
        for (int k = 0; k < XC_V + 2 * R; ++k) win[k] = wp[k];
        A *dp = dst + XC_PAD + q0;
#pragma unroll
        for (int v = 0; v < XC_V; ++v) {
            A acc = A(0);
#pragma unroll
            for (int j = -R; j <= R; ++j) acc = mac<A>(acc, (A)cf.g[j + R], win[R + v + j]);
            dp[v] = acc;
        }
        __syncthreads();
        A *t = src;
        src = dst;
        dst = t;
    }

    // write the chunk (+ periodic images of the array ends)
    const A *res = src + XC_PAD + H;
    if (full) {
        VT *d = reinterpret_cast<VT *>(outx + c0);
        for (int v = threadIdx.x; v < CHUNK / V; v += NT) {
            VT x;
            T *e = reinterpret_cast<T *>(&x);
#pragma unroll
            for (int u = 0; u < V; ++u) e[u] = (T)res[v * V + u];
            d[v] = x;
        }
    } else {
        for (int p = threadIdx.x; p < CHUNK && c0 + p < n; p += NT)
            outx[c0 + p] = (T)res[p];
    }
    if (images) {
        for (int p = threadIdx.x; p < CHUNK; p += NT) {
            const int64_t gi = c0 + p;
            if (gi >= n) break;
            if (gi < R) outx[gi + n] = (T)res[p];
            if (gi >= n - R) outx[gi - n] = (T)res[p];
        }
    }
}

// Launched with programmatic dependent launch: the next launch in the stream (the next sweeps
// of a call, or the next call) is dispatched while this grid runs, and waits in pdl_wait for
// this grid's completion before its first global-memory access.
template <typename T, int R, int NT>
__global__ void __launch_bounds__(NT, xc_minb<T, NT>())
xcorr_kernel(const T *__restrict__ in, T *__restrict__ out, Geom geo, XCoef<T> cf, int sweeps, int periodic,
             int images, int chunk_len) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_launch_dependents();
    pdl_wait();
    xcorr_chunk<T, R, NT>(in, out, geo, cf, sweeps, periodic, images, blockIdx.x, smem_raw, chunk_len);
}

template <typename T, int R>
static cudaError_t run(const void *in, void *out, const Geom &g, const void *coeffs, int sweeps,
                       bool periodic, bool images, cudaStream_t s) {
    using A = typename XAcc<T>::type;
    XCoef<T> cf{};
    for (int j = 0; j < 2 * R + 1; ++j) cf.g[j] = static_cast<const T *>(coeffs)[j];
    int chunk_len = xc_chunk<T>();
    bool wide = false;  // FP64: whole waves of 512-thread CTAs
    if (sizeof(T) == 8) {
        // whole waves of two 512-thread CTAs per SM (chunks of at most 4096 cells) while the
        // input and output fill at most 7/8 of L2 together, else 2048-cell chunks in
        // 256-thread CTAs (at 2^23 cells the two arrays are 134 MB, just under GB300's L2
        // capacity, and the 256-thread CTAs were 2.7 % faster)
        const int64_t wave = 2 * (int64_t)device_sms();
        const int64_t l2 = device_l2_bytes();
        wide = 2 * (int64_t)sizeof(T) * g.n[0] <= l2 - l2 / 8;
        if (wide) {
            const int64_t waves = std::max<int64_t>(1, (g.n[0] + wave * chunk_len - 1) / (wave * chunk_len));
            const int64_t per = (g.n[0] + wave * waves - 1) / (wave * waves);
            chunk_len = (int)std::min<int64_t>(chunk_len, std::max<int64_t>(256, (per + 1) & ~int64_t(1)));
        } else {
            chunk_len = XC_F64_MULTI_CHUNK;
        }
    }
    const size_t smem = sizeof(A) == 8 ? 2 * sizeof(A) * xc_f64_stride(chunk_len, sweeps * R)
                                       : 2 * sizeof(A) * XC_BUF;
    const unsigned blocks = (unsigned)((g.n[0] + chunk_len - 1) / chunk_len);
    auto k = xcorr_kernel<T, R, XC_THREADS>;
    if constexpr (sizeof(T) == 8) {
        if (wide) k = xcorr_kernel<T, R, XC_T64>;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(k, dim3(blocks), dim3(wide ? XC_T64 : XC_THREADS), smem, s, static_cast<const T *>(in),
                      static_cast<T *>(out), g, cf, sweeps, periodic ? 1 : 0, images ? 1 : 0, chunk_len);
}

template <typename T>
static cudaError_t run_r(int r, const void *in, void *out, const Geom &g, const void *coeffs,
                         int sweeps, bool periodic, bool images, cudaStream_t s) {
    switch (r) {
    case 0: return run<T, 0>(in, out, g, coeffs, sweeps, periodic, images, s);
    case 1: return run<T, 1>(in, out, g, coeffs, sweeps, periodic, images, s);
    case 2: return run<T, 2>(in, out, g, coeffs, sweeps, periodic, images, s);
    case 3: return run<T, 3>(in, out, g, coeffs, sweeps, periodic, images, s);
    case 4: return run<T, 4>(in, out, g, coeffs, sweeps, periodic, images, s);
    default: break;
    }
    if constexpr (std::is_same<T, float>::value) {
        switch (r) {
        case 5: return run<T, 5>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 6: return run<T, 6>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 7: return run<T, 7>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 8: return run<T, 8>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 9: return run<T, 9>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 10: return run<T, 10>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 11: return run<T, 11>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 12: return run<T, 12>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 13: return run<T, 13>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 14: return run<T, 14>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 15: return run<T, 15>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 16: return run<T, 16>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 17: return run<T, 17>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 18: return run<T, 18>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 19: return run<T, 19>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 20: return run<T, 20>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 21: return run<T, 21>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 22: return run<T, 22>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 23: return run<T, 23>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 24: return run<T, 24>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 25: return run<T, 25>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 26: return run<T, 26>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 27: return run<T, 27>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 28: return run<T, 28>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 29: return run<T, 29>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 30: return run<T, 30>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 31: return run<T, 31>(in, out, g, coeffs, sweeps, periodic, images, s);
        case 32: return run<T, 32>(in, out, g, coeffs, sweeps, periodic, images, s);
        default: break;
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_xcorr(int dtype, int r, const void *in, void *out, const Geom &g,
                         const void *coeffs, int sweeps, bool periodic, bool images,
                         cudaStream_t s) {
    if (sweeps < 1 || sweeps > xcorr_max_sweeps_per_launch(r)) return cudaErrorInvalidValue;
    switch (dtype) {
    case 0: return run_r<int32_t>(r, in, out, g, coeffs, sweeps, periodic, images, s);
    case 1: return run_r<double>(r, in, out, g, coeffs, sweeps, periodic, images, s);
    case 2: return run_r<float>(r, in, out, g, coeffs, sweeps, periodic, images, s);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ batched (serving)

// FP32, radius 3, one periodic sweep per item, with periodic images.
__global__ void __launch_bounds__(XC_THREADS)
xcorr_batch_kernel(const BatchHeader *hdr, const BatchXcorr *items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int total = hdr->xc_ctas, n = hdr->n_xc;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].cta_begin <= vb) lo = mid; else hi = mid - 1;
        }
        const BatchXcorr &it = items[lo];
        XCoef<float> cf{};
        for (int j = 0; j < 7; ++j) cf.g[j] = it.w[j];
        const Geom g = it.g;
        xcorr_chunk<float, 3>(it.in, it.out, g, cf, 1, 1, 1, vb - it.cta_begin, smem_raw);
        __syncthreads();
    }
}

static size_t xcorr_batch_smem() { return 2 * sizeof(float) * XC_BUF; }

int xcorr_batch_grid() {
    static int grid[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 152;
    if (!grid[dev]) {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, xcorr_batch_kernel, XC_THREADS, xcorr_batch_smem());
        grid[dev] = std::max(o, 1) * device_sms();
    }
    return grid[dev];
}

int xcorr_batch_chunk() { return xc_chunk<float>(); }

cudaError_t launch_xcorr_batch(const BatchHeader *hdr, const BatchXcorr *items, unsigned *err, int grid,
                               cudaStream_t s) {
    (void)err;
    xcorr_batch_kernel<<<grid, XC_THREADS, xcorr_batch_smem(), s>>>(hdr, items);
    return cudaGetLastError();
}

}  // namespace stn
