// norms.cu -- per-field FP64 reductions over the interior: sum f, sum f^2, max |f| and, for
// the MHD log-density, the mass sum exp(lnrho).  Used to judge accuracy and conservation
// (Sec. 5.1 verification; Eq. A1 for the mass).
//
// Two passes with a fixed reduction tree, so results are bit-reproducible run to run:
// pass 1: NB blocks stride over (row, segment) pieces of the interior (coalesced along x)
// and write NB x nfields x 4 partials; pass 2: one warp per (field, quantity) reduces the
// partials in a fixed order.
#include <mutex>

#include "internal.h"

namespace stn {

constexpr int NORM_THREADS = 256;
constexpr int NORM_BLOCKS = 2 * 152;
constexpr int NORM_SEG = 4096;
constexpr int NORM_U = 8;  // loads in flight per thread in pass 1

int norms_blocks() { return NORM_BLOCKS; }

template <typename S> __device__ __forceinline__ double to_d(S v) { return (double)v; }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
}

// max that propagates NaN (fmax drops it): a field that has gone NaN must report a NaN
// max |f|, not the largest finite value.
__device__ __forceinline__ double nanmax(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }

__device__ __forceinline__ void warp_reduce(double &s, double &s2, double &mx, double &ms) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        mx = nanmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        ms += __shfl_xor_sync(0xffffffffu, ms, o);
    }
}

template <typename S>
__global__ void __launch_bounds__(NORM_THREADS)
norms_pass1(Ptrs8 f, int nfields, Geom g, int mass0, double *partials) {
    __shared__ double red[4][NORM_THREADS / 32];
    const int64_t nx = g.n[0], rows = g.n[1] * g.n[2];
    const int64_t segs = (nx + NORM_SEG - 1) / NORM_SEG;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < nfields; ++q) {
        const S *base = static_cast<const S *>(f.p[q]);
        const bool do_mass = mass0 && q == 0;
        double s = 0.0, s2 = 0.0, ms = 0.0;
        // max |f| as the bit pattern of |f|: for non-negative doubles the unsigned order of the
        // patterns is the numeric order, every NaN pattern lies above +inf (so a NaN wins), and
        // no FP64 compare (a slow-pipe instruction on this GPU) is needed
        unsigned long long mxb = 0ull;
        auto add = [&](double v) {
            s += v;
            s2 += v * v;
            mxb = max(mxb, (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull);
            if (do_mass) ms += exp(v);
        };
        for (int64_t piece = blockIdx.x; piece < rows * segs; piece += gridDim.x) {
            const int64_t row = piece / segs, sg = piece - row * segs;
            const int64_t y = row % g.n[1], z = row / g.n[1];
            const S *p = base + g.idx(0, y, z);
            const int64_t xe = min(nx, (sg + 1) * NORM_SEG);
            int64_t x = sg * NORM_SEG + threadIdx.x;
            // NORM_U independent loads in flight per thread, then the same accumulation order
            // (x, x + NORM_THREADS, ...) as one element at a time
            for (; x + (NORM_U - 1) * NORM_THREADS < xe; x += NORM_U * NORM_THREADS) {
                S v[NORM_U];
#pragma unroll
                for (int u = 0; u < NORM_U; ++u) v[u] = p[x + u * NORM_THREADS];
#pragma unroll
                for (int u = 0; u < NORM_U; ++u) add(to_d(v[u]));
            }
            for (; x < xe; x += NORM_THREADS) add(to_d(p[x]));
        }
        double mx = __longlong_as_double((long long)mxb);
        warp_reduce(s, s2, mx, ms);
        if (lane == 0) { red[0][warp] = s; red[1][warp] = s2; red[2][warp] = mx; red[3][warp] = ms; }
        __syncthreads();
        if (warp == 0) {
            const bool in = lane < NORM_THREADS / 32;
            s = in ? red[0][lane] : 0.0;
            s2 = in ? red[1][lane] : 0.0;
            mx = in ? red[2][lane] : 0.0;
            ms = in ? red[3][lane] : 0.0;
            warp_reduce(s, s2, mx, ms);
            if (lane == 0) {
                double *o = partials + ((int64_t)blockIdx.x * nfields + q) * 4;
                o[0] = s; o[1] = s2; o[2] = mx; o[3] = ms;
            }
        }
        __syncthreads();
    }
}

__global__ void norms_pass2(const double *partials, int nblocks, int nfields, double *out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // warp w -> (field, quantity)
    if (w >= nfields * 4) return;
    const int q = w / 4, c = w % 4;
    double acc = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
        const double v = partials[((int64_t)b * nfields + q) * 4 + c];
        acc = c == 2 ? nanmax(acc, v) : acc + v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, acc, o);
        acc = c == 2 ? nanmax(acc, v) : acc + v;
    }
    if (lane == 0) out[q * 4 + c] = acc;
}

cudaError_t launch_norms(int storage, const Ptrs8 &f, int nfields, const Geom &g, bool mass0,
                         double *partials, double *out_dev, cudaStream_t s) {
    switch (storage) {
    case 0: norms_pass1<int32_t><<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(f, nfields, g, mass0, partials); break;
    case 1: norms_pass1<double><<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(f, nfields, g, mass0, partials); break;
    case 2: norms_pass1<float><<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(f, nfields, g, mass0, partials); break;
    case 3: norms_pass1<__nv_bfloat16><<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(f, nfields, g, mass0, partials); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    norms_pass2<<<1, 32 * 4 * nfields, 0, s>>>(partials, NORM_BLOCKS, nfields, out_dev);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Allocation-free variant of the same two-pass reduction.
//
// Some callers cannot call cudaMalloc: a serving loop that has committed its whole HBM
// budget to resident fields and must not allocate (or risk an allocation failure or an
// implicit device synchronisation) while requests are in flight, or a host application
// whose device memory is owned by another allocator.  For them the pass-1 partials live
// in this file-scope device array instead of plan-owned scratch.  Its size is fixed:
// NORM_BLOCKS blocks x at most NORM_STATIC_MAX_FIELDS fields x 4 doubles = 77 824 bytes,
// held by every GPU that loads the library until the process exits.  Pass 1 writes every
// slot that pass 2 reads, so nothing needs clearing between calls; calls that overlap on
// the GPU (two streams, or two host threads) share this one array and race.
constexpr int NORM_STATIC_MAX_FIELDS = 8;
static __device__ __align__(256) double g_norm_partials[NORM_BLOCKS * NORM_STATIC_MAX_FIELDS * 4];

int norms_static_max_fields() { return NORM_STATIC_MAX_FIELDS; }

// Results packed as {sum, sum of squares, max |f|} per field, then (when mass_volume > 0)
// sum exp(field 0) * mass_volume, written to device memory.
__global__ void norms_pass2_packed(const double *partials, int nblocks, int nfields, double mass_volume,
                                   double *out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w >= nfields * 4) return;
    const int q = w / 4, c = w % 4;
    if (c == 3 && (q != 0 || !(mass_volume > 0.0))) return;
    double acc = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
        const double v = partials[((int64_t)b * nfields + q) * 4 + c];
        acc = c == 2 ? nanmax(acc, v) : acc + v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, acc, o);
        acc = c == 2 ? nanmax(acc, v) : acc + v;
    }
    if (lane == 0) {
        if (c < 3) out[3 * q + c] = acc;
        else out[3 * nfields] = acc * mass_volume;
    }
}

// Device address of g_norm_partials for the current device.  Host code cannot use the
// array's name as a device pointer (it is a host-side stand-in), so the address is looked
// up once per device with that device current, on the first call made on that device.
static cudaError_t norm_partials_address(double **addr) {
    static std::mutex mu;
    static double *cache[128] = {};
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!cache[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm_partials);
        if (e != cudaSuccess) return e;
        cache[dev] = static_cast<double *>(p);
    }
    *addr = cache[dev];
    return cudaSuccess;
}

cudaError_t launch_norms_noalloc(int storage, const Ptrs8 &f, int nfields, const Geom &g,
                                 double mass_volume, double *out_dev, cudaStream_t s) {
    if (nfields < 1 || nfields > NORM_STATIC_MAX_FIELDS) return cudaErrorInvalidValue;
    double *partials = nullptr;
    cudaError_t e = norm_partials_address(&partials);
    if (e != cudaSuccess) return e;
    const int mass0 = mass_volume > 0.0 ? 1 : 0;
    switch (storage) {
    case 0: norms_pass1<int32_t><<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(f, nfields, g, mass0, partials); break;
    case 1: norms_pass1<double><<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(f, nfields, g, mass0, partials); break;
    case 2: norms_pass1<float><<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(f, nfields, g, mass0, partials); break;
    case 3: norms_pass1<__nv_bfloat16><<<NORM_BLOCKS, NORM_THREADS, 0, s>>>(f, nfields, g, mass0, partials); break;
    default: return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    norms_pass2_packed<<<1, 32 * 4 * nfields, 0, s>>>(partials, NORM_BLOCKS, nfields, mass_volume, out_dev);
    return cudaGetLastError();
}

}  // namespace stn
