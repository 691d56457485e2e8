// norms.cu -- per-field FP64 reductions over the interior: sum f, sum f^2, max |f| and, for
// the MHD log-density, the mass sum exp(lnrho).  Used to judge accuracy and conservation
// (Sec. 5.1 verification; Eq. A1 for the mass).
//
// Two passes with a fixed reduction tree, so results are bit-reproducible run to run:
// pass 1: the NB blocks' warps stride over (row, segment) pieces of the interior, one warp per
// piece (coalesced along x, NORM_U loads in flight per lane), and each block writes
// nfields x 4 partials; pass 2: one warp per (field, quantity) reduces the NB partials in a
// fixed order.
//
// Each value costs two FP64 instructions (the add to sum f and the fused multiply-add to
// sum f^2) and, for the mass, an FP64 exp; FP64 runs at 2 instructions per cycle per SM on
// GB300, so the pass is bound by the FP64 pipe, not by HBM.  A piece is a whole row of up to
// NORM_SEG cells (a 256-cell row of a 256^3 grid fills one piece), so the index arithmetic of
// a row is paid once per 256 or more values.
#include <mutex>

#include "internal.h"

namespace stn {

constexpr int NORM_THREADS = 256;
constexpr int NORM_WARPS = NORM_THREADS / 32;
constexpr int NORM_BLOCKS = 2 * 152;
constexpr int NORM_U = 8;                     // loads in flight per lane (no mass)
constexpr int NORM_SEG = 32 * NORM_U * 8;     // cells per piece: 2048

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

// Accumulates one field's pieces for this warp: sum f, sum f^2, max |f| as a bit pattern and,
// with MASS, sum exp(f).  MASS is a template parameter so that the other fields carry no mass
// accumulation at all: with a runtime flag the compiler kept the add to the mass sum, with a
// zero operand, on every value (2.1 FP64 adds per value instead of 1, counted by ncu).
// The pieces of warp gw: gw, gw + nw, ..., each a segment sg of row (y, z).  The division of
// the first index is done once; each stride of nw pieces then advances (sg, y, z) by constant
// steps with carries, so the loop runs no 64-bit division (which this GPU emulates, partly
// with FP64 instructions that compete with the accumulation).
struct PieceWalk {
    int64_t segs, n1, pieces;
    int64_t sg, y, z;     // current piece
    int64_t dsg, dy, dz;  // the stride nw in (segment, y, z) units
    __device__ PieceWalk(const Geom &g, int64_t gw, int64_t nw) {
        segs = (g.n[0] + NORM_SEG - 1) / NORM_SEG;
        n1 = g.n[1];
        pieces = segs * g.n[1] * g.n[2];
        const int64_t row = gw / segs, drow = nw / segs;
        sg = gw - row * segs;
        y = row % n1;
        z = row / n1;
        dsg = nw - drow * segs;
        dy = drow % n1;
        dz = drow / n1;
    }
    __device__ __forceinline__ void next() {
        sg += dsg;
        int64_t carry = 0;
        if (sg >= segs) { sg -= segs; carry = 1; }
        y += dy + carry;  // dy < n1 and carry <= 1: at most one wrap
        z += dz;
        if (y >= n1) { y -= n1; z += 1; }
    }
};

template <typename S, bool MASS>
__device__ __forceinline__ void norms_field(const S *__restrict__ base, const Geom &g, int64_t gw, int64_t nw,
                                            double &s, double &s2, unsigned &mhi, unsigned &mlo, double &ms) {
    const int lane = threadIdx.x & 31;
    const int64_t nx = g.n[0];
    PieceWalk pw(g, gw, nw);
    // max |f| as the bit pattern of |f|: for non-negative doubles the unsigned order of the
    // patterns is the numeric order, and every NaN pattern lies above +inf (so a NaN wins).  The
    // pattern is kept as two 32-bit words (mhi, mlo) updated with 32-bit integer operations:
    // a 64-bit compare-and-select here cost one more FP64-pipe instruction per value (ncu), as
    // many as the sum itself.
    auto add = [&](double v) {
        s = __dadd_rn(s, v);
        s2 = __fma_rn(v, v, s2);
        const unsigned hi = (unsigned)__double2hiint(v) & 0x7fffffffu, lo = (unsigned)__double2loint(v);
        const unsigned cand = hi == mhi ? max(mlo, lo) : lo;  // mlo if hi is, or becomes, the max
        mlo = hi >= mhi ? cand : mlo;
        mhi = max(mhi, hi);
        if constexpr (MASS) ms = __dadd_rn(ms, exp(v));
    };
    // warp gw takes pieces gw, gw + nw, ...; within a piece, lane l the cells l, l + 32, ...
    for (int64_t piece = gw; piece < pw.pieces; piece += nw, pw.next()) {
        const S *p = base + g.idx(0, pw.y, pw.z);
        const int64_t xe = min(nx, (pw.sg + 1) * NORM_SEG);
        int64_t x = pw.sg * NORM_SEG + lane;
        // U independent loads in flight per lane, then the same accumulation order (x, x + 32,
        // ...) as one element at a time.  The mass path keeps fewer: its exp calls are what
        // bound it, and values live across them spill.
        constexpr int U = MASS ? 2 : NORM_U;
        for (; x + 32 * (U - 1) < xe; x += 32 * U) {
            S v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = p[x + 32 * u];
#pragma unroll
            for (int u = 0; u < U; ++u) add(to_d(v[u]));
        }
        for (; x < xe; x += 32) add(to_d(p[x]));
    }
}

template <typename S>
__global__ void __launch_bounds__(NORM_THREADS)
norms_pass1(Ptrs8 f, int nfields, Geom g, int mass0, double *partials) {
    __shared__ double red[4][NORM_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * NORM_WARPS + warp, nw = (int64_t)gridDim.x * NORM_WARPS;
    for (int q = 0; q < nfields; ++q) {
        const S *base = static_cast<const S *>(f.p[q]);
        double s = 0.0, s2 = 0.0, ms = 0.0;
        unsigned mhi = 0u, mlo = 0u;
        if (mass0 && q == 0)
            norms_field<S, true>(base, g, gw, nw, s, s2, mhi, mlo, ms);
        else
            norms_field<S, false>(base, g, gw, nw, s, s2, mhi, mlo, ms);
        double mx = __hiloint2double((int)mhi, (int)mlo);
        warp_reduce(s, s2, mx, ms);
        if (lane == 0) { red[0][warp] = s; red[1][warp] = s2; red[2][warp] = mx; red[3][warp] = ms; }
        __syncthreads();
        if (warp == 0) {
            const bool in = lane < NORM_WARPS;
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
