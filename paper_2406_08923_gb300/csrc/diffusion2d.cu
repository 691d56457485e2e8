// diffusion2d.cu -- forward-Euler step of the 2D heat equation (Sec. 3.2, Eqs. 4-7), radius
// r = 1..4 (the order-2r central Laplacian; the 2D part of the radius sweep of Sec. 5.3).
//
// f' = g0 f + sum_{axis in x,y} sum_{a=1..R} g_{axis,a} (f(+a) + f(-a)).
//
// A 2D step has no streaming axis, so each CTA owns one 32 VX x 32 tile (VX = one 16-byte
// vector of cells per thread and row) and fetches its padded tile (+4 columns, +R rows per
// side) with a single TMA load.  A thread computes VX cells in 4 consecutive rows: the column
// of rows yb-R .. yb+3+R at its x comes from 16-byte shared loads and serves every row's y
// neighbours; x neighbours come from the 16-byte vectors on either side.  Interior threads
// store one vector per row; threads at a face store element-wise with their periodic images
// (Eq. 2).  The multiply-add order per cell is x, y for a = 1 .. R, as in the 3D kernels.
// Launched with programmatic dependent launch; the one wait is bounded.
#include <algorithm>

#include "internal.h"

namespace stn {
namespace {

template <typename T, int R>
struct D2 {
    static constexpr int VX = 16 / (int)sizeof(T);  // cells per thread and row
    static constexpr int TX = 32 * VX, HX = 4, TXP = TX + 2 * HX;
    static constexpr int BY = 8, RY = 4, TY = BY * RY;
    static constexpr int ROWS = TY + 2 * R;
    static constexpr uint32_t BOX_BYTES = TXP * ROWS * sizeof(T);
    static constexpr size_t SMEM = (size_t)BOX_BYTES + 128;
    static_assert(R >= 1 && R <= HX, "radius 1..4");
    static_assert((HX * sizeof(T)) % 16 == 0 && (TXP * sizeof(T)) % 16 == 0, "16-byte aligned rows");
};

template <typename T> struct W2 {  // folded weights, passed by value
    T g0, gx[4], gy[4];
};

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

template <typename T, int N>
__device__ __forceinline__ void ld16(const T *p, T (&e)[N]) {  // N = 16 / sizeof(T)
    using V = typename Vec16<T>::type;
    const V v = *reinterpret_cast<const V *>(p);
    const T *s = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int u = 0; u < N; ++u) e[u] = s[u];
}

template <typename T, int N>
__device__ __forceinline__ void st16(T *p, const T (&e)[N]) {
    using V = typename Vec16<T>::type;
    V v;
    T *d = reinterpret_cast<T *>(&v);
#pragma unroll
    for (int u = 0; u < N; ++u) d[u] = e[u];
    *reinterpret_cast<V *>(p) = v;
}

template <typename T, int R>
__global__ void __launch_bounds__(32 * D2<T, R>::BY)
heat2d_kernel(const __grid_constant__ CUtensorMap map_in, T *__restrict__ out, Geom g, W2<T> w, int images,
              unsigned *err) {
    using Cfg = D2<T, R>;
    constexpr int VX = Cfg::VX, RY = Cfg::RY, TXP = Cfg::TXP;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int x0 = blockIdx.x * Cfg::TX, y0 = blockIdx.y * Cfg::TY;
    const int nx = (int)g.n[0], ny = (int)g.n[1];
    const int x = x0 + VX * lane, yb = y0 + RY * wy;

    // FP64: the weights go through shared memory into registers, so that the FP64 multiply-adds
    // take register operands rather than (slower) constant-bank ones
    __shared__ T wsm[9];
    if (sizeof(T) == 8 && threadIdx.x < 9)
        wsm[threadIdx.x] = threadIdx.x == 0 ? w.g0 : (threadIdx.x < 5 ? w.gx[threadIdx.x - 1] : w.gy[threadIdx.x - 5]);
    if (threadIdx.x == 0) {
        tma_prefetch_desc(&map_in);
        mbar_init(&full, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (sizeof(T) == 8) {
        w.g0 = wsm[0];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            w.gx[a] = wsm[1 + a];
            w.gy[a] = wsm[5 + a];
        }
    }
    pdl_launch_dependents();
    pdl_wait();  // the input is the previous step's output
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&full, Cfg::BOX_BYTES);
        tma_load_3d(tile, &map_in, &full, (int)g.off[0] + x0 - Cfg::HX, (int)g.off[1] + y0 - R, 0);
    }
    const bool ok = mbar_wait_bounded(&full, 0);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(err, ERR_TIMEOUT);
            (void)mbar_wait_bounded(&full, 0, 100000000ull);  // drain the load before smem is released
        }
        return;
    }
    if (x >= nx || yb >= ny) return;

    // column of rows yb-R .. yb+RY+R-1 at this thread's x
    const T *col = tile + (wy * RY) * TXP + Cfg::HX + VX * lane;  // row yb-R of the column
    T Y[RY + 2 * R][VX];
#pragma unroll
    for (int d = 0; d < RY + 2 * R; ++d) ld16<T, VX>(col + d * TXP, Y[d]);
    T res[RY][VX];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        // x window: cells x-4 .. x+VX+3 of row r (4 per side covers R <= 4)
        constexpr int NL = 4 / VX;  // 16-byte vectors on each side
        T E[VX + 8];
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            T e[VX];
            ld16<T, VX>(col + (r + R) * TXP - 4 + q * VX, e);
#pragma unroll
            for (int u = 0; u < VX; ++u) E[q * VX + u] = e[u];
            ld16<T, VX>(col + (r + R) * TXP + VX + q * VX, e);
#pragma unroll
            for (int u = 0; u < VX; ++u) E[4 + VX + q * VX + u] = e[u];
        }
#pragma unroll
        for (int u = 0; u < VX; ++u) E[4 + u] = Y[r + R][u];
#pragma unroll
        for (int u = 0; u < VX; ++u) {
            T acc = w.g0 * E[4 + u];
#pragma unroll
            for (int a = 1; a <= R; ++a) {
                acc = fma(w.gx[a - 1], E[4 + u + a] + E[4 + u - a], acc);
                acc = fma(w.gy[a - 1], Y[r + R + a][u] + Y[r + R - a][u], acc);
            }
            res[r][u] = acc;
        }
    }
    const bool full_tile = x + VX <= nx && yb + RY <= ny;
    const bool edge = images && (x < R || x + VX > nx - R || yb < R || yb + RY > ny - R);
    if (full_tile && !edge) {
#pragma unroll
        for (int r = 0; r < RY; ++r) st16<T, VX>(out + g.idx(x, yb + r, 0), res[r]);
    } else {
#pragma unroll
        for (int r = 0; r < RY; ++r)
#pragma unroll
            for (int u = 0; u < VX; ++u)
                if (x + u < nx && yb + r < ny) store_with_images(out, g, R, images != 0, x + u, yb + r, 0, res[r][u]);
    }
}

template <typename T, int R>
cudaError_t run2d(const CUtensorMap *map, void *out, const Geom &g, const DiffCoef &dc, bool images, unsigned *err,
                  cudaStream_t s) {
    using Cfg = D2<T, R>;
    auto k = heat2d_kernel<T, R>;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    W2<T> w;
    w.g0 = (T)dc.g0;
    for (int a = 0; a < 4; ++a) {
        w.gx[a] = (T)dc.ga[0][a];
        w.gy[a] = (T)dc.ga[1][a];
    }
    const dim3 grid((unsigned)((g.n[0] + Cfg::TX - 1) / Cfg::TX), (unsigned)((g.n[1] + Cfg::TY - 1) / Cfg::TY));
    return launch_pdl(k, grid, dim3(32 * Cfg::BY), Cfg::SMEM, s, *map, static_cast<T *>(out), g, w, images ? 1 : 0,
                      err);
}

template <typename T>
cudaError_t run2d_r(const CUtensorMap *map, void *out, const Geom &g, const DiffCoef &c, bool images, unsigned *err,
                    cudaStream_t s) {
    switch (c.r) {
    case 1: return run2d<T, 1>(map, out, g, c, images, err, s);
    case 2: return run2d<T, 2>(map, out, g, c, images, err, s);
    case 3: return run2d<T, 3>(map, out, g, c, images, err, s);
    case 4: return run2d<T, 4>(map, out, g, c, images, err, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

void diffusion2d_box(int dtype, int r, int box[3]) {
    const int vx = dtype == 1 ? 2 : 4;
    box[0] = 32 * vx + 8;
    box[1] = D2<float, 1>::TY + 2 * r;
    box[2] = 1;
}

cudaError_t launch_diffusion2d(int dtype, const CUtensorMap *map, void *out, const Geom &g, const DiffCoef &c,
                               bool images, unsigned *err, cudaStream_t s) {
    if (dtype == 1) return run2d_r<double>(map, out, g, c, images, err, s);
    if (dtype == 2) return run2d_r<float>(map, out, g, c, images, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace stn
