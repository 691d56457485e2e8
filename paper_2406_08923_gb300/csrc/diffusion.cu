// diffusion.cu -- forward-Euler step of df/dt = alpha lap f (Sec. 3.2, Eqs. 4-7) in 3D.
//
// The Euler update and the three axis Laplacians fold into one 19-point cross-correlation
// (Eqs. 5 and 7): f' = g0 f + sum_axes sum_{a=1..3} g_{axis,a} (f(+a) + f(-a)).
//
// This file holds the FP64 kernel family (FP64 on GB300 is bound by the FP64 pipe, ~1/60 of
// the FP32 rate); FP32 has its own issue-lean kernel in diffusion_f32.cu.
//
// GB300 design (2.5D z-streaming):
//   * A CTA owns a TX x TY tile of the xy-plane (TX = 32 VX, TY = BY RY) and marches along z
//     over a short chunk of planes (4), so the grid is tens of waves of small CTAs.  Each padded input plane tile
//     (TX + 8) x (TY + 6) arrives by one TMA load (cp.async.bulk.tensor.3d) in a ring of
//     NSLOT shared-memory slots, completion on one mbarrier per slot; loads run NSLOT - 3
//     planes ahead of the compute.
//   * A thread owns VX = 2 VP consecutive x cells in RY rows and computes them as VP pairs
//     (the pair template also admits FP32 with Blackwell's packed FP32x2 FMA/ADD).  Shared
//     memory is read with 16-byte vector loads.
//   * Each iteration computes ZB consecutive z planes (register blocking in z).  The
//     z-columns (planes z-3..z+ZB+2) live in a register queue that shifts by ZB once per
//     iteration, so z-neighbours cost no shared-memory traffic and the per-iteration work
//     (mbarrier waits, the block barrier, refills) is amortised over VX x RY x ZB cells.
//   * Outputs are stored once as vectors.  Threads whose cells lie within r of a face also
//     store the periodic images (Eq. 2) on a slow path, so no separate halo pass is needed.
//   * Consecutive steps are launched with programmatic dependent launch (see pdl_wait).
//   * Waits are bounded (globaltimer); on expiry the CTA records ERR_TIMEOUT, drains its
//     in-flight TMA loads (again bounded) and returns.
#include <algorithm>

#include "internal.h"

namespace stn {

// Ring slot and mbarrier phase parity of plane j for a power-of-two ring depth N.
template <int N> __device__ __forceinline__ int slot_of(int j) { return (int)((unsigned)j & (N - 1)); }
template <int N> __device__ __forceinline__ uint32_t parity_of(int j) { return ((unsigned)j / (unsigned)N) & 1u; }

// Pair arithmetic: PK selects Blackwell's packed FP32x2 instructions for float; otherwise
// the two lanes are computed with scalar instructions.
template <typename T, bool PK> struct PairOps;
template <> struct PairOps<float, true> {
    using P = float2;
    static __device__ __forceinline__ P add(P a, P b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ P mul(P a, P b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ P fma2(P a, P b, P c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ P make(float a, float b) { return make_float2(a, b); }
};
template <> struct PairOps<float, false> {
    using P = float2;
    static __device__ __forceinline__ P add(P a, P b) { return make_float2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ P mul(P a, P b) { return make_float2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ P fma2(P a, P b, P c) {
        return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
    }
    static __device__ __forceinline__ P make(float a, float b) { return make_float2(a, b); }
};
template <bool PK> struct PairOps<double, PK> {
    using P = double2;
    static __device__ __forceinline__ P add(P a, P b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ P mul(P a, P b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ P fma2(P a, P b, P c) {
        return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
    }
    static __device__ __forceinline__ P make(double a, double b) { return make_double2(a, b); }
};

template <typename T> struct DC {
    T g0;
    T ga[3][4];  // [axis][a-1]
};

template <typename T, int VP, int BY, int RY, int ZB, int NSLOT, int R>
struct DiffCfg {
    static constexpr int VX = 2 * VP;
    static constexpr int HX = 4;  // x halo kept in shared memory: 16 B aligned TMA box start
    static constexpr int TX = 32 * VX;
    static constexpr int TY = BY * RY;
    static constexpr int TXP = TX + 2 * HX;
    static constexpr int ROWS = TY + 2 * R;
    static constexpr int SLOT_ELEMS = ((TXP * ROWS * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
    static constexpr uint32_t BOX_BYTES = TXP * ROWS * sizeof(T);
    static constexpr size_t SMEM = (size_t)NSLOT * SLOT_ELEMS * sizeof(T) + 128;
    // elements per shared-memory vector load: 16 bytes, or the whole VX group if smaller
    static constexpr int LV = (VX * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : VX;
    static_assert((TXP * sizeof(T)) % 16 == 0, "TMA box inner extent must be a multiple of 16 B");
    static_assert(TXP <= 256 && ROWS <= 256, "TMA box extents are limited to 256");
    static_assert(R >= 1 && R <= HX, "radius 1..4: the x window holds 4 neighbours per side");
    static_assert(NSLOT >= ZB + R + 1, "ring: ZB + R planes in use plus one refill");
    static_assert((NSLOT & (NSLOT - 1)) == 0, "ring depth is a power of two (slot = j & (NSLOT-1))");
    static_assert(VX % LV == 0 && HX % LV == 0 && TXP % LV == 0, "vector loads must stay aligned");
};

// Load `n` consecutive elements (n a multiple of LV) at an LV-aligned shared address.
template <typename T, int LV, int N>
__device__ __forceinline__ void ld_vec(const T *p, T (&dst)[N]) {
    static_assert(N % LV == 0, "");
#pragma unroll
    for (int i = 0; i < N / LV; ++i) {
        if constexpr (LV * sizeof(T) == 16) {
            const uint4 v = *reinterpret_cast<const uint4 *>(p + i * LV);
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int u = 0; u < LV; ++u) dst[i * LV + u] = e[u];
        } else if constexpr (LV * sizeof(T) == 8) {
            const uint2 v = *reinterpret_cast<const uint2 *>(p + i * LV);
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int u = 0; u < LV; ++u) dst[i * LV + u] = e[u];
        } else {
            dst[i] = p[i];
        }
    }
}

// One xy-tile of one z-chunk: the whole 2.5D pipeline of a CTA.  `map` may point at a
// __grid_constant__ parameter or at a descriptor in global memory (batched launches).
// Returns false if a bounded wait expired (ERR_TIMEOUT recorded, loads drained).
template <typename T, int VP, int BY, int RY, int ZB, int NSLOT, bool PK, bool PDL, int R>
__device__ __forceinline__ bool diffusion_tile(const CUtensorMap *map, T *__restrict__ out, const Geom &g,
                                               const DC<T> &c, int tile_x, int tile_y, int tile_z, int zc,
                                               int images, unsigned *err, T *ring, uint64_t *full) {
    using Cfg = DiffCfg<T, VP, BY, RY, ZB, NSLOT, R>;
    using O = PairOps<T, PK>;
    using P = typename O::P;
    constexpr int VX = Cfg::VX, LV = Cfg::LV;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int x0 = tile_x * Cfg::TX, y0 = tile_y * Cfg::TY;
    const int zc0 = tile_z * zc;
    const int nx = (int)g.n[0], ny = (int)g.n[1], nz = (int)g.n[2];
    const int zend = min(nz, zc0 + zc);
    const int count = zend - zc0;
    const int nplanes = count + 2 * R;  // planes zc0-R .. zend+R-1
    const int x = x0 + lane * VX;       // first of this thread's VX cells
    const int yb = y0 + wy * RY;        // first of its RY rows

    // The weights go through shared memory into registers, so that the FP64 multiply-adds take
    // register operands: left as kernel parameters they become constant-bank operands, which
    // slowed the FP64 cross-correlation's multiply-adds by 12 %.
    __shared__ T wsm[1 + 3 * R];
    if (threadIdx.x < 1 + 3 * R)
        wsm[threadIdx.x] = threadIdx.x == 0 ? c.g0 : c.ga[(threadIdx.x - 1) / R][(threadIdx.x - 1) % R];
    if (threadIdx.x == 0) {
        tma_prefetch_desc(map);
        for (int s = 0; s < NSLOT; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (PDL) {  // the input is the previous step's output: wait for that kernel to finish
        pdl_launch_dependents();
        pdl_wait();
    }

    const int bx = (int)g.off[0] + x0 - Cfg::HX;
    const int by0 = (int)g.off[1] + y0 - R;
    const int bz0 = (int)g.off[2] + zc0 - R;
    auto issue = [&](int j) {  // plane j (0-based from zc0-3) into its ring slot
        const int s = slot_of<NSLOT>(j);
        mbar_arrive_expect_tx(&full[s], Cfg::BOX_BYTES);
        tma_load_3d(ring + s * Cfg::SLOT_ELEMS, map, &full[s], bx, by0, bz0 + j);
    };
    int issued = 0;
    if (threadIdx.x == 0)
        for (; issued < NSLOT && issued < nplanes; ++issued) issue(issued);

    // element offset of (row 0 of this thread, first cell) inside a slot
    const int own = (wy * RY + R) * Cfg::TXP + Cfg::HX + lane * VX;

    // weights as pairs, in registers up to R = 3; at R = 4 the 8-warp tile would pass 128
    // registers and lose its second CTA per SM (measured 0.94 against 0.82 ms per step), so
    // there they stay kernel parameters
    auto wt = [&](int i) -> T { return R <= 3 ? wsm[i] : (i == 0 ? c.g0 : c.ga[(i - 1) / R][(i - 1) % R]); };
    const P G0 = O::make(wt(0), wt(0));
    P GA[3][R];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) GA[a][b] = O::make(wt(1 + a * R + b), wt(1 + a * R + b));

    // z queue: Q[k] holds plane z-R+k of the iteration's first output plane z (k < ZB + 2R)
    P Q[ZB + 2 * R][RY][VP];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {  // prologue: planes zc0-R .. zc0+R-1 into Q[0..2R-1]
        ok = ok && mbar_wait_bounded(&full[slot_of<NSLOT>(j)], parity_of<NSLOT>(j));
        const T *sp = ring + slot_of<NSLOT>(j) * Cfg::SLOT_ELEMS + own;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            T e[VX];
            if (ok) ld_vec<T, LV>(sp + r * Cfg::TXP, e);
            else {
#pragma unroll
                for (int u = 0; u < VX; ++u) e[u] = T(0);
            }
#pragma unroll
            for (int p = 0; p < VP; ++p) Q[j][r][p] = O::make(e[2 * p], e[2 * p + 1]);
        }
    }
    bool bad = __syncthreads_or(!ok);
    // planes j = 0..2 are never read from shared memory again: refill their slots
    if (!bad && threadIdx.x == 0)
        for (; issued < NSLOT + R && issued < nplanes; ++issued) issue(issued);

    // Periodic images (Eq. 2) of this thread's cells.  z- and y-images repeat the row's vector
    // store at a shifted plane/row (warp-uniform).  x-images: threads holding cells within 4 of
    // a face store their whole vector again, shifted by -+nx, into the halo and the unused
    // padding next to it (when nx is a multiple of VX); otherwise per-cell scalar stores.
    const bool full_tile = x + VX <= nx && yb + RY <= ny;
    const bool any_cell = x < nx && yb < ny;
    const bool xvec = (nx % VX == 0) && nx >= 8 && g.off[0] >= 4 && g.pad[0] >= g.off[0] + nx + 4;
    int xshift = 0;  // interior-coordinate shift of this thread's x-image, 0 if none
    int xmask = 0;   // scalar fallback: bit u set if cell x+u has an image
    if (xvec) {
        if (x < 4) xshift = nx;
        else if (x >= nx - 4) xshift = -nx;
    } else {
#pragma unroll
        for (int u = 0; u < VX; ++u) {
            if (x + u < R) { xmask |= 1 << u; xshift = nx; }
            else if (x + u >= nx - R) { xmask |= 1 << u; xshift = -nx; }
        }
    }
    int yshift[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) yshift[r] = (yb + r < R) ? ny : (yb + r >= ny - R) ? -ny : 0;
    if (!images) {
        xshift = 0;
        xmask = 0;
#pragma unroll
        for (int r = 0; r < RY; ++r) yshift[r] = 0;
    }
    const int64_t pitch_y = g.pad[0], pitch_z = g.pad[0] * g.pad[1];
    T *optr = out + g.idx(x, yb, zc0);

    for (int m = 0; !bad && m < count; m += ZB) {
        // leading planes j = m+2R .. m+2R+ZB-1 (those that exist) enter the queue at Q[2R..]
#pragma unroll
        for (int b = 0; b < ZB; ++b) {
            const int jl = m + 2 * R + b;
            if (jl < nplanes) {
                ok = ok && mbar_wait_bounded(&full[slot_of<NSLOT>(jl)], parity_of<NSLOT>(jl));
                if (ok && any_cell) {
                    const T *lp = ring + slot_of<NSLOT>(jl) * Cfg::SLOT_ELEMS + own;
#pragma unroll
                    for (int r = 0; r < RY; ++r) {
                        T le[VX];
                        ld_vec<T, LV>(lp + r * Cfg::TXP, le);
#pragma unroll
                        for (int p = 0; p < VP; ++p) Q[2 * R + b][r][p] = O::make(le[2 * p], le[2 * p + 1]);
                    }
                }
            }
        }
        if (ok && any_cell) {
#pragma unroll
            for (int b = 0; b < ZB; ++b) {
                if (m + b < count) {
                    const int z = zc0 + m + b;
                    const T *cp = ring + slot_of<NSLOT>(m + b + R) * Cfg::SLOT_ELEMS + own;
                    // y column: rows -3 .. RY+2 of this thread's cells, as pairs
                    P Y[RY + 2 * R][VP];
#pragma unroll
                    for (int d = 0; d < RY + 2 * R; ++d) {
                        T e[VX];
                        ld_vec<T, LV>(cp + (d - R) * Cfg::TXP, e);
#pragma unroll
                        for (int p = 0; p < VP; ++p) Y[d][p] = O::make(e[2 * p], e[2 * p + 1]);
                    }
                    P res[RY][VP];
#pragma unroll
                    for (int r = 0; r < RY; ++r) {
                        // x window: cells -4 .. VX+3 of row r
                        T E[VX + 8];
                        ld_vec<T, LV>(cp + r * Cfg::TXP - 4, E);
#pragma unroll
                        for (int p = 0; p < VP; ++p) {
                            const int i0 = 4 + 2 * p;  // E index of the pair's first cell
                            P acc = O::mul(G0, Y[r + R][p]);
                            // offset a: x pairs from E (even offsets aligned, odd offsets two
                            // scalar adds), then the y and z pairs
#pragma unroll
                            for (int a = 1; a <= R; ++a) {
                                const P sx = (a % 2 == 0)
                                                 ? O::add(O::make(E[i0 + a], E[i0 + 1 + a]), O::make(E[i0 - a], E[i0 + 1 - a]))
                                                 : O::make(E[i0 + a] + E[i0 - a], E[i0 + 1 + a] + E[i0 + 1 - a]);
                                acc = O::fma2(GA[0][a - 1], sx, acc);
                                acc = O::fma2(GA[1][a - 1], O::add(Y[r + R + a][p], Y[r + R - a][p]), acc);
                                acc = O::fma2(GA[2][a - 1], O::add(Q[b + R + a][r][p], Q[b + R - a][r][p]), acc);
                            }
                            res[r][p] = acc;
                        }
                    }
                    T *op = optr + b * pitch_z;
                    if (full_tile) {
                        const int zshift = images ? ((z < R) ? nz : (z >= nz - R) ? -nz : 0) : 0;
#pragma unroll
                        for (int zi = 0; zi < 2; ++zi) {
                            if (zi == 1 && zshift == 0) break;
                            T *zp = op + (zi ? (int64_t)zshift * pitch_z : 0);
#pragma unroll
                            for (int r = 0; r < RY; ++r) {
#pragma unroll
                                for (int yi = 0; yi < 2; ++yi) {
                                    if (yi == 1 && yshift[r] == 0) break;
                                    T *rp = zp + (int64_t)(r + (yi ? yshift[r] : 0)) * pitch_y;
#pragma unroll
                                    for (int xi = 0; xi < 2; ++xi) {
                                        if (xi == 1 && (!xvec || xshift == 0)) break;
                                        T *xp = rp + (xi ? xshift : 0);
                                        if constexpr (VP == 2 && sizeof(T) == 4) {  // one 16-byte store
                                            *reinterpret_cast<float4 *>(xp) =
                                                make_float4(res[r][0].x, res[r][0].y, res[r][1].x, res[r][1].y);
                                        } else {
#pragma unroll
                                            for (int p = 0; p < VP; ++p) *reinterpret_cast<P *>(xp + 2 * p) = res[r][p];
                                        }
                                    }
                                    if (xmask) {
#pragma unroll
                                        for (int p = 0; p < VP; ++p) {
                                            if (xmask & (1 << (2 * p))) rp[2 * p + xshift] = res[r][p].x;
                                            if (xmask & (2 << (2 * p))) rp[2 * p + 1 + xshift] = res[r][p].y;
                                        }
                                    }
                                }
                            }
                        }
                    } else {
                        // ragged tile: element-wise stores with bounds checks and all images
#pragma unroll
                        for (int r = 0; r < RY; ++r)
#pragma unroll
                            for (int p = 0; p < VP; ++p) {
                                const T v2[2] = {res[r][p].x, res[r][p].y};
#pragma unroll
                                for (int u = 0; u < 2; ++u)
                                    if (x + 2 * p + u < nx && yb + r < ny)
                                        store_with_images(out, g, R, images != 0, x + 2 * p + u, yb + r, z, v2[u]);
                            }
                    }
                }
            }
            // shift the queue by ZB planes
#pragma unroll
            for (int k = 0; k < 2 * R; ++k)
#pragma unroll
                for (int r = 0; r < RY; ++r)
#pragma unroll
                    for (int p = 0; p < VP; ++p) Q[k][r][p] = Q[k + ZB][r][p];
        }
        optr += ZB * pitch_z;
        bad = __syncthreads_or(!ok);
        // planes j < m + ZB + 3 are retired: refill the ring up to NSLOT planes ahead
        if (!bad && threadIdx.x == 0) {
            const int lim = min(nplanes, m + ZB + R + NSLOT);
            for (; issued < lim; ++issued) issue(issued);
        }
    }
    if (bad && threadIdx.x == 0) {
        atomicOr(err, ERR_TIMEOUT);
        // drain loads still in flight before the CTA's shared memory is released
        for (int j = max(0, issued - NSLOT); j < issued; ++j)
            (void)mbar_wait_bounded(&full[slot_of<NSLOT>(j)], parity_of<NSLOT>(j), 100000000ull);
    }
    return !bad;
}

template <typename T, int VP, int BY, int RY, int ZB, int NSLOT, bool PK, int R>
__global__ void __launch_bounds__(32 * BY)
diffusion_kernel(const __grid_constant__ CUtensorMap map_in, T *__restrict__ out, Geom g, DC<T> c,
                 int zc, int images, unsigned *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations are kept 128-byte aligned (dynamic smem has 128 spare bytes)
    T *ring = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full[NSLOT];
    diffusion_tile<T, VP, BY, RY, ZB, NSLOT, PK, true, R>(&map_in, out, g, c, blockIdx.x, blockIdx.y, blockIdx.z,
                                                          zc, images, err, ring, full);
}

// ------------------------------------------------------------------ variants / launch

// Number of z-chunks for a grid of `tiles` xy-tiles: maximise the fraction of the last wave
// that is occupied, with a mild penalty for the 6 extra planes each chunk re-reads.
int choose_zchunks(int tiles, int nz, int slots, double reread_weight) {
    int best = 1;
    double best_score = -1.0;
    for (int c = 1; c <= std::min(nz, 512); ++c) {
        const int zc = (nz + c - 1) / c;
        const int cc = (nz + zc - 1) / zc;
        if (cc != c) continue;
        const long ctas = (long)tiles * c;
        const long waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots);
        const double score = eff * (1.0 - reread_weight * 6.0 / (zc + 6.0)) - 1e-4 * c;
        if (score > best_score) {
            best_score = score;
            best = c;
        }
    }
    return best;
}

int zchunk_len(int zc, int nz, int zmode) {
    const int v = zmode == 1 ? (zc + 1) / 2 : zmode == 2 ? 2 * zc : zc;
    return std::max(1, std::min(nz, v));
}

int device_sms() {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms[dev] = 152;
    return sms[dev];
}

template <typename T, int VP, int BY, int RY, int ZB, int NSLOT, bool PK, int R>
static cudaError_t run(const CUtensorMap *map, void *out, const Geom &g, const DiffCoef &dc, bool images,
                       unsigned *err, cudaStream_t s, int zmode) {
    using Cfg = DiffCfg<T, VP, BY, RY, ZB, NSLOT, R>;
    DC<T> c;
    c.g0 = (T)dc.g0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 4; ++b) c.ga[a][b] = (T)dc.ga[a][b];
    auto k = diffusion_kernel<T, VP, BY, RY, ZB, NSLOT, PK, R>;
    static int occ[64] = {};  // resident CTAs per SM, per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (!occ[dev]) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, 32 * BY, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        occ[dev] = std::max(o, 1);
    }
    const int tx = (int)((g.n[0] + Cfg::TX - 1) / Cfg::TX), ty = (int)((g.n[1] + Cfg::TY - 1) / Cfg::TY);
    const int nz = (int)g.n[2];
    // FP64 is bound by the FP64 pipe, and the y/z halo re-reads of short chunks hit in L2, so
    // chunks are short (4 planes): tens of waves of small CTAs keep the pipe evenly fed through
    // every CTA's start-up and the grid's tail (5 % faster than whole waves of long chunks at
    // 256^3).
    const int zc = zchunk_len(std::min(nz, 4), nz, zmode);
    dim3 grid(tx, ty, (unsigned)((nz + zc - 1) / zc));
    return launch_pdl(k, grid, dim3(32 * BY), Cfg::SMEM, s, *map, static_cast<T *>(out), g, c, zc, images ? 1 : 0,
                      err);
}

// Variant table: (VP pairs per row, BY warps, RY rows, ZB planes, NSLOT, packed FP32x2).  The
// autotuner times each on the problem and keeps the fastest.  Radius 3 (the 6th-order step)
// carries the tuned set; the other radii of the sweep use its first shape.
#define DIFF_VARIANTS_F64(X) \
    X(1, 8, 1, 2, 8, false)  \
    X(1, 4, 1, 2, 8, false)  \
    X(1, 8, 1, 1, 8, false)  \
    X(1, 4, 2, 2, 8, false)
#define DIFF_VARIANTS_F64_OTHER(X) X(1, 8, 1, 2, 8, false)
static const char *F64_NAMES[] = {"vx2_by8_ry1_zb2_s8", "vx2_by4_ry1_zb2_s8", "vx2_by8_ry1_zb1_s8",
                                  "vx2_by4_ry2_zb2_s8"};
static const char *F64_NAMES_OTHER[] = {"?", "f64_r1_vx2_by8_ry1_zb2_s8", "f64_r2_vx2_by8_ry1_zb2_s8", "?",
                                        "f64_r4_vx2_by8_ry1_zb2_s8"};

int diffusion_num_variants(int dtype, int r) {
    if (dtype != 1) return diffusion_f32_num_variants(r);
    return r == 3 ? 4 : (r >= 1 && r <= 4 ? 1 : 0);
}

const char *diffusion_variant_name(int dtype, int r, int v) {
    if (dtype != 1) return diffusion_f32_variant_name(r, v);
    if (v < 0 || v >= diffusion_num_variants(dtype, r)) return "?";
    return r == 3 ? F64_NAMES[v] : F64_NAMES_OTHER[r];
}

void diffusion_box(int dtype, int r, int v, int box[3]) {
    if (dtype != 1) return diffusion_f32_box(r, v, box);
    int i = 0;
    auto put = [&](int vp, int by, int ry) {
        if (i++ == v) { box[0] = 64 * vp + 8; box[1] = by * ry + 2 * r; box[2] = 1; }
    };
#define X(VP, BY, RY, ZB, NS, PK) put(VP, BY, RY);
    if (r == 3) {
        DIFF_VARIANTS_F64(X)
    } else {
        DIFF_VARIANTS_F64_OTHER(X)
    }
#undef X
}

template <int R>
static cudaError_t dispatch_f64(int variant, const CUtensorMap *map, void *out, const Geom &g, const DiffCoef &c,
                                bool images, unsigned *err, cudaStream_t s, int zmode) {
    using T = double;
    int i = 0;
    cudaError_t res = cudaErrorInvalidValue;
#define X(VP, BY, RY, ZB, NS, PK) \
    if (i++ == variant) res = run<T, VP, BY, RY, ZB, NS, PK, R>(map, out, g, c, images, err, s, zmode);
    if constexpr (R == 3) {
        DIFF_VARIANTS_F64(X)
    } else {
        DIFF_VARIANTS_F64_OTHER(X)
    }
#undef X
    return res;
}

cudaError_t launch_diffusion(int dtype, const CUtensorMap *map, void *out, const Geom &g, const DiffCoef &c,
                             bool images, unsigned *err, cudaStream_t s, int variant, int zmode) {
    if (dtype == 2) return launch_diffusion_f32(map, static_cast<float *>(out), g, c, images, err, s, variant, zmode);
    if (dtype != 1) return cudaErrorInvalidValue;
    switch (c.r) {
    case 1: return dispatch_f64<1>(variant, map, out, g, c, images, err, s, zmode);
    case 2: return dispatch_f64<2>(variant, map, out, g, c, images, err, s, zmode);
    case 3: return dispatch_f64<3>(variant, map, out, g, c, images, err, s, zmode);
    case 4: return dispatch_f64<4>(variant, map, out, g, c, images, err, s, zmode);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace stn
