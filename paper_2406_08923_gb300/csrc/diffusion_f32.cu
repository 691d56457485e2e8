// diffusion_f32.cu -- FP32 forward-Euler step of the 3D heat equation (Sec. 3.2, Eqs. 4-7).
//
// The Euler update and the three axis Laplacians fold into one star-shaped cross-correlation
// (Eqs. 5 and 7): f' = g0 f + sum_axes sum_{a=1..R} g_{axis,a} (f(+a) + f(-a)), with the
// order-2R central Laplacian of radius R = 1..4 (R = 3 is the 6th-order, 19-point stencil;
// the other radii serve the radius sweep of Sec. 5.3).
//
// FP32 is bandwidth-class work on GB300 (8 B per cell-update against ~10 packed FP32
// instructions), so this kernel is built to spend as few issue slots per cell as possible:
//   * 2.5D z-streaming as in the FP64 kernel: a CTA owns a 128 x (BY RY) tile of the
//     xy-plane and marches along a chunk of z; each padded plane tile (136 x (BY RY + 2R))
//     arrives by one TMA load into a ring of NSLOT shared-memory slots (one mbarrier each).
//   * A thread owns 4 consecutive x cells (one float4) in RY rows.  The z-columns of its cells
//     (planes z-R .. z+ZB+R-1) live in a register queue.  The queue is never shifted: the
//     z-loop is unrolled over the queue's period and each unrolled iteration addresses the
//     queue with a compile-time rotation, so advancing by ZB planes costs no moves.
//   * The centre row of a cell comes from the queue; shared memory supplies only the 2R y
//     rows around the thread's RY rows (shared by those rows) and two 16-byte x-neighbour
//     loads per row (x-4 .. x-1 and x+4 .. x+7 cover any R <= 4).  Pairs of cells use Blackwell's packed FP32x2 FMA/ADD.
//   * Stores are one 16-byte vector per row.  Periodic images (Eq. 2) cost one predicated
//     vector store on the two x-face lanes (XVEC: nx a multiple of 4, the 4th element lands in
//     the row padding) or per-cell scalar stores otherwise; y- and z-images are behind one
//     test that is uniform per warp row and per plane.  Tiles that overhang the interior
//     store element-wise through an out-of-line path.
//   * Consecutive steps are launched with programmatic dependent launch: a step's CTAs set up
//     their barriers while the previous step drains, then wait for it before the first load.
//   * Waits are bounded (globaltimer); on expiry the CTA records ERR_TIMEOUT, drains its
//     in-flight TMA loads (again bounded) and returns.
// The multiply-add order per cell is the same as the FP64 kernel's (x, y, z pairs of offset
// 1, then 2, ..., then R), so results do not depend on the variant.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace stn {
namespace {

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

struct Coef32 {
    float g0;
    float ga[3][4];  // [axis][a-1]
};

template <int BY, int RY, int ZB, int NSLOT, int R>
struct H32 {
    static constexpr int TX = 128, HX = 4, TXP = TX + 2 * HX;
    static constexpr int TY = BY * RY, ROWS = TY + 2 * R;
    static constexpr int SLOT = ((TXP * ROWS * 4 + 127) / 128) * 128 / 4;  // floats, 128 B aligned
    static constexpr uint32_t BOX_BYTES = TXP * ROWS * 4;
    static constexpr size_t SMEM = (size_t)NSLOT * SLOT * 4 + 128;
    static constexpr int S = ZB + 2 * R;        // queue length (planes)
    static constexpr int U = S / gcd_c(S, ZB);  // iterations per queue period
    static_assert(R >= 1 && R <= HX, "radius 1..4: the x window holds 4 neighbours per side");
    static_assert(NSLOT >= ZB + R + 1, "ring: ZB + R planes in use plus one refill");
    static_assert((NSLOT & (NSLOT - 1)) == 0, "ring depth is a power of two (slot = j & (NSLOT-1))");
    static_assert(ROWS <= 256, "TMA box extents are limited to 256");
    static_assert(U <= 5, "the z-loop is unrolled over one queue period");
};

// Calls f(rotation, m + k ZB) for k = 0 .. U-1: one queue period of iterations, each with its
// compile-time rotation (k ZB) mod S.
template <int ZB, int S, typename F, int... K>
__device__ __forceinline__ void queue_period(F &f, int m, std::integer_sequence<int, K...>) {
    (f(std::integral_constant<int, (K * ZB) % S>{}, m + K * ZB), ...);
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void stg4(float *p, const float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// Element-wise store of a (possibly overhanging) group of 4 cells with all periodic images.
__device__ __noinline__ void store4_bounded(float *out, const Geom &g, int r, int images, int x, int y, int z,
                                           float4 v) {
    const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (x + u < g.n[0] && y < g.n[1]) store_with_images(out, g, r, images != 0, x + u, y, z, e[u]);
}

// One xy-tile of one z-chunk.  `map` may point at a __grid_constant__ parameter or at a
// descriptor in global memory (batched launches).  Returns false if a bounded wait expired.
template <int BY, int RY, int ZB, int NSLOT, int R, bool XVEC, bool PDL>
__device__ __forceinline__ bool heat32_tile(const CUtensorMap *map, float *__restrict__ out, const Geom &g,
                                            const Coef32 &c, int tile_x, int tile_y, int tile_z, int zc, int images,
                                            unsigned *err, float *ring, uint64_t *full) {
    using Cfg = H32<BY, RY, ZB, NSLOT, R>;
    constexpr int TXP = Cfg::TXP, S = Cfg::S;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int x0 = tile_x * Cfg::TX, y0 = tile_y * Cfg::TY, zc0 = tile_z * zc;
    const int nx = (int)g.n[0], ny = (int)g.n[1], nz = (int)g.n[2];
    const int count = min(nz, zc0 + zc) - zc0;
    const int nplanes = count + 2 * R;  // planes zc0-R .. zc0+count+R-1
    const int x = x0 + 4 * lane, yb = y0 + wy * RY;

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
    const int bx = (int)g.off[0] + x0 - Cfg::HX, by0 = (int)g.off[1] + y0 - R, bz0 = (int)g.off[2] + zc0 - R;
    int issued = 0;
    auto issue = [&](int j) {  // plane j (0-based from zc0-R) into its ring slot
        const int s = j & (NSLOT - 1);
        mbar_arrive_expect_tx(&full[s], Cfg::BOX_BYTES);
        tma_load_3d(ring + s * Cfg::SLOT, map, &full[s], bx, by0, bz0 + j);
    };
    auto slot = [&](int j) { return ring + (j & (NSLOT - 1)) * Cfg::SLOT; };
    auto parity = [](int j) { return ((unsigned)j / (unsigned)NSLOT) & 1u; };
    if (threadIdx.x == 0)
        for (; issued < NSLOT && issued < nplanes; ++issued) issue(issued);

    // float offset of (row 0 of this thread, first cell) inside a slot
    const int own = (wy * RY + R) * TXP + Cfg::HX + 4 * lane;
    const float2 G0 = make_float2(c.g0, c.g0);
    float2 GA[3][R];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) GA[a][b] = make_float2(c.ga[a][b], c.ga[a][b]);

    // z queue: logical entry k of an iteration with rotation ROT is Q[(ROT + k) % S]; entry k
    // holds plane (first output plane of the iteration) - R + k.
    float4 Q[S][RY];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {  // prologue: planes zc0-R .. zc0+R-1
        ok = ok && mbar_wait_bounded(&full[j & (NSLOT - 1)], parity(j));
        const float *sp = slot(j) + own;
#pragma unroll
        for (int r = 0; r < RY; ++r) Q[j][r] = ok ? lds4(sp + r * TXP) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    bool bad = __syncthreads_or(!ok);
    // planes 0..R-1 are never read from shared memory again: refill their slots
    if (!bad && threadIdx.x == 0)
        for (; issued < NSLOT + R && issued < nplanes; ++issued) issue(issued);

    // Store targets.  x-images: lanes whose cells lie within 4 (XVEC) or R of an x face.
    const bool full_tile = x + 4 <= nx && yb + RY <= ny;
    int xs = 0, xmask = 0;
    int ys[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) ys[r] = 0;
    if (images) {
        if (XVEC) {
            xs = x < 4 ? nx : (x >= nx - 4 ? -nx : 0);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (x + u < R) { xmask |= 1 << u; xs = nx; }
                else if (x + u >= nx - R && x + u < nx) { xmask |= 1 << u; xs = -nx; }
            }
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) ys[r] = (yb + r < R) ? ny : (yb + r >= ny - R ? -ny : 0);
    }
    const bool xi = XVEC ? xs != 0 : xmask != 0;
    const int pitch_y = (int)g.pad[0];
    const int64_t pitch_z = g.pad[0] * g.pad[1];
    float *optr = out + g.idx(x, yb, zc0);
    auto put = [&](float *p, const float4 v) {  // one row of 4 cells and its x-image
        stg4(p, v);
        if (XVEC) {
            if (xi) stg4(p + xs, v);
        } else if (xi) {
            if (xmask & 1) p[xs] = v.x;
            if (xmask & 2) p[1 + xs] = v.y;
            if (xmask & 4) p[2 + xs] = v.z;
            if (xmask & 8) p[3 + xs] = v.w;
        }
    };

    auto iter = [&](auto rot_c, int m) {
        constexpr int ROT = decltype(rot_c)::value;
        if (bad || m >= count) return;
        // leading planes j = m+2R .. m+2R+ZB-1 enter the queue at logical entries 2R .. 2R+ZB-1
#pragma unroll
        for (int b = 0; b < ZB; ++b) {
            const int jl = m + 2 * R + b;
            if (jl < nplanes) {
                ok = ok && mbar_wait_bounded(&full[jl & (NSLOT - 1)], parity(jl));
                const float *lp = slot(jl) + own;
#pragma unroll
                for (int r = 0; r < RY; ++r) Q[(ROT + 2 * R + b) % S][r] = lds4(lp + r * TXP);
            }
        }
        if (ok) {
#pragma unroll
            for (int b = 0; b < ZB; ++b) {
                if (m + b < count) {
                    const float *cp = slot(m + b + R) + own;
                    float4 Yn[R], Yp[R];  // rows -1 .. -R and RY .. RY+R-1
#pragma unroll
                    for (int a = 0; a < R; ++a) {
                        Yn[a] = lds4(cp - (a + 1) * TXP);
                        Yp[a] = lds4(cp + (RY + a) * TXP);
                    }
                    auto row = [&](int d) -> float4 {  // row d of the centre plane
                        return d < 0 ? Yn[-d - 1] : (d >= RY ? Yp[d - RY] : Q[(ROT + b + R) % S][d]);
                    };
                    float4 res[RY];
#pragma unroll
                    for (int r = 0; r < RY; ++r) {
                        const float4 C = Q[(ROT + b + R) % S][r];
                        const float4 Lv = lds4(cp + r * TXP - 4), Rv = lds4(cp + r * TXP + 4);
                        // x window E[k] = cell x-4+k, k = 0..11
                        const float E[12] = {Lv.x, Lv.y, Lv.z, Lv.w, C.x, C.y, C.z, C.w, Rv.x, Rv.y, Rv.z, Rv.w};
                        float2 sx[2][R], sy[2][R], sz[2][R];
#pragma unroll
                        for (int p = 0; p < 2; ++p)
#pragma unroll
                            for (int a = 1; a <= R; ++a) {
                                const int c0 = 4 + 2 * p;  // E index of the pair's first cell
                                if (a % 2 == 0)  // even offsets: aligned pairs, one packed add
                                    sx[p][a - 1] = __fadd2_rn(make_float2(E[c0 + a], E[c0 + 1 + a]),
                                                              make_float2(E[c0 - a], E[c0 + 1 - a]));
                                else  // odd offsets: two scalar adds
                                    sx[p][a - 1] = make_float2(E[c0 + a] + E[c0 - a], E[c0 + 1 + a] + E[c0 + 1 - a]);
                            }
#pragma unroll
                        for (int a = 1; a <= R; ++a) {
                            const float4 yp = row(r + a), ym = row(r - a);
                            const float4 zp = Q[(ROT + b + R + a) % S][r], zm = Q[(ROT + b + R - a) % S][r];
                            sy[0][a - 1] = __fadd2_rn(make_float2(yp.x, yp.y), make_float2(ym.x, ym.y));
                            sy[1][a - 1] = __fadd2_rn(make_float2(yp.z, yp.w), make_float2(ym.z, ym.w));
                            sz[0][a - 1] = __fadd2_rn(make_float2(zp.x, zp.y), make_float2(zm.x, zm.y));
                            sz[1][a - 1] = __fadd2_rn(make_float2(zp.z, zp.w), make_float2(zm.z, zm.w));
                        }
                        float2 o[2];
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            float2 acc = __fmul2_rn(G0, p ? make_float2(C.z, C.w) : make_float2(C.x, C.y));
#pragma unroll
                            for (int a = 0; a < R; ++a) {
                                acc = __ffma2_rn(GA[0][a], sx[p][a], acc);
                                acc = __ffma2_rn(GA[1][a], sy[p][a], acc);
                                acc = __ffma2_rn(GA[2][a], sz[p][a], acc);
                            }
                            o[p] = acc;
                        }
                        res[r] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                    }
                    const int z = zc0 + m + b;
                    const int zs = images ? (z < R ? nz : (z >= nz - R ? -nz : 0)) : 0;
                    float *op = optr + b * pitch_z;
                    if (full_tile) {
#pragma unroll
                        for (int r = 0; r < RY; ++r) {
                            float *p = op + r * pitch_y;
                            put(p, res[r]);
                            if (ys[r] | zs) {  // y- and z-images: uniform per warp row / per plane
                                const int64_t dy = (int64_t)ys[r] * pitch_y, dz = (int64_t)zs * pitch_z;
                                if (ys[r]) put(p + dy, res[r]);
                                if (zs) put(p + dz, res[r]);
                                if (ys[r] && zs) put(p + dy + dz, res[r]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < RY; ++r) store4_bounded(out, g, R, images, x, yb + r, z, res[r]);
                    }
                }
            }
        }
        optr += ZB * pitch_z;
        bad = __syncthreads_or(!ok);
        // planes j < m + ZB + R are retired: refill the ring up to NSLOT planes ahead
        if (!bad && threadIdx.x == 0) {
            const int lim = min(nplanes, m + ZB + R + NSLOT);
            for (; issued < lim; ++issued) issue(issued);
        }
    };
    for (int m = 0; !bad && m < count; m += Cfg::U * ZB)
        queue_period<ZB, S>(iter, m, std::make_integer_sequence<int, Cfg::U>{});
    if (bad && threadIdx.x == 0) {
        atomicOr(err, ERR_TIMEOUT);
        // drain loads still in flight before the CTA's shared memory is released
        for (int j = max(0, issued - NSLOT); j < issued; ++j)
            (void)mbar_wait_bounded(&full[j & (NSLOT - 1)], parity(j), 100000000ull);
    }
    return !bad;
}

template <int BY, int RY, int ZB, int NSLOT, int R, int MINB, bool XVEC>
__global__ void __launch_bounds__(32 * BY, MINB)
heat32_kernel(const __grid_constant__ CUtensorMap map_in, float *__restrict__ out, Geom g, Coef32 c, int zc,
              int images, unsigned *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full[NSLOT];
    heat32_tile<BY, RY, ZB, NSLOT, R, XVEC, true>(&map_in, out, g, c, blockIdx.x, blockIdx.y, blockIdx.z, zc,
                                                  images, err, ring, full);
}

// Persistent schedule: all nsteps steps in one cooperative launch, units published per step
// and face-neighbour waits instead of kernel boundaries (persist.cuh).  Step s reads the
// field written by step s-1 (the input for s = 0) and writes `out` when nsteps - 1 - s is
// even, `tmp` otherwise, so the last step writes `out` and the input is only read.
template <int BY, int RY, int ZB, int NSLOT, int R, int MINB, bool XVEC>
__global__ void __launch_bounds__(32 * BY, MINB)
heat32_persist_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_tmp,
                      const __grid_constant__ CUtensorMap map_out, float *tmp, float *out, Geom g, Coef32 c,
                      PersistGrid pg, int nsteps, int images, unsigned long long *sync, unsigned *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full[NSLOT];
    __shared__ unsigned long long s_base;
    if (threadIdx.x == 0) s_base = ld_relaxed_u64(sync);  // written by the previous launch
    __syncthreads();
    const unsigned long long base = s_base;
    const int W = pg.units();
    bool ok = true;
    for (int s = 0; ok && s < nsteps; ++s) {
        const bool to_out = ((nsteps - 1 - s) & 1) == 0;
        float *dst = to_out ? out : tmp;
        const CUtensorMap *src = s == 0 ? &map_in : (to_out ? &map_tmp : &map_out);
        for (int u = blockIdx.x; ok && u < W; u += gridDim.x) {
            const int t0 = u % pg.nt[0], t1 = (u / pg.nt[0]) % pg.nt[1], t2 = u / (pg.nt[0] * pg.nt[1]);
            if (s > 0) ok = wait_face_neighbours<R>(sync, pg, g, t0, t1, t2, base + s, base + 1);
            if (ok) {
                if (threadIdx.x == 0) fence_proxy_async_global();  // acquired stores -> this CTA's TMA loads
                ok = heat32_tile<BY, RY, ZB, NSLOT, R, XVEC, false>(src, dst, g, c, t0, t1, t2, pg.tl[2], images, err,
                                                                     ring, full);
            }
            fence_proxy_async_global();  // this thread's stores -> TMA loads of the next step
            __syncthreads();
            if (ok && threadIdx.x == 0) {
                publish_unit(sync, u, base + s + 1);
                for (int k = 0; k < NSLOT; ++k) mbar_inval(&full[k]);  // initialised again by the next unit
            }
        }
    }
    if (threadIdx.x == 0) {
        if (!ok) atomicOr(err, ERR_TIMEOUT);
        persist_exit(sync, base, nsteps, !ok);
    }
}

// Vector x-images need nx a multiple of 4 and one spare padding element beyond each x halo.
__host__ __device__ bool xvec_ok(const Geom &g) {
    return g.n[0] % 4 == 0 && g.n[0] >= 8 && g.off[0] >= 4 && g.pad[0] >= g.off[0] + g.n[0] + 4;
}

Coef32 coef32(const DiffCoef &dc) {
    Coef32 c;
    c.g0 = (float)dc.g0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 4; ++b) c.ga[a][b] = (float)dc.ga[a][b];
    return c;
}

// Resident CTAs per SM of kernel k (cached per device), after raising its shared-memory limit.
template <typename K> cudaError_t occupancy(K k, int threads, size_t smem, int cache[64], int *occ) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!cache[dev]) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, threads, smem);
        if (e != cudaSuccess) return e;
        cache[dev] = std::max(o, 1);
    }
    *occ = cache[dev];
    return cudaSuccess;
}

// Unit decomposition shared by both schedules: 128 x TY tiles of the xy-plane, z split into
// chunks so that the units fill the resident CTA slots (choose_zchunks), then zmode.
template <int BY, int RY, int ZB, int NSLOT, int R>
PersistGrid units_of(const Geom &g, int slots, int zmode) {
    using Cfg = H32<BY, RY, ZB, NSLOT, R>;
    const int tx = (int)((g.n[0] + Cfg::TX - 1) / Cfg::TX), ty = (int)((g.n[1] + Cfg::TY - 1) / Cfg::TY);
    const int nz = (int)g.n[2];
    const int chunks = choose_zchunks(tx * ty, nz, slots, 0.5);
    const int zc = zchunk_len((nz + chunks - 1) / chunks, nz, zmode);
    return PersistGrid{{tx, ty, (nz + zc - 1) / zc}, {Cfg::TX, Cfg::TY, zc}};
}

template <int BY, int RY, int ZB, int NSLOT, int R, int MINB, bool XVEC>
cudaError_t run(const CUtensorMap *map, float *out, const Geom &g, const Coef32 &c, bool images, unsigned *err,
                cudaStream_t s, int zmode) {
    using Cfg = H32<BY, RY, ZB, NSLOT, R>;
    auto k = heat32_kernel<BY, RY, ZB, NSLOT, R, MINB, XVEC>;
    static int occ_cache[64] = {};
    int occ = 0;
    cudaError_t e = occupancy(k, 32 * BY, Cfg::SMEM, occ_cache, &occ);
    if (e != cudaSuccess) return e;
    const PersistGrid pg = units_of<BY, RY, ZB, NSLOT, R>(g, occ * device_sms(), zmode);
    dim3 grid(pg.nt[0], pg.nt[1], pg.nt[2]);
    return launch_pdl(k, grid, dim3(32 * BY), Cfg::SMEM, s, *map, out, g, c, pg.tl[2], images ? 1 : 0, err);
}

// Persistent schedule.  With sync == nullptr only reports the number of units (the sync
// buffer needs PERSIST_HDR + units words).
template <int BY, int RY, int ZB, int NSLOT, int R, int MINB, bool XVEC>
cudaError_t run_persist(const CUtensorMap *maps, float *tmp, float *out, const Geom &g, const Coef32 &c, bool images,
                        int nsteps, unsigned long long *sync, int64_t sync_words, unsigned *err, cudaStream_t s,
                        int zmode, int64_t *units) {
    using Cfg = H32<BY, RY, ZB, NSLOT, R>;
    auto k = heat32_persist_kernel<BY, RY, ZB, NSLOT, R, MINB, XVEC>;
    static int occ_cache[64] = {};
    int occ = 0;
    cudaError_t e = occupancy(k, 32 * BY, Cfg::SMEM, occ_cache, &occ);
    if (e != cudaSuccess) return e;
    const PersistGrid pg = units_of<BY, RY, ZB, NSLOT, R>(g, occ * device_sms(), zmode);
    const int W = pg.units();
    if (units) *units = W;
    if (!sync) return cudaSuccess;
    if (PERSIST_HDR + (int64_t)W > sync_words) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min(W, occ * device_sms()));
    cfg.blockDim = dim3(32 * BY);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the neighbour waits rely on it
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, maps[0], maps[1], maps[2], tmp, out, g, c, pg, nsteps, images ? 1 : 0, sync,
                              err);
}

// Variant tables: (BY warps, RY rows, ZB planes per iteration, NSLOT ring depth, MINB resident
// CTAs the register budget is sized for).  The autotuner times each on the problem.  Radius 3
// (the 6th-order step) carries the tuned set; the other radii of the sweep use its first shape.
#define HEAT32_VARIANTS_R3(X) \
    X(4, 2, 2, 8, 3)          \
    X(4, 1, 2, 8, 4)          \
    X(8, 1, 2, 8, 2)          \
    X(4, 1, 2, 8, 3)          \
    X(8, 2, 2, 8, 2)
#define HEAT32_VARIANTS_OTHER(X) X(4, 2, 2, 8, 3)

// Each tile shape comes in both schedules: variants 0 .. n-1 launch once per step (PDL),
// variants n .. 2n-1 run all steps of a call in one persistent launch (suffix "_persist").
constexpr int N_R3 = 5, N_OTHER = 1;
const char *const NAMES_R3[] = {"f32_by4_ry2_zb2_s8_m3",         "f32_by4_ry1_zb2_s8_m4",
                                "f32_by8_ry1_zb2_s8_m2",         "f32_by4_ry1_zb2_s8_m3",
                                "f32_by8_ry2_zb2_s8_m2",         "f32_by4_ry2_zb2_s8_m3_persist",
                                "f32_by4_ry1_zb2_s8_m4_persist", "f32_by8_ry1_zb2_s8_m2_persist",
                                "f32_by4_ry1_zb2_s8_m3_persist", "f32_by8_ry2_zb2_s8_m2_persist"};
const char *const NAMES_OTHER[][2] = {{"?", "?"},
                                      {"f32_r1_by4_ry2_zb2_s8_m3", "f32_r1_by4_ry2_zb2_s8_m3_persist"},
                                      {"f32_r2_by4_ry2_zb2_s8_m3", "f32_r2_by4_ry2_zb2_s8_m3_persist"},
                                      {"?", "?"},
                                      {"f32_r4_by4_ry2_zb2_s8_m3", "f32_r4_by4_ry2_zb2_s8_m3_persist"}};

constexpr int n_shapes(int r) { return r == 3 ? N_R3 : N_OTHER; }

template <int R>
cudaError_t dispatch(int variant, const CUtensorMap *map, float *out, const Geom &g, const Coef32 &c, bool images,
                     unsigned *err, cudaStream_t s, int zmode) {
    const bool xv = xvec_ok(g);
    int i = 0;
    cudaError_t res = cudaErrorInvalidValue;
#define X(BY, RY, ZB, NS, MB)                                                          \
    if (i++ == variant)                                                                \
        res = xv ? run<BY, RY, ZB, NS, R, MB, true>(map, out, g, c, images, err, s, zmode) \
                 : run<BY, RY, ZB, NS, R, MB, false>(map, out, g, c, images, err, s, zmode);
    if constexpr (R == 3) {
        HEAT32_VARIANTS_R3(X)
    } else {
        HEAT32_VARIANTS_OTHER(X)
    }
#undef X
    return res;
}

template <int R>
cudaError_t dispatch_persist(int shape, const CUtensorMap *maps, float *tmp, float *out, const Geom &g,
                             const Coef32 &c, bool images, int nsteps, unsigned long long *sync, int64_t sync_words,
                             unsigned *err, cudaStream_t s, int zmode, int64_t *units) {
    const bool xv = xvec_ok(g);
    int i = 0;
    cudaError_t res = cudaErrorInvalidValue;
#define X(BY, RY, ZB, NS, MB)                                                                                   \
    if (i++ == shape)                                                                                           \
        res = xv ? run_persist<BY, RY, ZB, NS, R, MB, true>(maps, tmp, out, g, c, images, nsteps, sync, sync_words, \
                                                            err, s, zmode, units)                               \
                 : run_persist<BY, RY, ZB, NS, R, MB, false>(maps, tmp, out, g, c, images, nsteps, sync,         \
                                                             sync_words, err, s, zmode, units);
    if constexpr (R == 3) {
        HEAT32_VARIANTS_R3(X)
    } else {
        HEAT32_VARIANTS_OTHER(X)
    }
#undef X
    return res;
}

}  // namespace

int diffusion_f32_num_variants(int r) { return r >= 1 && r <= 4 ? 2 * n_shapes(r) : 0; }

bool diffusion_f32_persistent(int r, int v) { return v >= n_shapes(r) && v < diffusion_f32_num_variants(r); }

const char *diffusion_f32_variant_name(int r, int v) {
    if (v < 0 || v >= diffusion_f32_num_variants(r)) return "?";
    return r == 3 ? NAMES_R3[v] : NAMES_OTHER[r][v];
}

void diffusion_f32_box(int r, int v, int box[3]) {
    v %= n_shapes(r);  // both schedules of a shape load the same box
    int i = 0;
    box[0] = H32<1, 1, 2, 8, 1>::TXP;
    box[2] = 1;
#define X(BY, RY, ZB, NS, MB) \
    if (i++ == v) box[1] = BY * RY + 2 * r;
    if (r == 3) {
        HEAT32_VARIANTS_R3(X)
    } else {
        HEAT32_VARIANTS_OTHER(X)
    }
#undef X
}

cudaError_t launch_diffusion_f32_persist(const CUtensorMap *maps, float *tmp, float *out, const Geom &g,
                                         const DiffCoef &dc, bool images, int nsteps, unsigned long long *sync,
                                         int64_t sync_words, unsigned *err, cudaStream_t s, int variant, int zmode,
                                         int64_t *units) {
    if (!diffusion_f32_persistent(dc.r, variant)) return cudaErrorInvalidValue;
    const Coef32 c = coef32(dc);
    const int shape = variant - n_shapes(dc.r);
    switch (dc.r) {
    case 1: return dispatch_persist<1>(shape, maps, tmp, out, g, c, images, nsteps, sync, sync_words, err, s, zmode, units);
    case 2: return dispatch_persist<2>(shape, maps, tmp, out, g, c, images, nsteps, sync, sync_words, err, s, zmode, units);
    case 3: return dispatch_persist<3>(shape, maps, tmp, out, g, c, images, nsteps, sync, sync_words, err, s, zmode, units);
    case 4: return dispatch_persist<4>(shape, maps, tmp, out, g, c, images, nsteps, sync, sync_words, err, s, zmode, units);
    default: return cudaErrorInvalidValue;
    }
}

// Persistent variants exist for FP32 storage only (dtype 2).
bool diffusion_persistent(int dtype, int r, int v) { return dtype == 2 && diffusion_f32_persistent(r, v); }

cudaError_t launch_diffusion_persist(int dtype, const CUtensorMap *maps, void *tmp, void *out, const Geom &g,
                                     const DiffCoef &c, bool images, int nsteps, unsigned long long *sync,
                                     int64_t sync_words, unsigned *err, cudaStream_t s, int variant, int zmode,
                                     int64_t *units) {
    if (dtype != 2) return cudaErrorInvalidValue;
    return launch_diffusion_f32_persist(maps, static_cast<float *>(tmp), static_cast<float *>(out), g, c, images,
                                        nsteps, sync, sync_words, err, s, variant, zmode, units);
}

cudaError_t launch_diffusion_f32(const CUtensorMap *map, float *out, const Geom &g, const DiffCoef &dc, bool images,
                                 unsigned *err, cudaStream_t s, int variant, int zmode) {
    if (diffusion_f32_persistent(dc.r, variant)) return cudaErrorInvalidValue;  // one launch per call
    const Coef32 c = coef32(dc);
    switch (dc.r) {
    case 1: return dispatch<1>(variant, map, out, g, c, images, err, s, zmode);
    case 2: return dispatch<2>(variant, map, out, g, c, images, err, s, zmode);
    case 3: return dispatch<3>(variant, map, out, g, c, images, err, s, zmode);
    case 4: return dispatch<4>(variant, map, out, g, c, images, err, s, zmode);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ batched (serving)

// Tile shapes of the batched kernel (the server picks one per run from the autotuner's choice
// for FP32 heat plans): 0 = 128 x 8 cells (4 warps x 2 rows, the tile of the per-grid variants
// f32_by4_ry2_*), 1 = 128 x 16 (8 warps x 2 rows, f32_by8_ry2_*).
namespace {
template <int SH> struct DbShape;
template <> struct DbShape<0> { static constexpr int BY = 4, RY = 2, MINB = 2; };
template <> struct DbShape<1> { static constexpr int BY = 8, RY = 2, MINB = 2; };
constexpr int DB_ZB = 2, DB_NSLOT = 8;
template <int SH> using DbCfg = H32<DbShape<SH>::BY, DbShape<SH>::RY, DB_ZB, DB_NSLOT, R6>;
}  // namespace

template <int SH>
__global__ void __launch_bounds__(32 * DbShape<SH>::BY, DbShape<SH>::MINB)
diffusion_batch_kernel(const BatchHeader *hdr, const BatchHeat *items, unsigned *err) {
    constexpr int BY = DbShape<SH>::BY, RY = DbShape<SH>::RY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full[DB_NSLOT];
    const int total = hdr->heat_ctas, n = hdr->n_heat;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].cta_begin <= vb) lo = mid; else hi = mid - 1;
        }
        const BatchHeat &it = items[lo];
        int r = vb - it.cta_begin;
        const int tx = r % it.tiles_x;
        r /= it.tiles_x;
        const int ty = r % it.tiles_y, tz = r / it.tiles_y;
        Coef32 c;
        c.g0 = it.g0;
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) c.ga[a][b] = it.ga[a][b];
            c.ga[a][3] = 0.f;
        }
        const Geom g = it.g;
        const bool ok = xvec_ok(g)
                            ? heat32_tile<BY, RY, DB_ZB, DB_NSLOT, R6, true, false>(it.map, it.out, g, c, tx, ty, tz, it.zc,
                                                                                 1, err, ring, full)
                            : heat32_tile<BY, RY, DB_ZB, DB_NSLOT, R6, false, false>(it.map, it.out, g, c, tx, ty, tz,
                                                                                  it.zc, 1, err, ring, full);
        __syncthreads();
        if (!ok) return;
    }
}

template <int SH> static int batch_grid_t() {
    static int grid[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 152;
    if (!grid[dev]) {
        cudaFuncSetAttribute(diffusion_batch_kernel<SH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)DbCfg<SH>::SMEM);
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, diffusion_batch_kernel<SH>, 32 * DbShape<SH>::BY,
                                                      DbCfg<SH>::SMEM);
        grid[dev] = std::max(o, 1) * device_sms();
    }
    return grid[dev];
}

int diffusion_batch_grid(int shape) { return shape == 1 ? batch_grid_t<1>() : batch_grid_t<0>(); }

const char *diffusion_batch_shape_name(int shape) {
    return shape == 1 ? "batch_by8_ry2_zb2_s8" : "batch_by4_ry2_zb2_s8";
}

void diffusion_batch_tile(int shape, int *tx, int *ty, int box[3]) {
    *tx = shape == 1 ? DbCfg<1>::TX : DbCfg<0>::TX;
    *ty = shape == 1 ? DbCfg<1>::TY : DbCfg<0>::TY;
    box[0] = shape == 1 ? DbCfg<1>::TXP : DbCfg<0>::TXP;
    box[1] = shape == 1 ? DbCfg<1>::ROWS : DbCfg<0>::ROWS;
    box[2] = 1;
}

cudaError_t launch_diffusion_batch(int shape, const BatchHeader *hdr, const BatchHeat *items, unsigned *err, int grid,
                                   cudaStream_t s) {
    if (shape == 1)
        diffusion_batch_kernel<1><<<grid, 32 * DbShape<1>::BY, DbCfg<1>::SMEM, s>>>(hdr, items, err);
    else
        diffusion_batch_kernel<0><<<grid, 32 * DbShape<0>::BY, DbCfg<0>::SMEM, s>>>(hdr, items, err);
    return cudaGetLastError();
}

}  // namespace stn
