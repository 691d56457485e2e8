// mhd_pairs.cu -- the fused 8-field MHD step (Eqs. 8-9, A1-A4, RK3; Sec. 3.3) for FP32
// arithmetic (FP32 or BF16 storage), with the derivative stencils evaluated on pairs of fields
// by Blackwell's packed FP32x2 instructions.
//
// The scalar kernel (mhd.cu) is bound by issue slots: one thread per cell, ~380 scalar shared
// loads and ~450 derivative FP instructions per cell, at only 8 warps per SM (the 7-plane
// window of 8 fields fills shared memory).  Here, as each plane arrives (one TMA load per
// field into a small raw ring), the CTA re-lays it once as four float2 tiles of field pairs
// (lnrho, s), (ux, uy), (uz, Ax), (Ay, Az) in a ring of 8 pair planes (BF16 values are widened
// to FP32 once here, not at every use).  Every stencil point of a pair is then one 8-byte
// shared load and every weight one packed FMA, so the derivative phase needs half the loads
// and half the arithmetic instructions.  Each lane performs the same IEEE operations in the
// same order as the scalar kernel (a - b is formed as fma(b, -1, a), which rounds once to
// a - b), so results are identical to it; the pointwise right-hand side (mhd_rhs.cuh) and the
// Kahan-compensated 2N-storage RK update are shared with it.
//
// Pipeline per plane: wait for the raw plane, convert it into the pair ring (the plane being
// converted is never in the current 7-plane window), one barrier, refill the raw slot, compute
// one cell per thread.  Waits are bounded; on expiry ERR_TIMEOUT is recorded and in-flight
// loads are drained before the CTA returns.
//
// TMA-I/O variant: the RK register w and the Kahan term c of the next plane arrive by 16 TMA
// box loads into double-buffered shared staging; each thread updates its w and c in place and
// writes its new field values to a staging tile; after a proxy fence and a barrier one thread
// stores the plane's 24 boxes (fields through an interior view of each output array, so tiles
// that overhang the interior are clipped) with TMA.  This replaces 40 scalar global accesses per
// cell, whose issue queue and latency bound the plain variants at 8 warps per SM.  Periodic
// images of edge cells are still written by scalar stores.
#include <algorithm>

#include "mhd_rhs.cuh"

namespace stn {
namespace {

template <typename S, int TY, int NR, bool TMAIO = false>
struct MpCfg {
    static constexpr int TX = 32;
    static constexpr int HX = 16 / (int)sizeof(S) >= 4 ? 16 / (int)sizeof(S) : 4;  // raw tile x halo (TMA)
    static constexpr int TXP = TX + 2 * HX;                                          // raw row pitch
    static constexpr int PX = TX + 8;                                                // pair row pitch (halo 4)
    static constexpr int ROWS = TY + 2 * R6;
    static constexpr int RAW_FIELD = ((TXP * ROWS * (int)sizeof(S) + 127) / 128) * 128 / (int)sizeof(S);
    static constexpr int RAW_SLOT = 8 * RAW_FIELD;
    static constexpr int PAIR_FIELD = ((PX * ROWS * 8 + 127) / 128) * 128 / 8;  // float2 elements
    static constexpr int PAIR_SLOT = 4 * PAIR_FIELD;
    static constexpr uint32_t BOX_BYTES = TXP * ROWS * sizeof(S);
    static constexpr size_t RAW_BYTES = (size_t)NR * RAW_SLOT * sizeof(S);
    static constexpr size_t PAIR_BYTES = (size_t)8 * PAIR_SLOT * 8;
    // TMA-I/O staging per buffer: 16 boxes of w and c, then 8 boxes of new field values
    static constexpr int CELLS = TX * TY;
    static constexpr size_t STAGE_BYTES = TMAIO ? (size_t)24 * CELLS * sizeof(S) : 0;
    static constexpr size_t SMEM = RAW_BYTES + PAIR_BYTES + 2 * STAGE_BYTES + 128;
    static_assert((CELLS * sizeof(S)) % 128 == 0, "staging boxes stay 128-byte aligned");
    static_assert((TXP * sizeof(S)) % 16 == 0, "TMA box inner extent must be a multiple of 16 B");
    static_assert((NR & (NR - 1)) == 0 && NR >= 2, "raw ring depth is a power of two >= 2");
    static_assert(RAW_BYTES % 128 == 0, "pair ring stays 128-byte aligned");
};

// Field pairs: pair p holds fields (PF[p][0], PF[p][1]).
__device__ constexpr int PF[4][2] = {{F_LNRHO, F_SS}, {F_UX, F_UY}, {F_UZ, F_AX}, {F_AY, F_AZ}};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// The 7-plane window of the four pair tiles around one cell: p[k] points at the cell (pair 0)
// in plane z + k - 3.
template <int PFE, int PX>
struct PWin {
    const float2 *p[7];
    __device__ __forceinline__ float2 at(int q, int k, int dx, int dy) const { return p[k][q * PFE + dy * PX + dx]; }
};

// 6th-order stencils on a pair, the operations of the scalar d1/d2/dmix lane by lane.
template <typename W>
__device__ __forceinline__ float2 d1p(const W &w, int q, int axis, const float *c) {
    auto f = [&](int s) { return axis == 0 ? w.at(q, 3, s, 0) : axis == 1 ? w.at(q, 3, 0, s) : w.at(q, 3 + s, 0, 0); };
    float2 a = __fmul2_rn(f2(c[0]), sub2(f(1), f(-1)));
    a = __ffma2_rn(f2(c[1]), sub2(f(2), f(-2)), a);
    return __ffma2_rn(f2(c[2]), sub2(f(3), f(-3)), a);
}
template <typename W>
__device__ __forceinline__ float2 d2p(const W &w, int q, int axis, float c0, const float *c) {
    auto f = [&](int s) { return axis == 0 ? w.at(q, 3, s, 0) : axis == 1 ? w.at(q, 3, 0, s) : w.at(q, 3 + s, 0, 0); };
    float2 a = __fmul2_rn(f2(c0), f(0));
    a = __ffma2_rn(f2(c[0]), __fadd2_rn(f(1), f(-1)), a);
    a = __ffma2_rn(f2(c[1]), __fadd2_rn(f(2), f(-2)), a);
    return __ffma2_rn(f2(c[2]), __fadd2_rn(f(3), f(-3)), a);
}
template <typename W>
__device__ __forceinline__ float2 dmixp(const W &w, int q, int pair, const float *m) {
    auto f = [&](int s1, int s2) {
        return pair == 0 ? w.at(q, 3, s1, s2) : pair == 1 ? w.at(q, 3 + s2, s1, 0) : w.at(q, 3 + s2, 0, s1);
    };
    auto D = [&](int a) { return sub2(__fadd2_rn(f(a, a), f(-a, -a)), __fadd2_rn(f(a, -a), f(-a, a))); };
    float2 acc = __fmul2_rn(f2(m[0]), D(1));
    acc = __ffma2_rn(f2(m[1]), D(2), acc);
    return __ffma2_rn(f2(m[2]), D(3), acc);
}

// Hessian of a pair: h[0..2] = xx, yy, zz; h[3..5] = xy, xz, yz.
template <typename W>
__device__ __forceinline__ void hessp(const W &w, int q, const MK<float> &k, float2 *h) {
    h[0] = d2p(w, q, 0, k.d2c[0], k.d2[0]);
    h[1] = d2p(w, q, 1, k.d2c[1], k.d2[1]);
    h[2] = d2p(w, q, 2, k.d2c[2], k.d2[2]);
    h[3] = dmixp(w, q, 0, k.dm[0]);
    h[4] = dmixp(w, q, 1, k.dm[1]);
    h[5] = dmixp(w, q, 2, k.dm[2]);
}

// The right-hand side at one cell from the pair window (the same derivative quantities, in
// the same order, as the scalar kernel's mhd_rhs_cell).
template <typename W>
__device__ __forceinline__ void mhdp_rhs_cell(const W &w, const MK<float> &k, float *rhs, float *val) {
    MhdDerivs<float> d;
    const float2 v0 = w.at(0, 3, 0, 0), v1 = w.at(1, 3, 0, 0), v2 = w.at(2, 3, 0, 0), v3 = w.at(3, 3, 0, 0);
    d.val[F_LNRHO] = v0.x; d.val[F_SS] = v0.y;
    d.val[F_UX] = v1.x; d.val[F_UY] = v1.y;
    d.val[F_UZ] = v2.x; d.val[F_AX] = v2.y;
    d.val[F_AY] = v3.x; d.val[F_AZ] = v3.y;
    // (lnrho, s): gradients, and Laplacians when K != 0
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float2 g = d1p(w, 0, a, k.d1[a]);
        d.glr[a] = g.x;
        d.gs[a] = g.y;
    }
    d.laplr = d.laps = 0.f;
    if (k.K != 0.f) {
        float2 l = d2p(w, 0, 0, k.d2c[0], k.d2[0]);
        l = __fadd2_rn(l, d2p(w, 0, 1, k.d2c[1], k.d2[1]));
        l = __fadd2_rn(l, d2p(w, 0, 2, k.d2c[2], k.d2[2]));
        d.laplr = l.x;
        d.laps = l.y;
    }
    float2 g1[3], g2[3], g3[3], h1[6], h2[6], h3[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g1[a] = d1p(w, 1, a, k.d1[a]);  // (ux, uy)
        g2[a] = d1p(w, 2, a, k.d1[a]);  // (uz, Ax)
        g3[a] = d1p(w, 3, a, k.d1[a]);  // (Ay, Az)
    }
    hessp(w, 1, k, h1);
    hessp(w, 2, k, h2);
    hessp(w, 3, k, h3);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d.gu[0][a] = g1[a].x;
        d.gu[1][a] = g1[a].y;
        d.gu[2][a] = g2[a].x;
    }
    // lap u and grad div u (sums in the scalar kernel's order: components ux, uy, uz)
    d.lapu[0] = h1[0].x + h1[1].x + h1[2].x;
    d.lapu[1] = h1[0].y + h1[1].y + h1[2].y;
    d.lapu[2] = h2[0].x + h2[1].x + h2[2].x;
    d.gdivu[0] = (h1[0].x + h1[3].y) + h2[4].x;  // d_x d_x ux + d_x d_y uy + d_x d_z uz
    d.gdivu[1] = (h1[3].x + h1[1].y) + h2[5].x;  // d_y d_x ux + d_y d_y uy + d_y d_z uz
    d.gdivu[2] = (h1[4].x + h1[5].y) + h2[2].x;  // d_z d_x ux + d_z d_y uy + d_z d_z uz
    // B = curl A from the off-diagonal first derivatives
    const float ax_y = g2[1].y, ax_z = g2[2].y, ay_x = g3[0].x, ay_z = g3[2].x, az_x = g3[0].y, az_y = g3[1].y;
    d.bx = az_y - ay_z;
    d.by = ax_z - az_x;
    d.bz = ay_x - ax_y;
    d.lapa[0] = h2[0].y + h2[1].y + h2[2].y;
    d.lapa[1] = h3[0].x + h3[1].x + h3[2].x;
    d.lapa[2] = h3[0].y + h3[1].y + h3[2].y;
    d.gdiva[0] = (h2[0].y + h3[3].x) + h3[4].y;
    d.gdiva[1] = (h2[3].y + h3[1].x) + h3[5].y;
    d.gdiva[2] = (h2[4].y + h3[5].x) + h3[2].y;
    mhd_rhs_assemble(d, k, rhs);
#pragma unroll
    for (int q = 0; q < 8; ++q) val[q] = d.val[q];
}

// One xy-tile of one z-chunk of one RK substep (MODE 0) or RHS evaluation (MODE 1).
template <typename S, int TY, int NR, int MODE, bool TMAIO>
__device__ __forceinline__ bool mhdp_tile(const CUtensorMap *maps, const MhdIoMaps *io, const Ptrs8 &fout,
                                          const Ptrs8 &wbuf, const Ptrs8 &kbuf, const Ptrs8 &rbuf, const Geom &g,
                                          const MK<float> &k, int tile_x, int tile_y, int tile_z, int zc, int first,
                                          int last, int images, unsigned *err, S *raw, float2 *pairs, S *stage,
                                          uint64_t *full, uint64_t *wcbar) {
    static_assert(!TMAIO || MODE == 0, "TMA I/O serves the RK substep");
    using Cfg = MpCfg<S, TY, NR, TMAIO>;
    constexpr int CELLS = Cfg::CELLS;
    using W = PWin<Cfg::PAIR_FIELD, Cfg::PX>;
    constexpr int TX = Cfg::TX;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const int zc0 = tile_z * zc;
    const int nx = (int)g.n[0], ny = (int)g.n[1], nz = (int)g.n[2];
    const int zend = min(nz, zc0 + zc);
    const int nplanes = (zend - zc0) + 2 * R6;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < nx && y < ny;

    if (threadIdx.x == 0) {
        for (int q = 0; q < 8; ++q) tma_prefetch_desc(&maps[q]);
        for (int s = 0; s < NR; ++s) mbar_init(&full[s], 1);
        if (TMAIO) {
            mbar_init(&wcbar[0], 1);
            mbar_init(&wcbar[1], 1);
        }
        mbar_fence_init();
    }
    __syncthreads();
    // TMA I/O: staging buffer b holds w_0..w_7, c_0..c_7, f'_0..f'_7 boxes of CELLS elements
    auto stg = [&](int b, int q) { return stage + (size_t)(b * 24 + q) * CELLS; };
    int wc_issued = 0;              // planes whose w/c loads thread 0 has issued
    auto load_wc = [&](int m) {  // w (unless first) and c of plane zc0 + m into buffer m & 1
        const int b = m & 1, z = zc0 + m;
        wc_issued = m + 1;
        const uint32_t boxb = (uint32_t)(CELLS * sizeof(S));
        mbar_arrive_expect_tx(&wcbar[b], (first ? 8u : 16u) * boxb);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (!first) tma_load_3d(stg(b, q), &io->w[q], &wcbar[b], x0, y0, z);
            tma_load_3d(stg(b, 8 + q), &io->c[q], &wcbar[b], x0, y0, z);
        }
    };
    if (TMAIO && threadIdx.x == 0 && zc0 < zend) load_wc(0);
    const int bx = (int)g.off[0] + x0 - Cfg::HX;
    const int by0 = (int)g.off[1] + y0 - R6;
    const int bz0 = (int)g.off[2] + zc0 - R6;
    auto issue = [&](int j) {  // plane j (0-based from zc0-3) into raw slot j mod NR
        const int s = j & (NR - 1);
        mbar_arrive_expect_tx(&full[s], 8 * Cfg::BOX_BYTES);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            tma_load_3d(raw + s * Cfg::RAW_SLOT + q * Cfg::RAW_FIELD, &maps[q], &full[s], bx, by0, bz0 + j);
    };
    int issued = 0;
    if (threadIdx.x == 0)
        for (; issued < NR && issued < nplanes; ++issued) issue(issued);

    // wait for raw plane j, convert it into pair slot j mod 8; the caller synchronises
    auto convert = [&](int j) -> bool {
        const int s = j & (NR - 1);
        if (!mbar_wait_bounded(&full[s], ((unsigned)j / NR) & 1u)) return false;
        const S *src = raw + s * Cfg::RAW_SLOT;
        float2 *dst = pairs + (j & 7) * Cfg::PAIR_SLOT;
        for (int e = threadIdx.x; e < Cfg::PX * Cfg::ROWS; e += TX * TY) {
            const int row = e / Cfg::PX, col = e - row * Cfg::PX;
            const int ri = row * Cfg::TXP + col + (Cfg::HX - 4);
#pragma unroll
            for (int p = 0; p < 4; ++p)
                dst[p * Cfg::PAIR_FIELD + e] = make_float2(to_c<float>(src[PF[p][0] * Cfg::RAW_FIELD + ri]),
                                                           to_c<float>(src[PF[p][1] * Cfg::RAW_FIELD + ri]));
        }
        return true;
    };

    // dense index of (x, y, z) in the RK register / Kahan arrays, and padded index of the output
    const int64_t nxy = g.n[0] * g.n[1];
    int64_t cell = (int64_t)x + g.n[0] * y + nxy * zc0;
    int64_t oidx = g.idx(x, y, zc0);
    const int64_t opitch = g.pad[0] * g.pad[1];
    const bool edge_xy = x < R6 || x >= nx - R6 || y < R6 || y >= ny - R6;

    float wpre[8], kpre[8];
    auto prefetch = [&](int64_t c) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            wpre[q] = (MODE == 0 && !first) ? to_c<float>(static_cast<const S *>(wbuf.p[q])[c]) : 0.f;
            kpre[q] = (MODE == 0) ? to_c<float>(static_cast<const S *>(kbuf.p[q])[c]) : 0.f;
        }
    };
    if (!TMAIO && active && zc0 < zend) prefetch(cell);

    // prologue: planes 0 .. 5 into the pair ring
    bool ok = true, bad = false;
    for (int j = 0; !bad && j < 2 * R6; ++j) {
        ok = convert(j);
        bad = __syncthreads_or(!ok);
        if (!bad && threadIdx.x == 0 && issued < nplanes && issued == j + NR) issue(issued++);
    }

    const int own = (ty + R6) * Cfg::PX + tx + 4;
    for (int m = 0; !bad && m < zend - zc0; ++m) {
        const int jl = m + 2 * R6;  // the leading plane z + 3
        ok = convert(jl);
        bad = __syncthreads_or(!ok);
        if (bad) break;
        if (threadIdx.x == 0) {
            if (issued < nplanes && issued == jl + NR) issue(issued++);
            if (TMAIO && m + 1 < zend - zc0) {
                bulk_wait_read<0>();  // plane m-1's stores have read buffer (m+1) & 1
                load_wc(m + 1);
            }
        }
        const int b = m & 1;
        if (TMAIO && active) ok = mbar_wait_bounded(&wcbar[b], ((unsigned)m >> 1) & 1u);
        if (active && ok) {
            const int z = zc0 + m;
            W w;
#pragma unroll
            for (int kk = 0; kk < 7; ++kk) w.p[kk] = pairs + ((m + kk) & 7) * Cfg::PAIR_SLOT + own;
            float wcur[8], kcur[8];
            if (TMAIO) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    wcur[q] = first ? 0.f : to_c<float>(stg(b, q)[threadIdx.x]);
                    kcur[q] = to_c<float>(stg(b, 8 + q)[threadIdx.x]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) { wcur[q] = wpre[q]; kcur[q] = kpre[q]; }
                if (m + 1 < zend - zc0) prefetch(cell + nxy);  // next plane, overlapped with compute
            }
            float rhs[8], val[8];
            mhdp_rhs_cell(w, k, rhs, val);
            if (MODE == 1) {
#pragma unroll
                for (int q = 0; q < 8; ++q) static_cast<float *>(rbuf.p[q])[cell] = rhs[q];
            } else {
                S fnew[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float wv = first ? k.dt * rhs[q] : fmaf(k.alpha, wcur[q], k.dt * rhs[q]);
                    const float yv = k.beta * wv - kcur[q];
                    fnew[q] = to_s<S>(val[q] + yv);
                    const S cnew = to_s<S>((to_c<float>(fnew[q]) - val[q]) - yv);
                    if (TMAIO) {
                        stg(b, q)[threadIdx.x] = to_s<S>(wv);
                        stg(b, 8 + q)[threadIdx.x] = cnew;
                        stg(b, 16 + q)[threadIdx.x] = fnew[q];
                    } else {
                        if (!last) static_cast<S *>(wbuf.p[q])[cell] = to_s<S>(wv);
                        static_cast<S *>(kbuf.p[q])[cell] = cnew;
                    }
                }
                if (TMAIO) {
                    // the interior values go out with the plane's TMA stores; edge cells add images
                    if (images && (edge_xy || z < R6 || z >= nz - R6)) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            store_with_images(static_cast<S *>(fout.p[q]), g, R6, true, x, y, z, fnew[q]);
                    }
                } else if (images && (edge_xy || z < R6 || z >= nz - R6)) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        store_with_images(static_cast<S *>(fout.p[q]), g, R6, true, x, y, z, fnew[q]);
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) static_cast<S *>(fout.p[q])[oidx] = fnew[q];
                }
            }
        }
        if (TMAIO) {
            fence_proxy_async();  // the staging writes above, before the TMA stores read them
            bad = __syncthreads_or(!ok);
            if (!bad && threadIdx.x == 0) {
                const int z = zc0 + m;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    tma_store_3d(&io->fo[q], stg(b, 16 + q), x0, y0, z);
                    if (!last) tma_store_3d(&io->w[q], stg(b, q), x0, y0, z);
                    tma_store_3d(&io->c[q], stg(b, 8 + q), x0, y0, z);
                }
                bulk_commit();
            }
        }
        cell += nxy;
        oidx += opitch;
    }
    if (TMAIO && threadIdx.x == 0) bulk_wait_all();  // staging stays valid until the stores are done
    if (bad && threadIdx.x == 0) {
        atomicOr(err, ERR_TIMEOUT);
        for (int j = max(0, issued - NR); j < issued; ++j)
            (void)mbar_wait_bounded(&full[j & (NR - 1)], ((unsigned)j / NR) & 1u, 100000000ull);
        if (TMAIO)  // and the w/c loads still in flight (at most the last two planes)
            for (int j = max(0, wc_issued - 2); j < wc_issued; ++j)
                (void)mbar_wait_bounded(&wcbar[j & 1], ((unsigned)j >> 1) & 1u, 100000000ull);
    }
    return !bad;
}

template <typename S, int TY, int NR, int MODE, bool TMAIO>
__global__ void __launch_bounds__(32 * TY, 1)
mhdp_kernel(const __grid_constant__ MhdMaps maps, const __grid_constant__ MhdIoMaps io, Ptrs8 fout, Ptrs8 wbuf,
            Ptrs8 kbuf, Ptrs8 rbuf, Geom g, MK<float> k, int zc, int first, int last, int images, unsigned *err) {
    using Cfg = MpCfg<S, TY, NR, TMAIO>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    S *raw = reinterpret_cast<S *>(base);
    float2 *pairs = reinterpret_cast<float2 *>(base + Cfg::RAW_BYTES);
    S *stage = reinterpret_cast<S *>(base + Cfg::RAW_BYTES + Cfg::PAIR_BYTES);
    __shared__ __align__(8) uint64_t full[NR];
    __shared__ __align__(8) uint64_t wcbar[2];
    mhdp_tile<S, TY, NR, MODE, TMAIO>(maps.m, &io, fout, wbuf, kbuf, rbuf, g, k, blockIdx.x, blockIdx.y, blockIdx.z,
                                      zc, first, last, images, err, raw, pairs, stage, full, wcbar);
}

template <typename S, int TY, int NR, int MODE, bool TMAIO = false>
cudaError_t runp(int sub, const MhdMaps &maps, const MhdIoMaps *io, const Ptrs8 &fo, const Ptrs8 &w,
                 const Ptrs8 &kc, const Ptrs8 &rhs, const Geom &g, const MK<float> &k, bool images, unsigned *err,
                 cudaStream_t s) {
    using Cfg = MpCfg<S, TY, NR, TMAIO>;
    auto kern = mhdp_kernel<S, TY, NR, MODE, TMAIO>;
    static int occ[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (!occ[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, 32 * TY, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        occ[dev] = std::max(o, 1);
    }
    const int tx = (int)((g.n[0] + Cfg::TX - 1) / Cfg::TX), ty = (int)((g.n[1] + TY - 1) / TY);
    const int nz = (int)g.n[2];
    const int chunks = choose_zchunks(tx * ty, nz, occ[dev] * device_sms(), 0.5);
    const int zc = (nz + chunks - 1) / chunks;
    dim3 grid(tx, ty, (unsigned)((nz + zc - 1) / zc));
    static const MhdIoMaps none{};
    kern<<<grid, 32 * TY, Cfg::SMEM, s>>>(maps, io ? *io : none, fo, w, kc, rhs, g, k, zc, sub == 0 ? 1 : 0,
                                          sub == 2 ? 1 : 0, images ? 1 : 0, err);
    return cudaGetLastError();
}

// Variants: (TY rows of 32 cells, NR raw planes, TMA I/O).
#define MHDP_VARIANTS(X) X(8, 4, false) X(8, 2, false) X(8, 2, true)

}  // namespace

int mhd_pairs_num_variants() { return 3; }

const char *mhd_pairs_variant_name(int v) {
    static const char *names[] = {"pairs_tx32_ty8_raw4", "pairs_tx32_ty8_raw2", "pairs_tx32_ty8_raw2_tmaio"};
    return (v >= 0 && v < 3) ? names[v] : "?";
}

bool mhd_pairs_variant_uses_io(int v) { return v == 2; }
int mhd_pairs_io_box_rows(int v) { (void)v; return 8; }

void mhd_pairs_box(int storage, int v, int box[3]) {
    int i = 0;
#define X(TY, NR, IO)                                                                                 \
    if (i++ == v) {                                                                                   \
        box[0] = storage == 3 ? MpCfg<__nv_bfloat16, TY, NR>::TXP : MpCfg<float, TY, NR>::TXP;        \
        box[1] = TY + 2 * R6;                                                                         \
        box[2] = 1;                                                                                   \
    }
    MHDP_VARIANTS(X)
#undef X
}

cudaError_t launch_mhd_pairs(int storage, int mode, int sub, const MhdMaps &maps, const MhdIoMaps *io,
                             const Ptrs8 &fo, const Ptrs8 &w, const Ptrs8 &kc, const Ptrs8 &rhs, const Geom &g,
                             const MK<float> &k, bool images, unsigned *err, cudaStream_t s, int variant) {
    int i = 0;
    cudaError_t res = cudaErrorInvalidValue;
    // the TMA-I/O variant needs its descriptors and serves the RK substep; otherwise its plain twin
    const bool io_ok = io != nullptr && mode == 0;
#define X(TY, NR, IO)                                                                                       \
    if (i++ == variant) {                                                                                   \
        bool done = false;                                                                                  \
        if constexpr (IO) {                                                                                 \
            if (mode == 0 && io_ok) {                                                                       \
                res = runp<S, TY, NR, 0, true>(sub, maps, io, fo, w, kc, rhs, g, k, images, err, s);        \
                done = true;                                                                                \
            }                                                                                               \
        }                                                                                                   \
        if (!done)                                                                                          \
            res = mode == 0 ? runp<S, TY, NR, 0>(sub, maps, nullptr, fo, w, kc, rhs, g, k, images, err, s)  \
                            : runp<S, TY, NR, 1>(sub, maps, nullptr, fo, w, kc, rhs, g, k, images, err, s); \
    }
    if (storage == 2) {
        using S = float;
        MHDP_VARIANTS(X)
    } else if (storage == 3) {
        using S = __nv_bfloat16;
        MHDP_VARIANTS(X)
    }
#undef X
    return res;
}

}  // namespace stn
