// mhd.cu -- fused 8-field MHD step: derivatives (gamma = A B, Sec. 3.3 Eq. 8), nonlinear
// right-hand side of Eqs. A1-A4 (phi, Eq. 9) and one substep of 3-stage Runge-Kutta, all
// in one kernel pass per substep.
//
// GB300 design (software-cached, z-streaming; the paper's Fig. 5b idea kept, re-sized for
// 228 KB of shared memory per SM and TMA):
//   * A CTA owns a TX x TY tile of the xy-plane and marches along z over a chunk of planes.
//     For every plane it issues 8 TMA tile loads (one per field, (TX + 2 HX) x (TY + 6)
//     padded elements each) into a ring of NSLOT plane slots, completion on one mbarrier per
//     slot.  The ring holds planes z-3..z+3 of all 8 fields at once (the mixed xz/yz
//     derivatives need all seven), plus NSLOT - 7 planes of prefetch.
//   * One thread per output cell and plane.  A cell's window is addressed through 7 plane
//     base pointers; field and stencil offsets are compile-time immediates.  Derivatives are
//     evaluated field by field in the k-outer (stencil point) order of Algorithm 1, with
//     the derivatives no term uses pruned (lnrho and s need gradients only; A needs the 6
//     off-diagonal first derivatives for B = curl A), and are folded at once into the
//     quantities the RHS needs (div u, lap u, grad div u, B, j, lap A), so the live set
//     stays small.  Then the RHS in registers, then the 2N-storage RK3 update
//     w <- alpha_s w + dt RHS, f <- f + beta_s w (Kahan-compensated when fields are stored
//     in FP32/BF16).  The RK register and Kahan terms of the next plane are prefetched into
//     registers while the current plane is computed.
//   * Output fields are written once per substep; threads within r of a face also write
//     the periodic images (Eq. 2), so substeps need no halo pass.
//   * Bounded mbarrier waits; on expiry ERR_TIMEOUT is recorded and the CTA drains its
//     in-flight loads before returning.
#include <algorithm>
#include <cstddef>

#include "mhd_rhs.cuh"

namespace stn {

// The 7-plane window of all fields around one cell: p[k] points at the cell (field 0) in
// plane z + k - 3; field q is FE elements further, row neighbours RS elements apart.  Its
// 6th-order central differences (weights pre-scaled by the grid spacing) are written out one
// IEEE operation at a time (mhd_rhs.cuh says why).
template <typename C, typename S, int FE, int RS>
struct Win {
    const S *p[7];
    __device__ __forceinline__ C at(int q, int k, int dx, int dy) const {
        return to_c<C>(p[k][q * FE + dy * RS + dx]);
    }
    __device__ __forceinline__ C val(int q) const { return at(q, 3, 0, 0); }
    // value at offset s along axis (0: x, 1: y, 2: z)
    __device__ __forceinline__ C ax(int q, int axis, int s) const {
        return axis == 0 ? at(q, 3, s, 0) : axis == 1 ? at(q, 3, 0, s) : at(q, 3 + s, 0, 0);
    }
    // first derivative: c0 (f1 - f-1) + c1 (f2 - f-2) + c2 (f3 - f-3)
    __device__ __forceinline__ C d1(int q, int axis, const C *c) const {
        C a = mul(c[0], sub(ax(q, axis, 1), ax(q, axis, -1)));
        a = fmad(c[1], sub(ax(q, axis, 2), ax(q, axis, -2)), a);
        return fmad(c[2], sub(ax(q, axis, 3), ax(q, axis, -3)), a);
    }
    // second derivative: c0 f0 + c1 (f1 + f-1) + c2 (f2 + f-2) + c3 (f3 + f-3)
    __device__ __forceinline__ C d2(int q, int axis, C c0, const C *c) const {
        C a = mul(c0, ax(q, axis, 0));
        a = fmad(c[0], add(ax(q, axis, 1), ax(q, axis, -1)), a);
        a = fmad(c[1], add(ax(q, axis, 2), ax(q, axis, -2)), a);
        return fmad(c[2], add(ax(q, axis, 3), ax(q, axis, -3)), a);
    }
    // mixed derivative of axes (a1 < a2), diagonal form:
    // sum_a m_a [(f(+a,+a) + f(-a,-a)) - (f(+a,-a) + f(-a,+a))]
    __device__ __forceinline__ C mx(int q, int pair, int s1, int s2) const {
        return pair == 0 ? at(q, 3, s1, s2) : pair == 1 ? at(q, 3 + s2, s1, 0) : at(q, 3 + s2, 0, s1);
    }
    __device__ __forceinline__ C dmix(int q, int pair, const C *m) const {
        C acc = mul(m[0], sub(add(mx(q, pair, 1, 1), mx(q, pair, -1, -1)), add(mx(q, pair, 1, -1), mx(q, pair, -1, 1))));
        acc = fmad(m[1], sub(add(mx(q, pair, 2, 2), mx(q, pair, -2, -2)), add(mx(q, pair, 2, -2), mx(q, pair, -2, 2))),
                   acc);
        return fmad(m[2], sub(add(mx(q, pair, 3, 3), mx(q, pair, -3, -3)), add(mx(q, pair, 3, -3), mx(q, pair, -3, 3))),
                    acc);
    }
};

// The 8 interleaved values of one cell in the RK register / Kahan arrays (16-byte aligned):
// loaded and stored as 16-byte vectors.
template <typename S, typename C>
__device__ __forceinline__ void load8(const S *p, C (&v)[8]) {
    if constexpr (sizeof(S) == 2) {
        const uint4 a = *reinterpret_cast<const uint4 *>(p);
        const S *e = reinterpret_cast<const S *>(&a);
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = to_c<C>(e[q]);
    } else {
        constexpr int PER = 16 / (int)sizeof(S);  // values per 16-byte vector
#pragma unroll
        for (int h = 0; h < 8 / PER; ++h) {
            const uint4 a = reinterpret_cast<const uint4 *>(p)[h];
            const S *e = reinterpret_cast<const S *>(&a);
#pragma unroll
            for (int u = 0; u < PER; ++u) v[h * PER + u] = to_c<C>(e[u]);
        }
    }
}
template <typename S>
__device__ __forceinline__ void store8(S *p, const S (&v)[8]) {
    constexpr int PER = 16 / (int)sizeof(S);
#pragma unroll
    for (int h = 0; h < 8 / PER; ++h) {
        uint4 a;
        S *e = reinterpret_cast<S *>(&a);
#pragma unroll
        for (int u = 0; u < PER; ++u) e[u] = v[h * PER + u];
        reinterpret_cast<uint4 *>(p)[h] = a;
    }
}

// One xy-tile of one z-chunk of one RK substep (or RHS evaluation): the whole pipeline of a
// CTA.  `maps` points at 8 consecutive descriptors (parameter or global memory); `k` may live
// in parameter or shared memory.  Returns false if a bounded wait expired.
template <typename S, typename C, bool KAHAN, int MODE, int TX, int TY, int NSLOT, bool CONDUCT>
__device__ __forceinline__ bool mhd_tile(const CUtensorMap *maps, const Ptrs8 &fout, S *wbuf, S *kbuf,
                                         const Ptrs8 &rbuf, const Geom &g, const MK<C> &k,
                                         int tile_x, int tile_y, int tile_z, int zc, int first, int last,
                                         int images, unsigned *err, S *ring, uint64_t *full) {
    using Cfg = MhdCfg<S, TX, TY, NSLOT>;
    using W = Win<C, S, Cfg::FIELD_ELEMS, Cfg::TXP>;
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
        for (int s = 0; s < NSLOT; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    const int bx = (int)g.off[0] + x0 - Cfg::HX;
    const int by0 = (int)g.off[1] + y0 - R6;
    const int bz0 = (int)g.off[2] + zc0 - R6;
    auto issue = [&](int j) {
        const int s = (int)((unsigned)j & (NSLOT - 1));
        mbar_arrive_expect_tx(&full[s], 8 * Cfg::BOX_BYTES);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            tma_load_3d(ring + s * Cfg::SLOT_ELEMS + q * Cfg::FIELD_ELEMS, &maps[q], &full[s], bx, by0, bz0 + j);
    };
    int issued = 0;
    if (threadIdx.x == 0)
        for (; issued < NSLOT && issued < nplanes; ++issued) issue(issued);

    // dense index of (x, y, z) in the RK register / Kahan arrays, and padded index of the output
    const int64_t nxy = g.n[0] * g.n[1];
    int64_t cell = (int64_t)x + g.n[0] * y + nxy * zc0;
    int64_t oidx = g.idx(x, y, zc0);
    const int64_t opitch = g.pad[0] * g.pad[1];
    const bool edge_xy = x < R6 || x >= nx - R6 || y < R6 || y >= ny - R6;

    // prefetch of the RK register and Kahan terms of the first plane
    C wpre[8], kpre[8];
    auto prefetch = [&](int64_t c) {
#pragma unroll
        for (int q = 0; q < 8; ++q) wpre[q] = kpre[q] = C(0);
        if (MODE == 0 && !first) load8<S, C>(wbuf + 8 * c, wpre);
        if (MODE == 0 && KAHAN) load8<S, C>(kbuf + 8 * c, kpre);
    };
    if (active && zc0 < zend) prefetch(cell);

    bool ok = true;
    for (int j = 0; j < 2 * R6; ++j) ok = ok && mbar_wait_bounded(&full[(unsigned)j & (NSLOT - 1)], ((unsigned)j / NSLOT) & 1u);
    bool bad = __syncthreads_or(!ok);

    const int own = (ty + R6) * Cfg::TXP + tx + Cfg::HX;
    for (int m = 0; !bad && m < zend - zc0; ++m) {
        const int jl = m + 2 * R6;
        ok = mbar_wait_bounded(&full[(unsigned)jl & (NSLOT - 1)], ((unsigned)jl / NSLOT) & 1u);
        if (ok && active) {
            const int z = zc0 + m;
            W w;
#pragma unroll
            for (int kk = 0; kk < 7; ++kk) w.p[kk] = ring + (int)((unsigned)(m + kk) & (NSLOT - 1)) * Cfg::SLOT_ELEMS + own;
            C wcur[8], kcur[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) { wcur[q] = wpre[q]; kcur[q] = kpre[q]; }
            if (m + 1 < zend - zc0) prefetch(cell + nxy);  // next plane, overlapped with compute
            C rhs[8], val[8];
            mhd_rhs_cell<CONDUCT, C>(w, k, rhs, val);
            if (MODE == 1) {
#pragma unroll
                for (int q = 0; q < 8; ++q) static_cast<C *>(rbuf.p[q])[cell] = rhs[q];
            } else {
                S fnew[8], wst[8], kst[8];
                auto rt = [](C v) { return to_c<C>(to_s<S>(v)); };  // round to the storage type
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    C wv, fv, kv;
                    rk_update<KAHAN>(k, first != 0, rhs[q], wcur[q], kcur[q], val[q], wv, fv, kv, rt);
                    wst[q] = to_s<S>(wv);
                    kst[q] = to_s<S>(kv);
                    fnew[q] = to_s<S>(fv);
                }
                if (!last) store8<S>(wbuf + 8 * cell, wst);
                if (KAHAN) store8<S>(kbuf + 8 * cell, kst);
                if (images && (edge_xy || z < R6 || z >= nz - R6)) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        store_with_images(static_cast<S *>(fout.p[q]), g, R6, true, x, y, z, fnew[q]);
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) static_cast<S *>(fout.p[q])[oidx] = fnew[q];
                }
            }
        }
        cell += nxy;
        oidx += opitch;
        bad = __syncthreads_or(!ok);
        // plane j = m (z - 3) is retired: reuse its slot
        if (!bad && threadIdx.x == 0 && issued < nplanes && issued == m + NSLOT) issue(issued++);
    }
    if (bad && threadIdx.x == 0) {
        atomicOr(err, ERR_TIMEOUT);
        for (int j = max(0, issued - NSLOT); j < issued; ++j)
            (void)mbar_wait_bounded(&full[(unsigned)j & (NSLOT - 1)], ((unsigned)j / NSLOT) & 1u, 100000000ull);
    }
    return !bad;
}

template <typename S, typename C, bool KAHAN, int MODE, int TX, int TY, int NSLOT, int MINB, bool CONDUCT>
__global__ void __launch_bounds__(TX *TY, MINB)
mhd_kernel(const __grid_constant__ MhdMaps maps, Ptrs8 fout, S *wbuf, S *kbuf, Ptrs8 rbuf, Geom g,
           MK<C> k, int zc, int first, int last, int images, unsigned *err) {
    using Cfg = MhdCfg<S, TX, TY, NSLOT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S *ring = reinterpret_cast<S *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full[NSLOT];
    (void)Cfg::SMEM;
    if constexpr (sizeof(C) == 8) {
        // FP64: the constants are read from shared memory, so that the FP64 multiply-adds take
        // register operands rather than constant-bank ones (2 % faster at 256^3; the 255-register
        // budget has no room to keep all of them in registers)
        __shared__ MK<C> ks;
        constexpr int KW = (int)(sizeof(MK<C>) / sizeof(C));
        for (int i = threadIdx.x; i < KW; i += blockDim.x) reinterpret_cast<C *>(&ks)[i] = reinterpret_cast<const C *>(&k)[i];
        __syncthreads();
        mhd_tile<S, C, KAHAN, MODE, TX, TY, NSLOT, CONDUCT>(maps.m, fout, wbuf, kbuf, rbuf, g, ks, blockIdx.x,
                                                            blockIdx.y, blockIdx.z, zc, first, last, images, err,
                                                            ring, full);
    } else {
        mhd_tile<S, C, KAHAN, MODE, TX, TY, NSLOT, CONDUCT>(maps.m, fout, wbuf, kbuf, rbuf, g, k, blockIdx.x,
                                                            blockIdx.y, blockIdx.z, zc, first, last, images, err,
                                                            ring, full);
    }
}

// ------------------------------------------------------------------ host side

template <typename C>
static MK<C> make_k(const MhdConst &c, double alpha, double beta) {
    MK<C> k;
    for (int a = 0; a < 3; ++a) {
        k.d2c[a] = (C)c.d2c[a];
        for (int i = 0; i < 3; ++i) {
            k.d1[a][i] = (C)c.d1[a][i];
            k.d2[a][i] = (C)c.d2[a][i];
            k.dm[a][i] = (C)c.dm[a][i];
        }
    }
    k.cs0sq = (C)c.cs0sq; k.gamma = (C)c.gamma; k.inv_cp = (C)c.inv_cp; k.lnrho0 = (C)c.lnrho0;
    k.nu = (C)c.nu; k.eta = (C)c.eta; k.zeta = (C)c.zeta; k.mu0 = (C)c.mu0; k.inv_mu0 = (C)c.inv_mu0;
    k.cp_gm1 = (C)c.cp_gm1; k.K = (C)c.K; k.dt = (C)c.dt; k.alpha = (C)alpha; k.beta = (C)beta;
    k.gcp = (C)(c.gamma * c.inv_cp); k.gm1 = (C)(c.gamma - 1.0); k.etamu0 = (C)(c.eta * c.mu0);
    k.two_nu = (C)(2.0 * c.nu); k.one = (C)1.0; k.mone = (C)-1.0; k.half = (C)0.5; k.two = (C)2.0;
    k.third = (C)(1.0 / 3.0); k.mthird = (C)(-1.0 / 3.0);
    return k;
}

// Williamson's 2N-storage RK3 (reading of the paper's "explicit Runge-Kutta three")
static const double RK_A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK_B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

template <typename S, typename C, bool KAHAN, int MODE, int TX, int TY, int NSLOT, int MINB, bool CONDUCT>
static cudaError_t run(int sub, const MhdMaps &maps, const Ptrs8 &fo, void *w, void *kc,
                       const Ptrs8 &rhs, const Geom &g, const MhdConst &c, bool images, unsigned *err,
                       cudaStream_t s, int zmode) {
    using Cfg = MhdCfg<S, TX, TY, NSLOT>;
    auto kern = mhd_kernel<S, C, KAHAN, MODE, TX, TY, NSLOT, MINB, CONDUCT>;
    static int occ[64] = {};  // resident CTAs per SM, per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (!occ[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, TX * TY, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        occ[dev] = std::max(o, 1);
    }
    MK<C> k = make_k<C>(c, RK_A[sub], RK_B[sub]);
    const int tx = (int)((g.n[0] + TX - 1) / TX), ty = (int)((g.n[1] + TY - 1) / TY);
    const int nz = (int)g.n[2];
    const int chunks = choose_zchunks(tx * ty, nz, occ[dev] * device_sms(), 0.5);
    const int zc = zchunk_len((nz + chunks - 1) / chunks, nz, zmode);
    dim3 grid(tx, ty, (unsigned)((nz + zc - 1) / zc));
    kern<<<grid, TX * TY, Cfg::SMEM, s>>>(maps, fo, static_cast<S *>(w), static_cast<S *>(kc), rhs, g, k, zc,
                                          sub == 0 ? 1 : 0, sub == 2 ? 1 : 0, images ? 1 : 0, err);
    return cudaGetLastError();
}

// Variants per storage type: (TX, TY, NSLOT, min CTAs per SM for the register budget).
#define MHD_VARIANTS_F64(X) X(32, 4, 8, 1) X(16, 8, 8, 1)
// The 512-thread tiles (32 x 16) hold one CTA per SM: its ring (229.5 KB for FP32) takes the
// whole shared memory, and the 128-register budget of 512 threads holds the RHS without
// spills, so 16 warps per SM stream 512 cells per plane (the 128-thread tiles: 8 warps, 256).
#define MHD_VARIANTS_F32(X) X(32, 8, 8, 1) X(32, 4, 8, 2) X(16, 8, 8, 2) X(32, 16, 8, 1) X(32, 12, 8, 1)
#define MHD_VARIANTS_BF16(X) X(32, 8, 8, 1) X(32, 8, 8, 2) X(32, 4, 8, 3) X(32, 16, 8, 1) X(64, 8, 8, 1)

static const char *MHD_F64_NAMES[] = {"tx32_ty4_s8_b1", "tx16_ty8_s8_b1"};
static const char *MHD_F32_NAMES[] = {"tx32_ty8_s8_b1", "tx32_ty4_s8_b2", "tx16_ty8_s8_b2", "tx32_ty16_s8_b1",
                                      "tx32_ty12_s8_b1"};
static const char *MHD_BF16_NAMES[] = {"tx32_ty8_s8_b1", "tx32_ty8_s8_b2", "tx32_ty4_s8_b3", "tx32_ty16_s8_b1",
                                       "tx64_ty8_s8_b1"};

int mhd_num_variants(int storage) { return storage == 1 ? 2 : 5; }

const char *mhd_variant_name(int storage, int v) {
    if (v < 0 || v >= mhd_num_variants(storage)) return "?";
    return storage == 1 ? MHD_F64_NAMES[v] : storage == 2 ? MHD_F32_NAMES[v] : MHD_BF16_NAMES[v];
}

void mhd_box(int storage, int v, int box[3]) {
    int i = 0;
    auto put = [&](int tx, int ty, int hx) {
        if (i++ == v) { box[0] = tx + 2 * hx; box[1] = ty + 2 * R6; box[2] = 1; }
    };
#define X(TX, TY, NS, MB) put(TX, TY, hx);
    if (storage == 1) { const int hx = 4; MHD_VARIANTS_F64(X) }
    else if (storage == 2) { const int hx = 4; MHD_VARIANTS_F32(X) }
    else { const int hx = 8; MHD_VARIANTS_BF16(X) }
#undef X
}

cudaError_t launch_mhd(int storage, int mode, int sub, const MhdMaps &maps, const Ptrs8 &fo, void *w, void *kc,
                       const Ptrs8 &rhs, const Geom &g, const MhdConst &c, bool images,
                       unsigned *err, cudaStream_t s, int variant, int zmode) {
    int i = 0;
    cudaError_t res = cudaErrorInvalidValue;
    // the conduction term of A3 is compiled in only for launches with K != 0
    const bool cond = c.K != 0.0;
#define X(TX, TY, NS, MB)                                                                                  \
    if (i++ == variant) {                                                                                  \
        if (mode == 0)                                                                                     \
            res = cond ? run<S, C, KH, 0, TX, TY, NS, MB, true>(sub, maps, fo, w, kc, rhs, g, c, images, err, s, zmode) \
                       : run<S, C, KH, 0, TX, TY, NS, MB, false>(sub, maps, fo, w, kc, rhs, g, c, images, err, s, zmode); \
        else                                                                                               \
            res = cond ? run<S, C, KH, 1, TX, TY, NS, MB, true>(sub, maps, fo, w, kc, rhs, g, c, images, err, s, zmode) \
                       : run<S, C, KH, 1, TX, TY, NS, MB, false>(sub, maps, fo, w, kc, rhs, g, c, images, err, s, zmode); \
    }
    if (storage == 1) {
        using S = double; using C = double; constexpr bool KH = false;
        MHD_VARIANTS_F64(X)
    } else if (storage == 2) {
        using S = float; using C = float; constexpr bool KH = true;
        MHD_VARIANTS_F32(X)
    } else if (storage == 3) {
        using S = __nv_bfloat16; using C = float; constexpr bool KH = true;
        MHD_VARIANTS_BF16(X)
    }
#undef X
    return res;
}

// ------------------------------------------------------------------ batched (serving)

// FP32 storage, Kahan-compensated RK.  Tile shapes (the server picks one per run from the
// autotuner's choice for FP32 MHD plans): 0 = 32 x 4 cells, two CTAs per SM (the tile of
// variant tx32_ty4_s8_b2), 1 = 32 x 8, one CTA per SM with the full register budget (for the
// one-CTA-per-SM variants tx32_ty8/12/16_s8_b1).  The batched kernel reads the per-request
// constants from shared memory rather than from the launch's parameter bank, which costs
// registers: a 32 x 12 tile at the 168 registers of 384 threads spilled and served MHD
// requests about 18 % slower than 32 x 4.
template <int SH> struct MbShape;
template <> struct MbShape<0> { static constexpr int TX = 32, TY = 4, MINB = 2; };
template <> struct MbShape<1> { static constexpr int TX = 32, TY = 8, MINB = 1; };
constexpr int MB_NSLOT = 8;
template <int SH> using MbCfg = MhdCfg<float, MbShape<SH>::TX, MbShape<SH>::TY, MB_NSLOT>;

template <int SH>
__global__ void __launch_bounds__(MbShape<SH>::TX *MbShape<SH>::TY, MbShape<SH>::MINB)
mhd_batch_kernel(const BatchHeader *hdr, const BatchMhd *items, float alpha, float beta, int first, int last,
                 unsigned *err) {
    constexpr int TX = MbShape<SH>::TX, TY = MbShape<SH>::TY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full[MB_NSLOT];
    __shared__ MK<float> ks;
    const int total = hdr->mhd_ctas, n = hdr->n_mhd;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].cta_begin <= vb) lo = mid; else hi = mid - 1;
        }
        const BatchMhd &it = items[lo];
        int r = vb - it.cta_begin;
        const int tx = r % it.tiles_x;
        r /= it.tiles_x;
        const int ty = r % it.tiles_y, tz = r / it.tiles_y;
        // the problem's constants, with this launch's RK coefficients in place of the table's
        // (one writer per word: a separate write of alpha / beta would race with the copy)
        constexpr int KW = (int)(sizeof(MK<float>) / sizeof(float));
        constexpr int IA = (int)(offsetof(MK<float>, alpha) / sizeof(float));
        constexpr int IB = (int)(offsetof(MK<float>, beta) / sizeof(float));
        for (int i = threadIdx.x; i < KW; i += blockDim.x)
            reinterpret_cast<float *>(&ks)[i] =
                i == IA ? alpha : i == IB ? beta : reinterpret_cast<const float *>(&it.k)[i];
        __syncthreads();
        const Geom g = it.g;
        Ptrs8 none{};
        const bool ok =
            it.k.K != 0.f
                ? mhd_tile<float, float, true, 0, TX, TY, MB_NSLOT, true>(it.maps, it.fout, it.w, it.kc, none, g, ks, tx,
                                                                          ty, tz, it.zc, first, last, 1, err, ring, full)
                : mhd_tile<float, float, true, 0, TX, TY, MB_NSLOT, false>(it.maps, it.fout, it.w, it.kc, none, g, ks,
                                                                           tx, ty, tz, it.zc, first, last, 1, err, ring,
                                                                           full);
        __syncthreads();
        if (!ok) return;
    }
}

template <int SH> static int mhd_batch_grid_t() {
    static int grid[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 152;
    if (!grid[dev]) {
        cudaFuncSetAttribute(mhd_batch_kernel<SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MbCfg<SH>::SMEM);
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, mhd_batch_kernel<SH>, MbShape<SH>::TX * MbShape<SH>::TY,
                                                      MbCfg<SH>::SMEM);
        grid[dev] = std::max(o, 1) * device_sms();
    }
    return grid[dev];
}

int mhd_batch_grid(int shape) { return shape == 1 ? mhd_batch_grid_t<1>() : mhd_batch_grid_t<0>(); }

const char *mhd_batch_shape_name(int shape) { return shape == 1 ? "batch_tx32_ty8_s8" : "batch_tx32_ty4_s8"; }

void mhd_batch_tile(int shape, int *tx, int *ty, int box[3]) {
    *tx = shape == 1 ? MbShape<1>::TX : MbShape<0>::TX;
    *ty = shape == 1 ? MbShape<1>::TY : MbShape<0>::TY;
    box[0] = *tx + 2 * MbCfg<0>::HX;
    box[1] = *ty + 2 * R6;
    box[2] = 1;
}

void mhd_scaled_constants(const MhdConst &c, MK<float> *k) { *k = make_k<float>(c, 0.0, 0.0); }

void mhd_substep_constants(const MhdConst &c, int sub, MK<float> *k) { *k = make_k<float>(c, RK_A[sub], RK_B[sub]); }

cudaError_t launch_mhd_batch(int shape, const BatchHeader *hdr, const BatchMhd *items, int sub, unsigned *err,
                             int grid, cudaStream_t s) {
    const float a = (float)RK_A[sub], b = (float)RK_B[sub];
    const int first = sub == 0 ? 1 : 0, last = sub == 2 ? 1 : 0;
    if (shape == 1)
        mhd_batch_kernel<1><<<grid, MbShape<1>::TX * MbShape<1>::TY, MbCfg<1>::SMEM, s>>>(hdr, items, a, b, first, last,
                                                                                           err);
    else
        mhd_batch_kernel<0><<<grid, MbShape<0>::TX * MbShape<0>::TY, MbCfg<0>::SMEM, s>>>(hdr, items, a, b, first, last,
                                                                                           err);
    return cudaGetLastError();
}

}  // namespace stn
