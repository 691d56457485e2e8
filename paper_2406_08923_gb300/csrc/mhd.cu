// mhd.cu -- fused 8-field MHD step: derivatives (gamma = A B, Sec. 3.3 Eq. 8), nonlinear
// right-hand side of Eqs. A1-A4 (phi, Eq. 9) and one substep of 3-stage Runge-Kutta, all
// in one kernel pass per substep.
//
// GB300 design (software-cached, z-streaming; the paper's Fig. 5b idea kept, re-sized for
// 228 KB of shared memory per SM and TMA):
//   * A CTA owns a TX x TY tile of the xy-plane and marches along z over ZC planes.  For
//     every plane it issues 8 TMA tile loads (one per field, (TX + 2 HX) x (TY + 6) padded
//     elements each) into a ring of NSLOT plane slots, completion on one mbarrier per slot.
//     The ring holds planes z-3..z+3 of all 8 fields at once (the mixed xz/yz derivatives
//     need all seven), plus NSLOT - 7 planes of prefetch.
//   * One thread per output cell and plane.  It evaluates the 6th-order central 1st,
//     2nd and mixed derivatives each field needs straight from shared memory in the
//     k-outer (stencil point) order of Algorithm 1, with zero-weight points pruned
//     (lnrho and s need first derivatives only; u and A need the full Hessian), then the
//     RHS in registers, then the 2N-storage RK3 update w <- alpha_s w + dt RHS,
//     f <- f + beta_s w (Kahan-compensated when fields are stored in FP32/BF16).
//   * Output fields are written once per substep with their periodic images (Eq. 2), so
//     substeps need no halo pass; w and the Kahan terms are dense interior arrays.
//   * Bounded mbarrier waits; on expiry ERR_TIMEOUT is recorded and the CTA drains its
//     in-flight loads before returning.
#include "internal.h"

namespace stn {

enum { F_LNRHO = 0, F_UX, F_UY, F_UZ, F_AX, F_AY, F_AZ, F_SS };

template <typename C> struct MK {
    C d1[3][3], d2c[3], d2[3][3], dm[3][3];
    C cs0sq, gamma, inv_cp, lnrho0, nu, eta, zeta, mu0, inv_mu0, cp_gm1;
    C dt, alpha, beta;
};

template <typename S, int TX, int TY, int NSLOT>
struct MhdCfg {
    static constexpr int HX = 16 / (int)sizeof(S) >= 4 ? 16 / (int)sizeof(S) : 4;
    static constexpr int TXP = TX + 2 * HX;
    static constexpr int ROWS = TY + 2 * R6;
    static constexpr int FIELD_ELEMS = ((TXP * ROWS * (int)sizeof(S) + 127) / 128) * 128 / (int)sizeof(S);
    static constexpr int SLOT_ELEMS = 8 * FIELD_ELEMS;
    static constexpr uint32_t BOX_BYTES = TXP * ROWS * sizeof(S);
    static constexpr size_t SMEM = (size_t)NSLOT * SLOT_ELEMS * sizeof(S) + 128;
    static_assert((TXP * sizeof(S)) % 16 == 0, "TMA box inner extent must be a multiple of 16 B");
    static_assert(NSLOT >= 8, "ring holds 7 planes plus at least one in flight");
};

// Derivative helpers on shared-memory tiles.  p points at the cell; s is the stride of the
// axis within a plane (1 or the row pitch); pz[k] points at the cell in plane z + k - 3.
template <typename C, typename S>
__device__ __forceinline__ C ld(const S *p) { return to_c<C>(*p); }

template <typename C, typename S>
__device__ __forceinline__ C der1(const S *p, int s, const C *w) {
    C a = w[0] * (ld<C>(p + s) - ld<C>(p - s));
    a = fma(w[1], ld<C>(p + 2 * s) - ld<C>(p - 2 * s), a);
    return fma(w[2], ld<C>(p + 3 * s) - ld<C>(p - 3 * s), a);
}
template <typename C, typename S>
__device__ __forceinline__ C der1z(const S *const *pz, const C *w) {
    C a = w[0] * (ld<C>(pz[4]) - ld<C>(pz[2]));
    a = fma(w[1], ld<C>(pz[5]) - ld<C>(pz[1]), a);
    return fma(w[2], ld<C>(pz[6]) - ld<C>(pz[0]), a);
}
template <typename C, typename S>
__device__ __forceinline__ C der2(const S *p, int s, C wc, const C *w) {
    C a = wc * ld<C>(p);
    a = fma(w[0], ld<C>(p + s) + ld<C>(p - s), a);
    a = fma(w[1], ld<C>(p + 2 * s) + ld<C>(p - 2 * s), a);
    return fma(w[2], ld<C>(p + 3 * s) + ld<C>(p - 3 * s), a);
}
template <typename C, typename S>
__device__ __forceinline__ C der2z(const S *const *pz, C wc, const C *w) {
    C a = wc * ld<C>(pz[3]);
    a = fma(w[0], ld<C>(pz[4]) + ld<C>(pz[2]), a);
    a = fma(w[1], ld<C>(pz[5]) + ld<C>(pz[1]), a);
    return fma(w[2], ld<C>(pz[6]) + ld<C>(pz[0]), a);
}
// mixed derivative in one plane, strides s1, s2:
// sum_a m_a [(f(+a,+a) + f(-a,-a)) - (f(+a,-a) + f(-a,+a))]
template <typename C, typename S>
__device__ __forceinline__ C derm(const S *p, int s1, int s2, const C *m) {
    C acc = C(0);
#pragma unroll
    for (int a = 1; a <= 3; ++a) {
        C d = (ld<C>(p + a * s1 + a * s2) + ld<C>(p - a * s1 - a * s2)) -
              (ld<C>(p + a * s1 - a * s2) + ld<C>(p - a * s1 + a * s2));
        acc = a == 1 ? m[0] * d : fma(m[a - 1], d, acc);
    }
    return acc;
}
// mixed derivative between an in-plane axis (stride s) and z
template <typename C, typename S>
__device__ __forceinline__ C dermz(const S *const *pz, int s, const C *m) {
    C acc = C(0);
#pragma unroll
    for (int a = 1; a <= 3; ++a) {
        C d = (ld<C>(pz[3 + a] + a * s) + ld<C>(pz[3 - a] - a * s)) -
              (ld<C>(pz[3 - a] + a * s) + ld<C>(pz[3 + a] - a * s));
        acc = a == 1 ? m[0] * d : fma(m[a - 1], d, acc);
    }
    return acc;
}

template <typename C> __device__ __forceinline__ C exp_c(C v);
template <> __device__ __forceinline__ double exp_c<double>(double v) { return exp(v); }
template <> __device__ __forceinline__ float exp_c<float>(float v) { return expf(v); }

// Gradient (3) and, when `hess`, Hessian (xx, yy, zz, xy, xz, yz) of one field.
template <typename C, typename S, bool HESS>
__device__ __forceinline__ void field_derivs(const S *const *pz, int rs, const MK<C> &k, C *g, C *h) {
    const S *p = pz[3];
    g[0] = der1<C>(p, 1, k.d1[0]);
    g[1] = der1<C>(p, rs, k.d1[1]);
    g[2] = der1z<C>(pz, k.d1[2]);
    if (HESS) {
        h[0] = der2<C>(p, 1, k.d2c[0], k.d2[0]);
        h[1] = der2<C>(p, rs, k.d2c[1], k.d2[1]);
        h[2] = der2z<C>(pz, k.d2c[2], k.d2[2]);
        h[3] = derm<C>(p, 1, rs, k.dm[0]);
        h[4] = dermz<C>(pz, 1, k.dm[1]);
        h[5] = dermz<C>(pz, rs, k.dm[2]);
    }
}

// The right-hand side of Eqs. A1-A4 at one cell (H = C = K = 0).
template <typename C, typename S>
__device__ __forceinline__ void mhd_rhs_cell(const S *const (*pz)[7], int rs, const MK<C> &k, C *rhs,
                                             C *val) {
    C glr[3], gs[3], gu[3][3], hu[3][6], ga[3][3], ha[3][6];
    field_derivs<C, S, false>(pz[F_LNRHO], rs, k, glr, nullptr);
    field_derivs<C, S, false>(pz[F_SS], rs, k, gs, nullptr);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        field_derivs<C, S, true>(pz[F_UX + c], rs, k, gu[c], hu[c]);
        field_derivs<C, S, true>(pz[F_AX + c], rs, k, ga[c], ha[c]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) val[q] = ld<C>(pz[q][3]);
    const C lnrho = val[F_LNRHO], ss = val[F_SS];
    const C ux = val[F_UX], uy = val[F_UY], uz = val[F_UZ];

    // gu[i][a] = d u_i / d x_a ; hu[i][.] = (xx, yy, zz, xy, xz, yz) of u_i
    const C divu = gu[0][0] + gu[1][1] + gu[2][2];
    C lapu[3], gdivu[3], lapa[3], gdiva[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lapu[c] = hu[c][0] + hu[c][1] + hu[c][2];
        lapa[c] = ha[c][0] + ha[c][1] + ha[c][2];
    }
    // grad(div v)_x = vx_xx + vy_xy + vz_xz, _y = vx_xy + vy_yy + vz_yz, _z = vx_xz + vy_yz + vz_zz
    gdivu[0] = hu[0][0] + hu[1][3] + hu[2][4];
    gdivu[1] = hu[0][3] + hu[1][1] + hu[2][5];
    gdivu[2] = hu[0][4] + hu[1][5] + hu[2][2];
    gdiva[0] = ha[0][0] + ha[1][3] + ha[2][4];
    gdiva[1] = ha[0][3] + ha[1][1] + ha[2][5];
    gdiva[2] = ha[0][4] + ha[1][5] + ha[2][2];

    // traceless rate of shear
    const C third = C(1) / C(3);
    const C sxx = gu[0][0] - third * divu, syy = gu[1][1] - third * divu, szz = gu[2][2] - third * divu;
    const C sxy = C(0.5) * (gu[0][1] + gu[1][0]);
    const C sxz = C(0.5) * (gu[0][2] + gu[2][0]);
    const C syz = C(0.5) * (gu[1][2] + gu[2][1]);
    const C s2 = sxx * sxx + syy * syy + szz * szz + C(2) * (sxy * sxy + sxz * sxz + syz * syz);

    // B = curl A, j = (grad div A - lap A) / mu0
    const C bx = ga[2][1] - ga[1][2], by = ga[0][2] - ga[2][0], bz = ga[1][0] - ga[0][1];
    const C jx = (gdiva[0] - lapa[0]) * k.inv_mu0;
    const C jy = (gdiva[1] - lapa[1]) * k.inv_mu0;
    const C jz = (gdiva[2] - lapa[2]) * k.inv_mu0;

    // closure: rho = exp(lnrho), cs^2 = cs0^2 exp(gamma s/cp + (gamma-1)(lnrho - lnrho0)),
    // T = cs^2 / (cp (gamma - 1))
    const C rho = exp_c<C>(lnrho);
    const C inv_rho = C(1) / rho;
    const C cs2 = k.cs0sq * exp_c<C>(k.gamma * ss * k.inv_cp + (k.gamma - C(1)) * (lnrho - k.lnrho0));
    const C inv_rhoT = k.cp_gm1 * inv_rho / cs2;

    // A1
    rhs[F_LNRHO] = -(ux * glr[0] + uy * glr[1] + uz * glr[2]) - divu;
    // A2
    const C jxb[3] = {jy * bz - jz * by, jz * bx - jx * bz, jx * by - jy * bx};
    const C sg[3] = {sxx * glr[0] + sxy * glr[1] + sxz * glr[2],
                     sxy * glr[0] + syy * glr[1] + syz * glr[2],
                     sxz * glr[0] + syz * glr[1] + szz * glr[2]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C adv = ux * gu[c][0] + uy * gu[c][1] + uz * gu[c][2];
        rhs[F_UX + c] = -adv - cs2 * (gs[c] * k.inv_cp + glr[c]) + jxb[c] * inv_rho +
                        k.nu * (lapu[c] + third * gdivu[c] + C(2) * sg[c]) + k.zeta * gdivu[c];
    }
    // A3
    const C j2 = jx * jx + jy * jy + jz * jz;
    rhs[F_SS] = -(ux * gs[0] + uy * gs[1] + uz * gs[2]) +
                (k.eta * k.mu0 * j2 + C(2) * rho * k.nu * s2 + k.zeta * rho * divu * divu) * inv_rhoT;
    // A4
    rhs[F_AX] = (uy * bz - uz * by) + k.eta * lapa[0];
    rhs[F_AY] = (uz * bx - ux * bz) + k.eta * lapa[1];
    rhs[F_AZ] = (ux * by - uy * bx) + k.eta * lapa[2];
}

template <typename S, typename C, bool KAHAN, int MODE, int TX, int TY, int NSLOT, int ZC>
__global__ void __launch_bounds__(TX *TY, 1)
mhd_kernel(const __grid_constant__ MhdMaps maps, Ptrs8 fout, Ptrs8 wbuf, Ptrs8 kbuf, Ptrs8 rbuf,
           Geom g, MK<C> k, int first, int last, int images, unsigned *err) {
    using Cfg = MhdCfg<S, TX, TY, NSLOT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S *ring = reinterpret_cast<S *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full[NSLOT];

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int64_t x0 = (int64_t)blockIdx.x * TX, y0 = (int64_t)blockIdx.y * TY;
    const int64_t zc0 = (int64_t)blockIdx.z * ZC;
    const int64_t zend = min((int64_t)g.n[2], zc0 + ZC);
    const int nplanes = (int)(zend - zc0) + 2 * R6;
    const int64_t x = x0 + tx, y = y0 + ty;
    const bool active = x < g.n[0] && y < g.n[1];

    if (threadIdx.x == 0) {
        for (int q = 0; q < 8; ++q) tma_prefetch_desc(&maps.m[q]);
        for (int s = 0; s < NSLOT; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    const int bx = (int)(g.off[0] + x0 - Cfg::HX);
    const int by0 = (int)(g.off[1] + y0 - R6);
    const int bz0 = (int)(g.off[2] + zc0 - R6);
    auto issue = [&](int j) {
        const int s = j % NSLOT;
        mbar_arrive_expect_tx(&full[s], 8 * Cfg::BOX_BYTES);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            tma_load_3d(ring + s * Cfg::SLOT_ELEMS + q * Cfg::FIELD_ELEMS, &maps.m[q], &full[s], bx, by0, bz0 + j);
    };
    int issued = 0;
    if (threadIdx.x == 0)
        for (; issued < NSLOT && issued < nplanes; ++issued) issue(issued);

    bool ok = true;
    for (int j = 0; j < 2 * R6; ++j) ok = ok && mbar_wait_bounded(&full[j % NSLOT], (j / NSLOT) & 1);
    bool bad = __syncthreads_or(!ok);

    const int own = (ty + R6) * Cfg::TXP + tx + Cfg::HX;
    const int64_t nxy = g.n[0] * g.n[1];
    for (int m = 0; !bad && m < (int)(zend - zc0); ++m) {
        const int jl = m + 2 * R6;
        ok = mbar_wait_bounded(&full[jl % NSLOT], (jl / NSLOT) & 1);
        if (ok && active) {
            const int64_t z = zc0 + m;
            const S *pz[8][7];
#pragma unroll
            for (int kk = 0; kk < 7; ++kk) {
                const S *base = ring + ((m + kk) % NSLOT) * Cfg::SLOT_ELEMS + own;
#pragma unroll
                for (int q = 0; q < 8; ++q) pz[q][kk] = base + q * Cfg::FIELD_ELEMS;
            }
            C rhs[8], val[8];
            mhd_rhs_cell<C, S>(pz, Cfg::TXP, k, rhs, val);
            const int64_t cell = x + g.n[0] * y + nxy * z;
            if (MODE == 1) {
#pragma unroll
                for (int q = 0; q < 8; ++q) static_cast<C *>(rbuf.p[q])[cell] = rhs[q];
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    S *wq = static_cast<S *>(wbuf.p[q]);
                    C wv = first ? k.dt * rhs[q] : fma(k.alpha, to_c<C>(wq[cell]), k.dt * rhs[q]);
                    if (!last) wq[cell] = to_s<S>(wv);
                    S fnew;
                    if (KAHAN) {
                        S *kq = static_cast<S *>(kbuf.p[q]);
                        const C cq = to_c<C>(kq[cell]);
                        const C yv = k.beta * wv - cq;
                        fnew = to_s<S>(val[q] + yv);
                        kq[cell] = to_s<S>((to_c<C>(fnew) - val[q]) - yv);
                    } else {
                        fnew = to_s<S>(fma(k.beta, wv, val[q]));
                    }
                    store_with_images(static_cast<S *>(fout.p[q]), g, R6, images != 0, x, y, z, fnew);
                }
            }
        }
        bad = __syncthreads_or(!ok);
        // plane j = m (z - 3) is retired: reuse its slot
        if (!bad && threadIdx.x == 0 && issued < nplanes && issued == m + NSLOT) issue(issued++);
    }
    if (bad && threadIdx.x == 0) {
        atomicOr(err, ERR_TIMEOUT);
        for (int j = max(0, issued - NSLOT); j < issued; ++j)
            (void)mbar_wait_bounded(&full[j % NSLOT], (j / NSLOT) & 1, 100000000ull);
    }
}

// ------------------------------------------------------------------ host side

static const double W1[3] = {3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0};
static const double W2C = -49.0 / 18.0;
static const double W2[3] = {3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};
static const double WM[3] = {270.0, -27.0, 2.0};

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
    k.cp_gm1 = (C)c.cp_gm1; k.dt = (C)c.dt; k.alpha = (C)alpha; k.beta = (C)beta;
    return k;
}

static const double RK_A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK_B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

template <typename S, typename C, bool KAHAN, int MODE, int TX, int TY, int NSLOT, int ZC>
static cudaError_t run(int sub, const MhdMaps &maps, const Ptrs8 &fo, const Ptrs8 &w,
                       const Ptrs8 &kc, const Ptrs8 &rhs, const Geom &g, const MhdConst &c,
                       bool images, unsigned *err, cudaStream_t s) {
    using Cfg = MhdCfg<S, TX, TY, NSLOT>;
    auto kern = mhd_kernel<S, C, KAHAN, MODE, TX, TY, NSLOT, ZC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    MK<C> k = make_k<C>(c, RK_A[sub], RK_B[sub]);
    dim3 grid((unsigned)((g.n[0] + TX - 1) / TX), (unsigned)((g.n[1] + TY - 1) / TY),
              (unsigned)((g.n[2] + ZC - 1) / ZC));
    kern<<<grid, TX * TY, Cfg::SMEM, s>>>(maps, fo, w, kc, rhs, g, k, sub == 0 ? 1 : 0,
                                          sub == 2 ? 1 : 0, images ? 1 : 0, err);
    return cudaGetLastError();
}

// Variants per storage type: (TX, TY, NSLOT, ZC).
#define MHD_VARIANTS_F64(X) X(32, 4, 8, 64) X(16, 8, 8, 64)
#define MHD_VARIANTS_F32(X) X(32, 8, 9, 64) X(32, 4, 9, 64)
#define MHD_VARIANTS_BF16(X) X(32, 8, 9, 64) X(32, 4, 10, 64)

int mhd_num_variants(int storage) { (void)storage; return 2; }

const char *mhd_variant_name(int storage, int v) {
    static const char *f64[] = {"tx32_ty4_s8_zc64", "tx16_ty8_s8_zc64"};
    static const char *f32[] = {"tx32_ty8_s9_zc64", "tx32_ty4_s9_zc64"};
    static const char *b16[] = {"tx32_ty8_s9_zc64", "tx32_ty4_s10_zc64"};
    if (v < 0 || v >= 2) return "?";
    return storage == 1 ? f64[v] : storage == 2 ? f32[v] : b16[v];
}

void mhd_box(int storage, int v, int box[3]) {
    int i = 0;
    auto put = [&](int tx, int ty, int hx) {
        if (i++ == v) { box[0] = tx + 2 * hx; box[1] = ty + 2 * R6; box[2] = 1; }
    };
#define X(TX, TY, NS, ZC) put(TX, TY, hx);
    if (storage == 1) { const int hx = 4; MHD_VARIANTS_F64(X) }
    else if (storage == 2) { const int hx = 4; MHD_VARIANTS_F32(X) }
    else { const int hx = 8; MHD_VARIANTS_BF16(X) }
#undef X
}

cudaError_t launch_mhd(int storage, int mode, int sub, const MhdMaps &maps, const Ptrs8 &fo,
                       const Ptrs8 &w, const Ptrs8 &kc, const Ptrs8 &rhs, const Geom &g,
                       const MhdConst &c, bool images, unsigned *err, cudaStream_t s,
                       int variant) {
    int i = 0;
    cudaError_t res = cudaErrorInvalidValue;
#define X(TX, TY, NS, ZC)                                                                   \
    if (i++ == variant) {                                                                   \
        if (mode == 0)                                                                      \
            res = run<S, C, KH, 0, TX, TY, NS, ZC>(sub, maps, fo, w, kc, rhs, g, c, images, err, s); \
        else                                                                                \
            res = run<S, C, KH, 1, TX, TY, NS, ZC>(sub, maps, fo, w, kc, rhs, g, c, images, err, s); \
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

}  // namespace stn
