// mhd_rhs.cuh -- the pointwise part of the MHD step: the right-hand side of Eqs. A1-A4
// (phi of Eq. 9) from the derivative quantities of one cell, shared by the per-grid MHD kernels
// (mhd.cu) and the batched serving kernel.
//
// Every operation is written out as one IEEE-rounded operation (add, sub, mul, fused
// multiply-add, divide, exp), with nothing left for the compiler to contract, so each variant
// performs exactly the same operations on every cell and all variants of one storage type agree
// bit for bit whatever their tile shape.  A sum that contains a product is written as a fused
// multiply-add, never as a rounded product fed to an add or subtract: that keeps the sequence
// valid for code generators that fuse such pairs on their own (measured on GB300 for packed
// FP32x2 multiplies, which are fused into a following packed add even with explicit rounding).
#pragma once

#include "internal.h"

namespace stn {

enum { F_LNRHO = 0, F_UX, F_UY, F_UZ, F_AX, F_AY, F_AZ, F_SS };

__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double dvd(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double ex(double a) { return exp(a); }

__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float dvd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float ex(float a) { return expf(a); }

// Derivative quantities of one cell (6th-order stencils, Sec. 3.3): values, grad lnrho,
// grad s, grad u, lap u, grad div u, B = curl A, lap A, grad div A, and (K != 0 only) lap lnrho,
// lap s.
template <typename C> struct MhdDerivs {
    C val[8];
    C glr[3], gs[3];
    C gu[3][3], lapu[3], gdivu[3];
    C bx, by, bz, lapa[3], gdiva[3];
    C laplr, laps;
};

// The right-hand side of Eqs. A1-A4 (H = C = 0).  The conduction term of A3 with constant K
// uses T = T0 exp(phi), phi = gamma s/cp + (gamma-1)(lnrho - lnrho0):
// div(K grad T)/(rho T) = (K/rho)(lap phi + |grad phi|^2).  It is compiled in only for
// CONDUCT (launches with K != 0), so the K = 0 kernels carry none of its registers.
template <bool CONDUCT, typename C>
__device__ __forceinline__ void mhd_rhs_assemble(const MhdDerivs<C> &d, const MK<C> &k, C *rhs) {
    // j = (grad div A - lap A) / mu0
    const C jx = mul(sub(d.gdiva[0], d.lapa[0]), k.inv_mu0);
    const C jy = mul(sub(d.gdiva[1], d.lapa[1]), k.inv_mu0);
    const C jz = mul(sub(d.gdiva[2], d.lapa[2]), k.inv_mu0);

    const C lnrho = d.val[F_LNRHO], ss = d.val[F_SS];
    const C ux = d.val[F_UX], uy = d.val[F_UY], uz = d.val[F_UZ];
    const C divu = add(add(d.gu[0][0], d.gu[1][1]), d.gu[2][2]);
    // traceless rate of shear S and S:S
    const C sxx = fmad(k.mthird, divu, d.gu[0][0]);
    const C syy = fmad(k.mthird, divu, d.gu[1][1]);
    const C szz = fmad(k.mthird, divu, d.gu[2][2]);
    const C sxy = mul(k.half, add(d.gu[0][1], d.gu[1][0]));
    const C sxz = mul(k.half, add(d.gu[0][2], d.gu[2][0]));
    const C syz = mul(k.half, add(d.gu[1][2], d.gu[2][1]));
    C s2 = fmad(szz, szz, fmad(syy, syy, mul(sxx, sxx)));
    const C so = fmad(syz, syz, fmad(sxz, sxz, mul(sxy, sxy)));
    s2 = fmad(k.two, so, s2);

    // closure: rho = exp(lnrho), cs^2 = cs0^2 exp(gamma s/cp + (gamma-1)(lnrho - lnrho0)),
    // T = cs^2 / (cp (gamma - 1))
    const C rho = ex(lnrho);
    const C inv_rho = dvd(k.one, rho);
    const C cs2 = mul(k.cs0sq, ex(fmad(k.gcp, ss, mul(k.gm1, sub(lnrho, k.lnrho0)))));
    const C inv_rhoT = dvd(mul(k.cp_gm1, inv_rho), cs2);

    // A1: -u . grad lnrho - div u
    const C ug = fmad(uz, d.glr[2], fmad(uy, d.glr[1], mul(ux, d.glr[0])));
    rhs[F_LNRHO] = mul(k.mone, add(ug, divu));
    // A2: -(u . grad) u - cs^2 grad(s/cp + lnrho) + j x B / rho
    //     + nu (lap u + grad div u / 3 + 2 S . grad lnrho) + zeta grad div u
    // cross products a x B as a_i B_j + a_j (-B_i), with -B formed once (exact)
    const C mbx = mul(k.mone, d.bx), mby = mul(k.mone, d.by), mbz = mul(k.mone, d.bz);
    const C jxb[3] = {fmad(jy, d.bz, mul(jz, mby)), fmad(jz, d.bx, mul(jx, mbz)), fmad(jx, d.by, mul(jy, mbx))};
    const C sg[3] = {fmad(sxz, d.glr[2], fmad(sxy, d.glr[1], mul(sxx, d.glr[0]))),
                     fmad(syz, d.glr[2], fmad(syy, d.glr[1], mul(sxy, d.glr[0]))),
                     fmad(szz, d.glr[2], fmad(syz, d.glr[1], mul(sxz, d.glr[0])))};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C adv = fmad(uz, d.gu[c][2], fmad(uy, d.gu[c][1], mul(ux, d.gu[c][0])));
        // advection + pressure gradient: adv + cs^2 (grad s / cp + grad lnrho)
        const C ap = fmad(cs2, fmad(d.gs[c], k.inv_cp, d.glr[c]), adv);
        const C visc = fmad(k.two, sg[c], fmad(k.third, d.gdivu[c], d.lapu[c]));
        C r = fmad(jxb[c], inv_rho, mul(k.mone, ap));
        r = fmad(k.nu, visc, r);
        rhs[F_UX + c] = fmad(k.zeta, d.gdivu[c], r);
    }
    // A3: -u . grad s + (eta mu0 j^2 + 2 rho nu S:S + zeta rho (div u)^2) / (rho T)
    const C j2 = fmad(jz, jz, fmad(jy, jy, mul(jx, jx)));
    C heat = mul(k.etamu0, j2);
    heat = fmad(mul(k.two_nu, rho), s2, heat);
    heat = fmad(mul(mul(k.zeta, rho), divu), divu, heat);
    const C us = fmad(uz, d.gs[2], fmad(uy, d.gs[1], mul(ux, d.gs[0])));
    rhs[F_SS] = fmad(heat, inv_rhoT, mul(k.mone, us));
    if constexpr (CONDUCT) {
        const C gphi0 = fmad(k.gcp, d.gs[0], mul(k.gm1, d.glr[0]));
        const C gphi1 = fmad(k.gcp, d.gs[1], mul(k.gm1, d.glr[1]));
        const C gphi2c = fmad(k.gcp, d.gs[2], mul(k.gm1, d.glr[2]));
        const C gphi2 = fmad(gphi2c, gphi2c, fmad(gphi1, gphi1, mul(gphi0, gphi0)));
        const C lapphi = fmad(k.gcp, d.laps, mul(k.gm1, d.laplr));
        rhs[F_SS] = fmad(mul(k.K, inv_rho), add(lapphi, gphi2), rhs[F_SS]);
    }
    // A4: u x B + eta lap A
    rhs[F_AX] = fmad(k.eta, d.lapa[0], fmad(uy, d.bz, mul(uz, mby)));
    rhs[F_AY] = fmad(k.eta, d.lapa[1], fmad(uz, d.bx, mul(ux, mbz)));
    rhs[F_AZ] = fmad(k.eta, d.lapa[2], fmad(ux, d.by, mul(uy, mbx)));
}

// Ring geometry of the z-streaming MHD kernels: a TX x TY tile of cells, every plane of the 8
// fields staged with a halo of HX columns (16 bytes, at least the radius) and R6 rows.
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
    static_assert((NSLOT & (NSLOT - 1)) == 0, "ring depth is a power of two");
};

// The derivative stage (gamma = A B, Eq. 8) and the right-hand side at one cell (or one pair of
// cells): the derivatives are evaluated field by field, only those some term uses (lnrho and s:
// gradients, plus Laplacians when K != 0; u: gradient and Hessian; A: the off-diagonal first
// derivatives for B = curl A, and the Hessian), folded at once into the quantities the RHS
// needs, then assembled by mhd_rhs_assemble.  The window W supplies the cell values and the
// 6th-order first, second and mixed differences (weights pre-scaled by the grid spacing).
template <bool CONDUCT, typename C, typename W>
__device__ __forceinline__ void mhd_rhs_cell(const W &w, const MK<C> &k, C *rhs, C *val) {
    MhdDerivs<C> d;
#pragma unroll
    for (int q = 0; q < 8; ++q) d.val[q] = w.val(q);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d.glr[a] = w.d1(F_LNRHO, a, k.d1[a]);
        d.gs[a] = w.d1(F_SS, a, k.d1[a]);
    }
    if constexpr (CONDUCT) {
        d.laplr = add(add(w.d2(F_LNRHO, 0, k.d2c[0], k.d2[0]), w.d2(F_LNRHO, 1, k.d2c[1], k.d2[1])),
                      w.d2(F_LNRHO, 2, k.d2c[2], k.d2[2]));
        d.laps = add(add(w.d2(F_SS, 0, k.d2c[0], k.d2[0]), w.d2(F_SS, 1, k.d2c[1], k.d2[1])),
                     w.d2(F_SS, 2, k.d2c[2], k.d2[2]));
    }
    // velocity: gu[i][a] = d u_i / d x_a; lap u; grad div u accumulated over the components
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int q = F_UX + c;
#pragma unroll
        for (int a = 0; a < 3; ++a) d.gu[c][a] = w.d1(q, a, k.d1[a]);
        const C hxx = w.d2(q, 0, k.d2c[0], k.d2[0]);
        const C hyy = w.d2(q, 1, k.d2c[1], k.d2[1]);
        const C hzz = w.d2(q, 2, k.d2c[2], k.d2[2]);
        const C hxy = w.dmix(q, 0, k.dm[0]);
        const C hxz = w.dmix(q, 1, k.dm[1]);
        const C hyz = w.dmix(q, 2, k.dm[2]);
        d.lapu[c] = add(add(hxx, hyy), hzz);
        // grad(div u)_a = sum_c d_a d_c u_c
        const C hc[3] = {c == 0 ? hxx : c == 1 ? hxy : hxz, c == 0 ? hxy : c == 1 ? hyy : hyz,
                         c == 0 ? hxz : c == 1 ? hyz : hzz};
#pragma unroll
        for (int a = 0; a < 3; ++a) d.gdivu[a] = c == 0 ? hc[a] : add(d.gdivu[a], hc[a]);
    }
    // vector potential: B = curl A, j = (grad div A - lap A) / mu0 (in mhd_rhs_assemble)
    {
        const C ax_y = w.d1(F_AX, 1, k.d1[1]), ax_z = w.d1(F_AX, 2, k.d1[2]);
        const C ay_x = w.d1(F_AY, 0, k.d1[0]), ay_z = w.d1(F_AY, 2, k.d1[2]);
        const C az_x = w.d1(F_AZ, 0, k.d1[0]), az_y = w.d1(F_AZ, 1, k.d1[1]);
        d.bx = sub(az_y, ay_z);
        d.by = sub(ax_z, az_x);
        d.bz = sub(ay_x, ax_y);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int q = F_AX + c;
        const C hxx = w.d2(q, 0, k.d2c[0], k.d2[0]);
        const C hyy = w.d2(q, 1, k.d2c[1], k.d2[1]);
        const C hzz = w.d2(q, 2, k.d2c[2], k.d2[2]);
        const C hxy = w.dmix(q, 0, k.dm[0]);
        const C hxz = w.dmix(q, 1, k.dm[1]);
        const C hyz = w.dmix(q, 2, k.dm[2]);
        d.lapa[c] = add(add(hxx, hyy), hzz);
        const C hc[3] = {c == 0 ? hxx : c == 1 ? hxy : hxz, c == 0 ? hxy : c == 1 ? hyy : hyz,
                         c == 0 ? hxz : c == 1 ? hyz : hzz};
#pragma unroll
        for (int a = 0; a < 3; ++a) d.gdiva[a] = c == 0 ? hc[a] : add(d.gdiva[a], hc[a]);
    }
    mhd_rhs_assemble<CONDUCT>(d, k, rhs);
#pragma unroll
    for (int q = 0; q < 8; ++q) val[q] = d.val[q];
}

// The 2N-storage RK3 update of one value (w <- alpha_s w + dt RHS; f <- f + beta_s w) in the
// compute type.  With Kahan compensation (FP32/BF16 storage) the stored term kn holds the
// NEGATED compensation -c, so that y = beta w - c is one fused multiply-add: y = beta w + kn,
// f' = f + y, kn' = y - (f' - f) (= -((f' - f) - y) exactly).  `rt` rounds to the storage
// type and back.
template <bool KAHAN, typename C, typename R>
__device__ __forceinline__ void rk_update(const MK<C> &k, bool first, C rhs, C wold, C kn, C val, C &wnew, C &fnew,
                                          C &knew, R rt) {
    const C dtr = mul(k.dt, rhs);
    wnew = first ? dtr : fmad(k.alpha, wold, dtr);
    if (KAHAN) {
        const C y = fmad(k.beta, wnew, kn);
        fnew = rt(add(val, y));
        knew = sub(y, sub(fnew, val));
    } else {
        fnew = rt(fmad(k.beta, wnew, val));
        knew = kn;
    }
}

}  // namespace stn
