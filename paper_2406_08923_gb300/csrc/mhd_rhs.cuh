// mhd_rhs.cuh -- the pointwise part of the MHD step: the right-hand side of Eqs. A1-A4
// (phi of Eq. 9) from the derivative quantities of one cell, shared by the per-grid MHD kernels
// and the batched serving kernel (mhd.cu).
#pragma once

#include "internal.h"

namespace stn {

enum { F_LNRHO = 0, F_UX, F_UY, F_UZ, F_AX, F_AY, F_AZ, F_SS };

template <typename C> __device__ __forceinline__ C exp_c(C v);
template <> __device__ __forceinline__ double exp_c<double>(double v) { return exp(v); }
template <> __device__ __forceinline__ float exp_c<float>(float v) { return expf(v); }

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
    const C jx = (d.gdiva[0] - d.lapa[0]) * k.inv_mu0;
    const C jy = (d.gdiva[1] - d.lapa[1]) * k.inv_mu0;
    const C jz = (d.gdiva[2] - d.lapa[2]) * k.inv_mu0;

    const C lnrho = d.val[F_LNRHO], ss = d.val[F_SS];
    const C ux = d.val[F_UX], uy = d.val[F_UY], uz = d.val[F_UZ];
    const C divu = d.gu[0][0] + d.gu[1][1] + d.gu[2][2];
    // traceless rate of shear
    const C third = C(1) / C(3);
    const C sxx = d.gu[0][0] - third * divu, syy = d.gu[1][1] - third * divu, szz = d.gu[2][2] - third * divu;
    const C sxy = C(0.5) * (d.gu[0][1] + d.gu[1][0]);
    const C sxz = C(0.5) * (d.gu[0][2] + d.gu[2][0]);
    const C syz = C(0.5) * (d.gu[1][2] + d.gu[2][1]);
    const C s2 = sxx * sxx + syy * syy + szz * szz + C(2) * (sxy * sxy + sxz * sxz + syz * syz);

    // closure: rho = exp(lnrho), cs^2 = cs0^2 exp(gamma s/cp + (gamma-1)(lnrho - lnrho0)),
    // T = cs^2 / (cp (gamma - 1))
    const C rho = exp_c<C>(lnrho);
    const C inv_rho = C(1) / rho;
    const C cs2 = k.cs0sq * exp_c<C>(k.gamma * ss * k.inv_cp + (k.gamma - C(1)) * (lnrho - k.lnrho0));
    const C inv_rhoT = k.cp_gm1 * inv_rho / cs2;

    // A1
    rhs[F_LNRHO] = -(ux * d.glr[0] + uy * d.glr[1] + uz * d.glr[2]) - divu;
    // A2
    const C jxb[3] = {jy * d.bz - jz * d.by, jz * d.bx - jx * d.bz, jx * d.by - jy * d.bx};
    const C sg[3] = {sxx * d.glr[0] + sxy * d.glr[1] + sxz * d.glr[2],
                     sxy * d.glr[0] + syy * d.glr[1] + syz * d.glr[2],
                     sxz * d.glr[0] + syz * d.glr[1] + szz * d.glr[2]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C adv = ux * d.gu[c][0] + uy * d.gu[c][1] + uz * d.gu[c][2];
        rhs[F_UX + c] = -adv - cs2 * (d.gs[c] * k.inv_cp + d.glr[c]) + jxb[c] * inv_rho +
                        k.nu * (d.lapu[c] + third * d.gdivu[c] + C(2) * sg[c]) + k.zeta * d.gdivu[c];
    }
    // A3
    const C j2 = jx * jx + jy * jy + jz * jz;
    rhs[F_SS] = -(ux * d.gs[0] + uy * d.gs[1] + uz * d.gs[2]) +
                (k.eta * k.mu0 * j2 + C(2) * rho * k.nu * s2 + k.zeta * rho * divu * divu) * inv_rhoT;
    if constexpr (CONDUCT) {
        const C gp = k.gamma * k.inv_cp, gm1 = k.gamma - C(1);
        C gphi2 = C(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const C gphi = gp * d.gs[a] + gm1 * d.glr[a];
            gphi2 = fma(gphi, gphi, gphi2);
        }
        rhs[F_SS] += k.K * inv_rho * (gp * d.laps + gm1 * d.laplr + gphi2);
    }
    // A4
    rhs[F_AX] = (uy * d.bz - uz * d.by) + k.eta * d.lapa[0];
    rhs[F_AY] = (uz * d.bx - ux * d.bz) + k.eta * d.lapa[1];
    rhs[F_AZ] = (ux * d.by - uy * d.bx) + k.eta * d.lapa[2];
}

}  // namespace stn
