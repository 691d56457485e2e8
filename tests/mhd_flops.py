"""Algorithmic floating-point work of one MHD cell-substep (Sec. 3.3 differences, Eqs. A1-A4,
the 2N-storage RK3 update), counted by evaluating it once with an operation-counting number.

Test infrastructure: the count is the numerator of the MHD roofline in the benchmark, and
tests/test_mhd_flops.py checks that this evaluation reproduces the oracle's right-hand side
and RK update at the same cell, so the count describes a correct evaluation of the method.

What is counted is the work the equations require, in the cheapest form of each stencil
that the 6th-order weights allow, with nothing a term does not use:

* 1st derivative (antisymmetric weights): 3 differences, 3 products, 2 sums = 8 flops.
* 2nd derivative (symmetric weights): 3 pair sums, 4 products, 3 sums = 10 flops.
* mixed derivative (diagonal form): per offset a, D(a) = (f(a,a) + f(-a,-a)) - (f(a,-a) +
  f(-a,a)) = 3 flops; then 3 products and 2 sums = 14 flops.
* Derivatives required by A1-A4 with H = C = K = 0: the gradients of lnrho and s (6), the
  velocity gradient (9), the six off-diagonal derivatives of A that B = curl A needs, and the
  Hessians of u and A (18 second and 18 mixed derivatives): 21 x 8 + 18 x 10 + 18 x 14 = 600.
* The right-hand side of A1-A4 as written (the zeta terms included), with 1/rho and
  1/(rho T) formed once: products, sums and divisions, each one flop; exp separately.
* The RK update of 8 fields: w <- alpha_s w + dt RHS (1 product on the first substep, where
  w starts at zero, 3 flops otherwise) and f <- f + beta_s w (2 flops).

Stencil weights scaled by the grid spacing (1/dx, 1/dx^2, 1/(720 dx dy)) are per-grid
constants, not per-cell work.  A fused multiply-add counts as two flops.
"""
from __future__ import annotations

import math

import numpy as np


class Count:
    """Operation counters shared by every Num of one evaluation."""

    def __init__(self):
        self.add = self.mul = self.div = self.exp = 0

    @property
    def flops(self):
        return self.add + self.mul + self.div


class Num:
    """A double that counts the arithmetic done with it (constants are plain floats)."""

    __slots__ = ("v", "c")

    def __init__(self, v, c):
        self.v, self.c = float(v), c

    def _o(self, other):
        return other.v if isinstance(other, Num) else float(other)

    def __add__(self, o):
        self.c.add += 1
        return Num(self.v + self._o(o), self.c)

    __radd__ = __add__

    def __sub__(self, o):
        self.c.add += 1
        return Num(self.v - self._o(o), self.c)

    def __rsub__(self, o):
        self.c.add += 1
        return Num(self._o(o) - self.v, self.c)

    def __mul__(self, o):
        self.c.mul += 1
        return Num(self.v * self._o(o), self.c)

    __rmul__ = __mul__

    def __truediv__(self, o):
        self.c.div += 1
        return Num(self.v / self._o(o), self.c)

    def __rtruediv__(self, o):
        self.c.div += 1
        return Num(self._o(o) / self.v, self.c)

    def __neg__(self):  # a sign flip folds into the next sum
        return Num(-self.v, self.c)


def nexp(x: Num) -> Num:
    x.c.exp += 1
    return Num(math.exp(x.v), x.c)


# textbook 6th-order weights (Fornberg 1988): d1 on offsets 1..3, d2 centre and offsets 1..3,
# mixed diagonal form per offset
W1 = (3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0)
W2C, W2 = -49.0 / 18.0, (3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0)
WM = (270.0, -27.0, 2.0)


def cell_substep(fhat, cell, h, par, w, substep):
    """RHS of Eqs. A1-A4 and one 2N-storage RK3 substep at one cell.

    fhat: 8 padded boxes (z, y, x) with a halo of 3; cell = (k, j, i) interior indices;
    h = (dx, dy, dz); par: dict of cs0, gamma, cp, lnrho0, nu, eta, zeta, mu0, dt;
    w: the 8 RK registers at the cell (floats).  Returns (rhs, f_new, w_new, Count)."""
    cnt = Count()
    k, j, i = (c + 3 for c in cell)

    def at(q, dx=0, dy=0, dz=0):
        return Num(fhat[q][k + dz, j + dy, i + dx], cnt)

    def off(axis, s):
        return {0: (s, 0, 0), 1: (0, s, 0), 2: (0, 0, s)}[axis]

    def d1(q, a):
        c = [W1[m] / h[a] for m in range(3)]
        t = [at(q, *off(a, m + 1)) - at(q, *off(a, -m - 1)) for m in range(3)]
        return c[0] * t[0] + c[1] * t[1] + c[2] * t[2]

    def d2(q, a):
        c0, c = W2C / h[a] ** 2, [W2[m] / h[a] ** 2 for m in range(3)]
        t = [at(q, *off(a, m + 1)) + at(q, *off(a, -m - 1)) for m in range(3)]
        return c0 * at(q) + c[0] * t[0] + c[1] * t[1] + c[2] * t[2]

    def dmix(q, a, b):
        def f(sa, sb):
            d = [0, 0, 0]
            d[a] += sa
            d[b] += sb
            return at(q, *d)

        m = [WM[s] / (720.0 * h[a] * h[b]) for s in range(3)]
        t = [(f(s, s) + f(-s, -s)) - (f(s, -s) + f(-s, s)) for s in (1, 2, 3)]
        return m[0] * t[0] + m[1] * t[1] + m[2] * t[2]

    LNRHO, UX, AX, SS = 0, 1, 4, 7
    val = [at(q) for q in range(8)]
    glr = [d1(LNRHO, a) for a in range(3)]
    gs = [d1(SS, a) for a in range(3)]
    gu = [[d1(UX + c, a) for a in range(3)] for c in range(3)]

    def hessian(q):
        hd = [d2(q, a) for a in range(3)]
        hxy, hxz, hyz = dmix(q, 0, 1), dmix(q, 0, 2), dmix(q, 1, 2)
        return [[hd[0], hxy, hxz], [hxy, hd[1], hyz], [hxz, hyz, hd[2]]]

    Hu = [hessian(UX + c) for c in range(3)]
    lapu = [Hu[c][0][0] + Hu[c][1][1] + Hu[c][2][2] for c in range(3)]
    gdivu = [Hu[0][c][0] + Hu[1][c][1] + Hu[2][c][2] for c in range(3)]
    # B = curl A from the off-diagonal first derivatives of A
    ax_y, ax_z = d1(AX, 1), d1(AX, 2)
    ay_x, ay_z = d1(AX + 1, 0), d1(AX + 1, 2)
    az_x, az_y = d1(AX + 2, 0), d1(AX + 2, 1)
    B = [az_y - ay_z, ax_z - az_x, ay_x - ax_y]
    HA = [hessian(AX + c) for c in range(3)]
    lapa = [HA[c][0][0] + HA[c][1][1] + HA[c][2][2] for c in range(3)]
    gdiva = [HA[0][c][0] + HA[1][c][1] + HA[2][c][2] for c in range(3)]

    cs0, gam, cp, lnrho0 = par["cs0"], par["gamma"], par["cp"], par["lnrho0"]
    nu, eta, zeta, mu0, dt = par["nu"], par["eta"], par["zeta"], par["mu0"], par["dt"]
    jj = [(gdiva[c] - lapa[c]) * (1.0 / mu0) for c in range(3)]
    lnrho, ss, u = val[LNRHO], val[SS], val[UX:UX + 3]
    divu = gu[0][0] + gu[1][1] + gu[2][2]
    third_divu = divu * (1.0 / 3.0)
    S = [[None] * 3 for _ in range(3)]
    for a in range(3):
        S[a][a] = gu[a][a] - third_divu
    for a, b in ((0, 1), (0, 2), (1, 2)):
        S[a][b] = S[b][a] = 0.5 * (gu[a][b] + gu[b][a])
    s2 = (S[0][0] * S[0][0] + S[1][1] * S[1][1] + S[2][2] * S[2][2]
          + 2.0 * (S[0][1] * S[0][1] + S[0][2] * S[0][2] + S[1][2] * S[1][2]))
    rho = nexp(lnrho)
    inv_rho = 1.0 / rho
    cs2 = (cs0 * cs0) * nexp((gam / cp) * ss + (gam - 1.0) * (lnrho - lnrho0))
    inv_rhoT = (cp * (gam - 1.0)) * inv_rho / cs2  # 1/(rho T), T = cs2 / (cp (gamma - 1))

    rhs = [None] * 8
    # A1
    rhs[LNRHO] = -(u[0] * glr[0] + u[1] * glr[1] + u[2] * glr[2]) - divu
    # A2
    jxb = [jj[1] * B[2] - jj[2] * B[1], jj[2] * B[0] - jj[0] * B[2], jj[0] * B[1] - jj[1] * B[0]]
    for c in range(3):
        adv = u[0] * gu[c][0] + u[1] * gu[c][1] + u[2] * gu[c][2]
        sg = S[c][0] * glr[0] + S[c][1] * glr[1] + S[c][2] * glr[2]
        rhs[UX + c] = (-adv - cs2 * (gs[c] * (1.0 / cp) + glr[c]) + jxb[c] * inv_rho
                       + nu * (lapu[c] + gdivu[c] * (1.0 / 3.0) + 2.0 * sg) + zeta * gdivu[c])
    # A3 (H = C = K = 0)
    j2 = jj[0] * jj[0] + jj[1] * jj[1] + jj[2] * jj[2]
    rhs[SS] = (-(u[0] * gs[0] + u[1] * gs[1] + u[2] * gs[2])
               + ((eta * mu0) * j2 + (2.0 * nu) * rho * s2 + zeta * rho * divu * divu) * inv_rhoT)
    # A4
    uxb = [u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2], u[0] * B[1] - u[1] * B[0]]
    for c in range(3):
        rhs[AX + c] = uxb[c] + eta * lapa[c]

    # Williamson 2N-storage RK3 substep
    alpha = (0.0, -5.0 / 9.0, -153.0 / 128.0)[substep]
    beta = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)[substep]
    w_new, f_new = [], []
    for q in range(8):
        wq = dt * rhs[q] if substep == 0 else alpha * Num(w[q], cnt) + dt * rhs[q]
        w_new.append(wq)
        f_new.append(val[q] + beta * wq)
    return [r.v for r in rhs], [f.v for f in f_new], [x.v for x in w_new], cnt


def flops_per_cell_substep(rng_seed=0):
    """(flops per cell-substep averaged over the 3 substeps, exps per cell-substep, detail)."""
    rng = np.random.default_rng(rng_seed)
    fhat = [rng.uniform(-0.1, 0.1, size=(7, 7, 7)) for _ in range(8)]
    h = (0.3, 0.4, 0.5)
    par = dict(cs0=1.0, gamma=5.0 / 3.0, cp=1.0, lnrho0=0.0, nu=5e-3, eta=5e-3, zeta=1e-3, mu0=1.0, dt=0.01)
    per = []
    for s in range(3):
        *_, c = cell_substep(fhat, (0, 0, 0), h, par, [0.1] * 8, s)
        per.append((c.flops, c.exp, c.add, c.mul, c.div))
    avg = sum(p[0] for p in per) / 3.0
    return avg, per[0][1], per


if __name__ == "__main__":
    avg, nexp_, per = flops_per_cell_substep()
    print(f"flops per cell-substep (mean over substeps): {avg:.2f}; exp per cell-substep: {nexp_}")
    for s, p in enumerate(per):
        print(f"  substep {s}: {p[0]} flops ({p[2]} add/sub, {p[3]} mul, {p[4]} div)")
