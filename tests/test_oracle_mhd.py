"""Pins of the oracle's MHD right-hand side (Eqs. A1-A4) and RK3 step (Sec. 3.3).

Each case chooses fields for which every derivative is a closed form (single sine modes, so
each stencil returns its discrete Fourier symbol times the mode), so the expected RHS follows
from Eqs. A1-A4 by hand.  Together the cases exercise every term with its sign and constant:
advection, the pressure term with cs^2(lnrho, s), the Lorentz force j x B / rho with
j = grad div A - lap A, viscosity with the 1/3 grad div u and 2 S.grad lnrho terms, bulk
viscosity, viscous/ohmic/bulk heating over rho T, and the induction term u x B + eta lap A.

RK3: for a force-free (Beltrami) vector potential with u = 0 the system is linear in A, and
one step multiplies A by the 3-stage, 3rd-order stability polynomial 1 + z + z^2/2 + z^3/6
with z = eta lam2 dt.
"""
import numpy as np
import pytest

import oracle
from oracle import MhdParams
from paper_2406_08923_gb300 import synth
from symbols import grid, lam1, lam2, mu

N = 16
LNRHO, UX, UY, UZ, AX, AY, AZ, SS = range(8)


def _par(**kw):
    base = dict(cs0=1.3, gamma=5.0 / 3.0, cp=1.7, lnrho0=0.3, nu=0.02, eta=0.03, zeta=0.05, mu0=1.5)
    base.update(kw)
    return MhdParams.for_grid(N, **base)


def _temp(p, lnrho, ss):
    cs2 = p.cs0 ** 2 * np.exp(p.gamma * ss / p.cp + (p.gamma - 1) * (lnrho - p.lnrho0))
    return cs2, cs2 / (p.cp * (p.gamma - 1))


def _check(got, exp, tol=1e-12):
    for q in range(8):
        e = np.broadcast_to(exp[q], got[q].shape)
        np.testing.assert_allclose(got[q], e, rtol=0, atol=tol, err_msg=f"field {q}")


def test_uniform_state_has_zero_rhs():
    p = _par()
    f = np.empty((8, N, N, N))
    for q, v in enumerate((0.2, 0.5, -0.3, 0.1, 1.0, -2.0, 0.7, 0.4)):
        f[q] = v
    rhs = oracle.mhd_rhs(f, p)
    assert np.abs(rhs).max() < 1e-13


def test_sound_wave_pressure_term():
    p = _par()
    (Z, Y, X), h = grid(N)
    k, eps = 2, 1e-2
    f = np.zeros((8, N, N, N))
    f[LNRHO] = eps * np.sin(k * X)
    cs2, _ = _temp(p, f[LNRHO], 0.0)
    exp = np.zeros_like(f)
    exp[UX] = -cs2 * lam1(k, h) * eps * np.cos(k * X)
    _check(oracle.mhd_rhs(f, p), exp)


def test_entropy_gradient_pressure_term():
    p = _par()
    (Z, Y, X), h = grid(N)
    k, eps = 3, 2e-2
    f = np.zeros((8, N, N, N))
    f[SS] = eps * np.sin(k * Y)
    cs2, _ = _temp(p, 0.0, f[SS])
    exp = np.zeros_like(f)
    exp[UY] = -cs2 * lam1(k, h) * eps * np.cos(k * Y) / p.cp
    _check(oracle.mhd_rhs(f, p), exp)


def test_shear_with_density_gradient():
    p = _par()
    (Z, Y, X), h = grid(N)
    k, q, eps, dl = 2, 3, 1e-2, 3e-2
    f = np.zeros((8, N, N, N))
    f[UY] = eps * np.sin(k * X)
    f[LNRHO] = dl * np.sin(q * Y)
    g = lam1(k, h) * eps * np.cos(k * X)     # d uy / dx
    G = lam1(q, h) * dl * np.cos(q * Y)      # d lnrho / dy
    cs2, T = _temp(p, f[LNRHO], 0.0)
    exp = np.zeros_like(f)
    exp[LNRHO] = -f[UY] * G
    exp[UX] = p.nu * g * G                   # nu * 2 S_xy dlnrho/dy, S_xy = g/2
    exp[UY] = -cs2 * G + p.nu * lam2(k, h) * f[UY]
    exp[SS] = p.nu * g * g / T               # 2 rho nu S:S / (rho T), S:S = g^2/2
    _check(oracle.mhd_rhs(f, p), exp)


def test_compressive_flow_and_bulk_viscosity():
    p = _par()
    (Z, Y, X), h = grid(N)
    k, eps = 2, 1e-2
    f = np.zeros((8, N, N, N))
    f[UX] = eps * np.sin(k * X)
    g = lam1(k, h) * eps * np.cos(k * X)     # div u
    l2 = lam2(k, h) * f[UX]                  # d2 ux / dx2 = d/dx div u
    cs2, T = _temp(p, 0.0, 0.0)
    exp = np.zeros_like(f)
    exp[LNRHO] = -g
    exp[UX] = -f[UX] * g + p.nu * (l2 + l2 / 3.0) + p.zeta * l2
    exp[SS] = (2 * p.nu * (2.0 / 3.0) * g * g + p.zeta * g * g) / T
    _check(oracle.mhd_rhs(f, p), exp)


def test_grad_div_u_uses_mixed_derivatives():
    p = _par()
    (Z, Y, X), h = grid(N)
    k, eps = 2, 1e-2
    th = k * (X + Y)
    f = np.zeros((8, N, N, N))
    f[UX] = eps * np.sin(th)
    dxu = lam1(k, h) * eps * np.cos(th)
    dyu = dxu
    l2 = lam2(k, h) * f[UX]
    m = mu(k, k, h, h) * f[UX]
    cs2, T = _temp(p, 0.0, 0.0)
    exp = np.zeros_like(f)
    exp[LNRHO] = -dxu
    exp[UX] = -f[UX] * dxu + p.nu * (2 * l2 + l2 / 3.0) + p.zeta * l2
    exp[UY] = p.nu * m / 3.0 + p.zeta * m
    # S: Sxx = dxu - dxu/3, Syy = Szz = -dxu/3, Sxy = dyu/2
    SS2 = (2 * dxu / 3) ** 2 + 2 * (dxu / 3) ** 2 + 2 * (dyu / 2) ** 2
    exp[SS] = (2 * p.nu * SS2 + p.zeta * dxu * dxu) / T
    _check(oracle.mhd_rhs(f, p), exp)


def test_lorentz_force_ohmic_heating_and_induction():
    p = _par()
    (Z, Y, X), h = grid(N)
    k, eps, U, l0 = 3, 1e-2, 0.4, 0.2
    f = np.zeros((8, N, N, N))
    f[AZ] = eps * np.sin(k * X)
    f[UX] = U
    f[LNRHO] = l0
    By = -lam1(k, h) * eps * np.cos(k * X)
    jz = -lam2(k, h) * f[AZ] / p.mu0
    rho = np.exp(l0)
    cs2, T = _temp(p, l0, 0.0)
    exp = np.zeros_like(f)
    exp[UX] = -jz * By / rho                 # (j x B)_x = jy Bz - jz By
    exp[SS] = p.eta * p.mu0 * jz * jz / (rho * T)
    exp[AZ] = U * By + p.eta * lam2(k, h) * f[AZ]   # (u x B)_z = ux By - uy Bx
    _check(oracle.mhd_rhs(f, p), exp)


def test_grad_div_A_in_current():
    p = _par()
    (Z, Y, X), h = grid(N)
    k, eps = 2, 1e-2
    th = k * (X + Y)
    f = np.zeros((8, N, N, N))
    f[AX] = eps * np.sin(th)
    l2 = lam2(k, h) * f[AX]
    m = mu(k, k, h, h) * f[AX]
    jx = (l2 - 2 * l2) / p.mu0               # grad div A - lap A
    jy = m / p.mu0
    Bz = -lam1(k, h) * eps * np.cos(th)      # dAy/dx - dAx/dy
    _, T = _temp(p, 0.0, 0.0)
    exp = np.zeros_like(f)
    exp[UX] = jy * Bz
    exp[UY] = -jx * Bz
    exp[SS] = p.eta * p.mu0 * (jx * jx + jy * jy) / T
    exp[AX] = p.eta * 2 * l2
    _check(oracle.mhd_rhs(f, p), exp)


def test_grid_spacing_per_axis_on_a_non_cubic_grid():
    # (nz, ny, nx) = (12, 16, 20): every axis has its own spacing 2 pi / n_axis, so a density
    # mode along x and one along z each give the pressure force with their own symbol.
    nz, ny, nx = 12, 16, 20
    base = dict(cs0=1.3, gamma=5.0 / 3.0, cp=1.7, lnrho0=0.3, nu=0.02, eta=0.03, zeta=0.05, mu0=1.5)
    p = MhdParams.for_grid((nz, ny, nx), **base)
    Z, Y, X = np.meshgrid(*(2 * np.pi * np.arange(m) / m for m in (nz, ny, nx)), indexing="ij")
    kx, kz, eps = 3, 2, 1e-2
    f = np.zeros((8, nz, ny, nx))
    f[LNRHO] = eps * np.sin(kx * X) + eps * np.sin(kz * Z)
    cs2, _ = _temp(p, f[LNRHO], 0.0)
    exp = np.zeros_like(f)
    exp[UX] = -cs2 * lam1(kx, 2 * np.pi / nx) * eps * np.cos(kx * X)
    exp[UZ] = -cs2 * lam1(kz, 2 * np.pi / nz) * eps * np.cos(kz * Z)
    _check(oracle.mhd_rhs(f, p), exp)


def test_entropy_advection_by_a_uniform_flow():
    # u uniform, lnrho uniform, s = eps sin(k x): A3 reduces to ds/dt = -u . grad s (no shear, no
    # current), A2 to the entropy part of the pressure term, A1 and A4 to zero.
    p = _par()
    (Z, Y, X), h = grid(N)
    k, eps, U, l0 = 2, 2e-2, (0.4, -0.3, 0.25), 0.1
    f = np.zeros((8, N, N, N))
    f[LNRHO] = l0
    f[UX], f[UY], f[UZ] = U
    f[SS] = eps * np.sin(k * X)
    dsdx = lam1(k, h) * eps * np.cos(k * X)
    cs2, _ = _temp(p, l0, f[SS])
    exp = np.zeros_like(f)
    exp[UX] = -cs2 * dsdx / p.cp
    exp[SS] = -U[0] * dsdx
    _check(oracle.mhd_rhs(f, p), exp)


def test_lorentz_force_and_induction_every_component():
    # A = (a sin(q z), c sin(m x), b sin(k x)) is divergence-free, so j = -lap A / mu0 and
    # B = curl A = (0, dAx/dz - dAz/dx, dAy/dx); with a uniform u every component of u x B and
    # j x B is nonzero somewhere, so each is checked with its own sign.
    p = _par()
    (Z, Y, X), h = grid(N)
    (q, a), (m, c), (k, b) = (2, 1e-2), (3, -2e-2), (1, 1.5e-2)
    U, l0 = (0.3, -0.45, 0.2), -0.15
    f = np.zeros((8, N, N, N))
    f[LNRHO] = l0
    f[UX], f[UY], f[UZ] = U
    f[AX] = a * np.sin(q * Z)
    f[AY] = c * np.sin(m * X)
    f[AZ] = b * np.sin(k * X)
    lapA = (lam2(q, h) * f[AX], lam2(m, h) * f[AY], lam2(k, h) * f[AZ])
    j = [-v / p.mu0 for v in lapA]
    B = (np.zeros_like(X),
         lam1(q, h) * a * np.cos(q * Z) - lam1(k, h) * b * np.cos(k * X),
         lam1(m, h) * c * np.cos(m * X))
    uxB = (U[1] * B[2] - U[2] * B[1], U[2] * B[0] - U[0] * B[2], U[0] * B[1] - U[1] * B[0])
    jxB = (j[1] * B[2] - j[2] * B[1], j[2] * B[0] - j[0] * B[2], j[0] * B[1] - j[1] * B[0])
    rho = np.exp(l0)
    _, T = _temp(p, l0, 0.0)
    exp = np.zeros_like(f)
    for cidx in range(3):
        exp[UX + cidx] = jxB[cidx] / rho
        exp[AX + cidx] = uxB[cidx] + p.eta * lapA[cidx]
    exp[SS] = p.eta * p.mu0 * (j[0] ** 2 + j[1] ** 2 + j[2] ** 2) / (rho * T)
    _check(oracle.mhd_rhs(f, p), exp)


@pytest.mark.parametrize("dt", [0.1, 0.3])
def test_rk3_stability_polynomial_on_beltrami_field(dt):
    p = _par(eta=0.5)
    (Z, Y, X), h = grid(N)
    k, eps = 3, 1e-2
    f = np.zeros((8, N, N, N))
    f[AX] = eps * np.sin(k * Z)
    f[AY] = eps * np.cos(k * Z)
    out = oracle.mhd_rk3(f, p, dt, 1)
    z = p.eta * lam2(k, h) * dt
    P = 1 + z + z * z / 2 + z ** 3 / 6
    np.testing.assert_allclose(out[AX], P * f[AX], atol=1e-14)
    np.testing.assert_allclose(out[AY], P * f[AY], atol=1e-14)
    assert np.abs(out[[LNRHO, UX, UY, UZ, AZ]]).max() < 1e-14
    # entropy is heated uniformly (ohmic heating of a spatially uniform |j|)
    assert np.ptp(out[SS]) < 1e-14 and out[SS].mean() > 0
    # the polynomial differs from exp(z) at 4th order: the test can see a wrong scheme
    assert abs(P - np.exp(z)) > 1e-5


def test_rk3_is_third_order_in_time_on_a_nonlinear_state():
    # Sec. 3.3: a 3rd-order scheme.  On a random smooth state large enough that advection and the
    # Lorentz force matter, the error at a fixed time falls 8x per halving of dt, measured
    # against the same scheme at a 16x smaller step (the grid is fixed, so the spatial error
    # cancels).  The linear stability polynomial above cannot see the nonlinear order condition.
    n = 8
    p = MhdParams.for_grid(n, nu=0.02, eta=0.03, zeta=0.01)
    f = synth.mhd_fields(n, seed=3) * 100.0
    T = 0.4
    ref = oracle.mhd_rk3(f, p, T / 256, 256)
    assert np.abs(ref - f).max() > 0.1  # the state moves well beyond the linear regime
    errs = np.array([np.abs(oracle.mhd_rk3(f, p, T / m, m) - ref).max() for m in (8, 16, 32)])
    slopes = np.log2(errs[:-1] / errs[1:])
    assert np.all(slopes > 2.8) and np.all(slopes < 3.3), slopes


def test_rhs_converges_at_sixth_order_under_refinement():
    # The same smooth fields (sums of sine modes, evaluated on each grid) at n = 24, 48, 96: the
    # right-hand side at the coarse grid's points changes by a factor ~2^6 per refinement in
    # every field, conduction included, as the 6th-order differences of Sec. 3.3 require.
    res = {}
    for n in (24, 48, 96):
        p = MhdParams.for_grid(n, nu=0.02, eta=0.03, zeta=0.01, K=0.1)
        res[n] = oracle.mhd_rhs(synth.mhd_fields(n, seed=5, kmax=2, amp=0.1), p)
    e1 = np.abs(res[24] - res[48][:, ::2, ::2, ::2]).max(axis=(1, 2, 3))
    e2 = np.abs(res[48] - res[96][:, ::2, ::2, ::2]).max(axis=(1, 2, 3))
    slopes = np.log2(e1 / e2)
    assert np.all(slopes > 5.5) and np.all(slopes < 6.5), slopes


def test_box_step_matches_periodic_step():
    n = 12
    p = MhdParams.for_grid(n)
    f = synth.mhd_fields(n, seed=3) * 30.0
    dt = p.dt_default()
    ref = oracle.mhd_rk3(f, p, dt, 1)
    c = (4, 7, 2)
    m = 2 * 9 + 1
    idx = [np.arange(ci - 9, ci + 10) % n for ci in c]
    box = f[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
    out = oracle.mhd_rk3_box(box, p, dt, 3)
    np.testing.assert_allclose(out[:, 9, 9, 9], ref[:, c[0], c[1], c[2]], rtol=1e-13, atol=1e-16)
    assert out.shape[1] == m


def test_heat_conduction_from_an_entropy_mode():
    # u = A = 0, lnrho uniform, s = eps sin(k y): only A3 changes; with phi = gamma s/cp,
    # div(K grad T)/(rho T) = (K/rho)(lap phi + |grad phi|^2) and every derivative is a symbol.
    p = _par(K=0.7)
    (Z, Y, X), h = grid(N)
    k, eps, lr = 3, 2e-2, 0.4
    f = np.zeros((8, N, N, N))
    f[LNRHO] = lr
    f[SS] = eps * np.sin(k * Y)
    g = p.gamma / p.cp
    rho = np.exp(lr)
    cs2, _ = _temp(p, lr, f[SS])
    exp = np.zeros_like(f)
    exp[UY] = -cs2 * (lam1(k, h) * eps * np.cos(k * Y)) / p.cp   # the pressure term (already pinned)
    lap_phi = g * lam2(k, h) * eps * np.sin(k * Y)
    grad_phi2 = (g * lam1(k, h) * eps * np.cos(k * Y)) ** 2
    exp[SS] = p.K / rho * (lap_phi + grad_phi2)
    _check(oracle.mhd_rhs(f, p), exp)
    # K = 0 leaves A3 without the term
    assert np.abs(oracle.mhd_rhs(f, _par(K=0.0))[SS]).max() < 1e-15


def test_heat_conduction_from_a_density_mode():
    # lnrho = lr + eps sin(k z): phi = (gamma-1)(lnrho - lnrho0), rho varies cell by cell
    p = _par(K=0.25)
    (Z, Y, X), h = grid(N)
    k, eps, lr = 2, 3e-2, -0.2
    f = np.zeros((8, N, N, N))
    f[LNRHO] = lr + eps * np.sin(k * Z)
    gm1 = p.gamma - 1.0
    rho = np.exp(f[LNRHO])
    lap_phi = gm1 * lam2(k, h) * eps * np.sin(k * Z)
    grad_phi2 = (gm1 * lam1(k, h) * eps * np.cos(k * Z)) ** 2
    got = oracle.mhd_rhs(f, p)
    np.testing.assert_allclose(got[SS], p.K / rho * (lap_phi + grad_phi2), rtol=0, atol=1e-12)
