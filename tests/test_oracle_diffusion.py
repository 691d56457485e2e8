"""Pins of the oracle's forward-Euler diffusion step (Eq. 4, Sec. 3.2).

* A single Fourier mode stays a single mode and its amplitude after n steps is
  (1 + dt alpha sum_axes lam2(k_axis))^n (the discrete symbol; exact up to rounding).
* Sum f is conserved (the 2nd-derivative weights sum to zero), sum f^2 does not grow at
  dt = 0.1 dx^2 (stable), and a quadratic with a caller-filled halo is updated exactly.
* 1D and 2D cases reduce to the same closed form with fewer axes.
"""
import numpy as np

import oracle
from paper_2406_08923_gb300 import synth
from symbols import grid, lam2


def test_single_mode_amplitude_3d():
    n, steps, alpha = 16, 25, 0.7
    (Z, Y, X), h = grid(n)
    k = (2, 3, 5)
    f0 = np.sin(k[0] * X + k[1] * Y + k[2] * Z + 0.4)
    dt = 0.1 * h * h
    out = oracle.diffusion(f0, dt, alpha, (h, h, h), steps)
    amp = (1 + dt * alpha * sum(lam2(kk, h) for kk in k)) ** steps
    np.testing.assert_allclose(out, amp * f0, atol=1e-13)
    # and clearly not the identity
    assert amp < 0.9


def test_single_mode_1d_and_2d():
    n = 24
    h = 2 * np.pi / n
    x = np.arange(n) * h
    f1 = np.cos(4 * x)
    dt = 0.1 * h * h
    np.testing.assert_allclose(oracle.diffusion(f1, dt, 1.0, (h, 1, 1), 7),
                               (1 + dt * lam2(4, h)) ** 7 * f1, atol=1e-13)
    Y, X = np.meshgrid(x, x, indexing="ij")
    f2 = np.sin(3 * X - 5 * Y)
    np.testing.assert_allclose(oracle.diffusion(f2, dt, 1.0, (h, h, 1), 5),
                               (1 + dt * (lam2(3, h) + lam2(5, h))) ** 5 * f2, atol=1e-13)


def test_anisotropic_grid_mode():
    nz, ny, nx = 12, 10, 16
    hx, hy, hz = 2 * np.pi / nx, 2 * np.pi / ny, 2 * np.pi / nz
    Z, Y, X = np.meshgrid(np.arange(nz) * hz, np.arange(ny) * hy, np.arange(nx) * hx, indexing="ij")
    f0 = np.cos(2 * X) * np.sin(3 * Y) * np.cos(Z)
    dt = 0.05 * min(hx, hy, hz) ** 2
    amp = (1 + dt * (lam2(2, hx) + lam2(3, hy) + lam2(1, hz))) ** 3
    np.testing.assert_allclose(oracle.diffusion(f0, dt, 1.0, (hx, hy, hz), 3), amp * f0, atol=1e-13)


def test_conservation_and_decay():
    n = 20
    f0 = synth.heat_field(n, seed=7)
    h = 2 * np.pi / n
    cur = f0
    s0 = cur.sum()
    e_prev = (cur ** 2).sum()
    for _ in range(10):
        cur = oracle.diffusion(cur, 0.1 * h * h, 1.0, (h, h, h), 1)
        assert abs(cur.sum() - s0) < 1e-10 * np.abs(f0).sum()
        e = (cur ** 2).sum()
        assert e <= e_prev * (1 + 1e-14)
        e_prev = e


def test_quadratic_with_caller_halo():
    # lap(x^2 + 2 y^2 - z^2 + xy) = 2 + 4 - 2 = 4, exact for the 6th-order stencil
    n, h, dt, alpha = 6, 0.25, 0.01, 3.0
    c = (np.arange(n + 6) - 5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = X ** 2 + 2 * Y ** 2 - Z ** 2 + X * Y
    out = oracle.diffusion_box(f, dt, alpha, (h, h, h), (n, n, n))
    np.testing.assert_allclose(out, f[3:-3, 3:-3, 3:-3] + dt * alpha * 4.0, atol=1e-12)
