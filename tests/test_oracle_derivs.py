"""Pins of the oracle's 6th-order central differences (Sec. 3.3).

* Polynomial exactness on a caller-filled box: exact for degree <= 6 (1st derivative),
  <= 7 (2nd), and x^a y^b with a + b <= 7 (mixed).  The 7-point central stencils with this
  property are unique, so this pins every weight.
* Closed-form Fourier symbols on the periodic grid (indexing, wrap, axis order, scaling).
* Convergence order 6 under grid refinement against the analytic derivative.
"""
import itertools

import numpy as np
import pytest

import oracle
from symbols import grid, lam1, lam2, mu

NAMES = ("dx", "dy", "dz", "dxx", "dyy", "dzz", "dxy", "dxz", "dyz")


def _poly_box(px, py, pz, h, n=5):
    """Box of interior n^3 (padded n + 6) with coordinates centred near 0, spacing h."""
    c = (np.arange(n + 6) - (n + 6) // 2) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = X ** px * Y ** py * Z ** pz
    return f, (X, Y, Z)


def _analytic(px, py, pz, X, Y, Z):
    def d(p, x, k):  # k-th derivative of x^p
        c = 1.0
        for i in range(k):
            c *= (p - i)
        return c * x ** (p - k) if p >= k else 0.0 * x
    base = {"x": (px, X), "y": (py, Y), "z": (pz, Z)}
    out = {}
    for name in NAMES:
        ks = {"x": name[1:].count("x"), "y": name[1:].count("y"), "z": name[1:].count("z")}
        v = 1.0
        for ax, (p, coord) in base.items():
            v = v * d(p, coord, ks[ax])
        out[name] = v
    return out


@pytest.mark.parametrize("h", [1.0, 0.5])
def test_polynomial_exactness(h):
    sl = (slice(3, -3),) * 3
    for px, py, pz in itertools.product(range(8), repeat=3):
        deg = px + py + pz
        if deg > 7:
            continue
        f, (X, Y, Z) = _poly_box(px, py, pz, h)
        got = oracle.derivs_box(f, (h, h, h))
        exp = _analytic(px, py, pz, X[sl], Y[sl], Z[sl])
        scale = max(1.0, np.abs(f).max()) / h ** 2
        for q, name in enumerate(NAMES):
            order = len(name) - 1
            axes = name[1:]
            # expected-exact range of each stencil
            if order == 1:
                exact = {"x": px, "y": py, "z": pz}[axes] <= 6
            elif axes[0] == axes[1]:
                exact = {"x": px, "y": py, "z": pz}[axes[0]] <= 7
            else:
                a, b = ({"x": px, "y": py, "z": pz}[c] for c in axes)
                exact = a + b <= 7
            if exact:
                np.testing.assert_allclose(got[q], np.broadcast_to(exp[name], got[q].shape),
                                           rtol=0, atol=1e-11 * scale,
                                           err_msg=f"{name} on x^{px} y^{py} z^{pz}")


def test_inexact_beyond_order():
    # x^7 is NOT differentiated exactly by the first-derivative stencil (order is exactly 6)
    f, (X, Y, Z) = _poly_box(7, 0, 0, 1.0)
    got = oracle.derivs_box(f, (1.0, 1.0, 1.0))[0]
    exp = 7 * X[3:-3, 3:-3, 3:-3] ** 6
    assert np.abs(got - exp).max() > 1.0


@pytest.mark.parametrize("k", [1, 3, 5])
def test_fourier_symbols(k):
    n = 16
    (Z, Y, X), h = grid(n)
    ph = 0.37
    for ax, C in enumerate((X, Y, Z)):
        f = np.sin(k * C + ph)
        d = oracle.derivs_box(oracle.pad_periodic(f), (h, h, h))
        np.testing.assert_allclose(d[ax], lam1(k, h) * np.cos(k * C + ph), atol=1e-12)
        np.testing.assert_allclose(d[3 + ax], lam2(k, h) * f, atol=1e-11)
        for q in range(3):
            if q != ax:
                assert np.abs(d[q]).max() < 1e-12
    # mixed: sin(kx x + ky y + kz z + ph) -> mu * same
    kx, ky, kz = k, k + 1, 2
    f = np.sin(kx * X + ky * Y + kz * Z + ph)
    d = oracle.derivs_box(oracle.pad_periodic(f), (h, h, h))
    np.testing.assert_allclose(d[6], mu(kx, ky, h, h) * f, atol=1e-11)
    np.testing.assert_allclose(d[7], mu(kx, kz, h, h) * f, atol=1e-11)
    np.testing.assert_allclose(d[8], mu(ky, kz, h, h) * f, atol=1e-11)


def test_anisotropic_spacing_scaling():
    # spacing enters as 1/h (1st), 1/h^2 (2nd), 1/(ha hb) (mixed), per axis
    n = 12
    hs = (0.3, 0.5, 0.7)
    c = [np.arange(n + 6) * hh for hh in hs]
    Z, Y, X = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    f = 2 * X ** 2 + 3 * Y * Z - X * Y + Z ** 2
    d = oracle.derivs_box(f, hs)
    sl = (slice(3, -3),) * 3
    np.testing.assert_allclose(d[0], (4 * X - Y)[sl], atol=1e-10)
    np.testing.assert_allclose(d[1], (3 * Z - X)[sl], atol=1e-10)
    np.testing.assert_allclose(d[2], (3 * Y + 2 * Z)[sl], atol=1e-10)
    np.testing.assert_allclose(d[3:6], np.broadcast_to(np.array([4.0, 0.0, 2.0])[:, None, None, None], d[3:6].shape), atol=1e-9)
    np.testing.assert_allclose(d[6:9], np.broadcast_to(np.array([-1.0, 0.0, 3.0])[:, None, None, None], d[6:9].shape), atol=1e-9)


def test_non_cubic_box_keeps_axis_order():
    # interior (nz, ny, nx) = (5, 7, 9): every derivative plane comes back as (nz, ny, nx)
    hs = (0.3, 0.5, 0.7)
    ext = (9, 7, 5)  # nx, ny, nz
    c = [np.arange(m + 6) * hh for m, hh in zip(ext, hs)]
    Z, Y, X = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    f = X ** 3 - 2 * X * Y + Y * Z ** 2
    d = oracle.derivs_box(f, hs)
    assert d.shape == (9, 5, 7, 9)
    sl = (slice(3, -3),) * 3
    X, Y, Z = X[sl], Y[sl], Z[sl]
    exp = (3 * X ** 2 - 2 * Y, -2 * X + Z ** 2, 2 * Y * Z, 6 * X, 0 * X, 2 * Y, -2 + 0 * X, 0 * X, 2 * Z)
    for q, e in enumerate(exp):
        np.testing.assert_allclose(d[q], e, atol=1e-9, err_msg=NAMES[q])


def test_convergence_order_six():
    errs = []
    ns = (16, 32, 64)
    for n in ns:
        (Z, Y, X), h = grid(n)
        f = np.sin(2 * X + 1.0) * np.cos(Y)
        d = oracle.derivs_box(oracle.pad_periodic(f), (h, h, h))
        e1 = np.abs(d[0] - 2 * np.cos(2 * X + 1.0) * np.cos(Y)).max()
        e2 = np.abs(d[3] + 4 * f).max()
        e3 = np.abs(d[6] + 2 * np.cos(2 * X + 1.0) * np.sin(Y)).max()
        errs.append((e1, e2, e3))
    errs = np.array(errs)
    slopes = np.log2(errs[:-1] / errs[1:])
    assert np.all(slopes > 5.6) and np.all(slopes < 6.6), slopes
