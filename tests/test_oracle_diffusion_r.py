"""Pins of the oracle's radius-r diffusion step (Eq. 4 with the order-2r central Laplacian; the
radius sweep of the diffusion equation, Sec. 5.3).

Nothing here re-evaluates the oracle's weight formula: the weights are checked against the
published table of centred finite-difference weights (Fornberg 1988), and the step against
polynomial exactness, the convergence order 2r, separable multi-axis closed forms and the
invariants of the periodic problem.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

# Fornberg (1988), centred 2nd-derivative weights of order 2, 4, 6, 8: (c_0, c_1, ..., c_r).
PUBLISHED = {
    1: [Fr(-2), Fr(1)],
    2: [Fr(-5, 2), Fr(4, 3), Fr(-1, 12)],
    3: [Fr(-49, 18), Fr(3, 2), Fr(-3, 20), Fr(1, 90)],
    4: [Fr(-205, 72), Fr(8, 5), Fr(-1, 5), Fr(8, 315), Fr(-1, 560)],
}
ONE = (1.0, 1.0, 1.0)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_delta_response_is_the_published_weights(r):
    n = 2 * r + 3
    fhat = np.zeros(n + 2 * r)
    fhat[r + n // 2] = 1.0
    out = oracle.diffusion_r_box(fhat, r, 1.0, 1.0, ONE, (n,))
    lap = out.copy()
    lap[n // 2] -= 1.0
    want = np.zeros(n)
    want[n // 2] = float(PUBLISHED[r][0])
    for k in range(1, r + 1):
        want[n // 2 + k] = want[n // 2 - k] = float(PUBLISHED[r][k])
    np.testing.assert_allclose(lap, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_polynomial_exactness_up_to_degree_2r_plus_1(r):
    h, x0, n = 0.1, 0.3, 9
    x = x0 + h * (np.arange(n + 2 * r) - r)
    for m in range(0, 2 * r + 2):
        out = oracle.diffusion_r_box(x ** m, r, 1.0, 1.0, (h, 1.0, 1.0), (n,))
        lap = out - x[r:r + n] ** m
        exact = m * (m - 1) * x[r:r + n] ** (m - 2) if m >= 2 else np.zeros(n)
        np.testing.assert_allclose(lap, exact, rtol=1e-8, atol=1e-8, err_msg=f"r={r} degree {m}")
    m = 2 * r + 2  # one degree more is not reproduced
    out = oracle.diffusion_r_box(x ** m, r, 1.0, 1.0, (h, 1.0, 1.0), (n,))
    err = np.abs(out - x[r:r + n] ** m - m * (m - 1) * x[r:r + n] ** (m - 2)).max()
    assert err > 1e-6


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_convergence_order_is_2r(r):
    ns = (12, 16, 24)
    errs = []
    for n in ns:
        h = 2 * np.pi / n
        x = h * np.arange(n)
        f = np.sin(x)
        lap = oracle.diffusion_r(f, r, 1.0, 1.0, (h, 1.0, 1.0), 1) - f
        errs.append(np.abs(lap + np.sin(x)).max())
    slopes = [np.log(errs[i] / errs[i + 1]) / np.log(ns[i + 1] / ns[i]) for i in range(2)]
    assert all(abs(s - 2 * r) < 0.35 for s in slopes), (r, errs, slopes)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_separable_quadratics_in_2d_and_3d(r):
    # lap(x^2 + 3 y^2 - z^2 + x y) = 2 + 6 - 2 = 6 for any r, any spacing
    hx, hy, hz = 0.3, 0.7, 0.45
    nx, ny, nz = 2 * r + 2, 2 * r + 3, 2 * r + 1
    z, y, x = np.meshgrid(hz * (np.arange(nz + 2 * r) - r), hy * (np.arange(ny + 2 * r) - r),
                          hx * (np.arange(nx + 2 * r) - r), indexing="ij")
    f = x ** 2 + 3 * y ** 2 - z ** 2 + x * y
    out = oracle.diffusion_r_box(f, r, 0.5, 2.0, (hx, hy, hz), (nz, ny, nx))
    inner = f[r:r + nz, r:r + ny, r:r + nx]
    np.testing.assert_allclose(out - inner, 6.0, rtol=0, atol=1e-9)
    # 2D, anisotropic and of degree 4 (exact for r >= 2): lap(x^4 + y^4) = 12 x^2 + 12 y^2
    f2 = x[0] ** 4 + y[0] ** 4
    out2 = oracle.diffusion_r_box(f2, r, 1.0, 1.0, (hx, hy, 1.0), (ny, nx))
    want = 12 * x[0, r:r + ny, r:r + nx] ** 2 + 12 * y[0, r:r + ny, r:r + nx] ** 2
    got = out2 - f2[r:r + ny, r:r + nx]
    if r >= 2:
        np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-9)
    else:  # the order-2 Laplacian adds h^2/12 * f'''' = 2 hx^2 + 2 hy^2
        np.testing.assert_allclose(got, want + 2 * hx ** 2 + 2 * hy ** 2, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_periodic_invariants(r):
    rng = np.random.default_rng(1)
    f = rng.standard_normal((10, 11, 12))
    h = 2 * np.pi / 12
    g = oracle.diffusion_r(f, r, 0.1 * h * h, 1.0, (h, h, h), 5)
    assert abs(g.sum() - f.sum()) < 1e-10 * np.abs(f).sum()
    assert (g ** 2).sum() < (f ** 2).sum()


def test_radius_3_is_the_sixth_order_step():
    rng = np.random.default_rng(2)
    f = rng.standard_normal((9, 10, 11))
    h = (0.4, 0.5, 0.6)
    a = oracle.diffusion_r(f, 3, 0.01, 1.0, h, 3)
    b = oracle.diffusion(f, 0.01, 1.0, h, 3)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13)


def test_radius_outside_1_to_4_is_rejected():
    with pytest.raises(AssertionError):
        oracle.diffusion_r(np.zeros(9), 5, 0.1, 1.0, ONE, 1)
