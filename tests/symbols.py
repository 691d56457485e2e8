"""Closed-form Fourier symbols of the 6th-order central differences (test helper).

For f = sin(k x + phase) sampled with spacing h, the 7-point first-derivative stencil returns
lam1 * cos(k x + phase) and the second-derivative stencil lam2 * sin(k x + phase), exactly up
to rounding; the diagonal mixed stencil applied to sin(kx x + ky y + phase) returns
mu * sin(kx x + ky y + phase).  The weights are the textbook 6th-order central weights
(Fornberg 1988); their uniqueness is pinned separately by polynomial exactness.
"""
import numpy as np

D1 = (3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0)          # offsets 1, 2, 3 (antisymmetric)
D2C, D2 = -49.0 / 18.0, (3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0)
DM = (270.0, -27.0, 2.0)                             # / 720


def lam1(k, h):
    return 2.0 / h * sum(w * np.sin((a + 1) * k * h) for a, w in enumerate(D1))


def lam2(k, h):
    return (D2C + 2.0 * sum(w * np.cos((a + 1) * k * h) for a, w in enumerate(D2))) / h ** 2


def mu(kx, ky, hx, hy):
    s = sum(m * np.sin((a + 1) * kx * hx) * np.sin((a + 1) * ky * hy) for a, m in enumerate(DM))
    return -4.0 * s / (720.0 * hx * hy)


def grid(n):
    """Coordinates (z, y, x) of an n^3 periodic grid with spacing 2 pi / n."""
    h = 2.0 * np.pi / n
    c = np.arange(n) * h
    return np.meshgrid(c, c, c, indexing="ij"), h
