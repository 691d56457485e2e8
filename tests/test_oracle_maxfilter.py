"""Pins of the oracle's max filter, the nonlinear 1D stencil f'_i = max_{j=-r..r} f^_{i+j}
(Sec. 2.1): scipy's maximum_filter1d with periodic wrap, brute force on tiny inputs, caller
halos, and the composition law (r1 then r2 equals r1 + r2)."""
import numpy as np
import pytest

import oracle

scipy_ndimage = pytest.importorskip("scipy.ndimage")


@pytest.mark.parametrize("r", [0, 1, 3, 17, 100])
def test_periodic_matches_scipy(r):
    rng = np.random.default_rng(5)
    for data in (rng.standard_normal(1001), rng.integers(-10 ** 9, 10 ** 9, 1001).astype(np.int32)):
        got = oracle.maxfilter1d(data, r)
        want = scipy_ndimage.maximum_filter1d(data, size=2 * r + 1, mode="wrap")
        assert np.array_equal(got, want.astype(got.dtype))
        assert got.dtype == (np.int32 if data.dtype == np.int32 else np.float64)


def test_brute_force_tiny():
    rng = np.random.default_rng(6)
    n, r = 9, 2
    data = rng.integers(-50, 50, n).astype(np.int32)
    got = oracle.maxfilter1d(data, r, 1)
    want = [max(int(data[(i + j) % n]) for j in range(-r, r + 1)) for i in range(n)]
    assert got.tolist() == want


def test_caller_halo_box():
    rng = np.random.default_rng(7)
    r, n = 4, 50
    fhat = rng.standard_normal(n + 2 * r)
    got = oracle.maxfilter1d_box(fhat, r)
    want = np.lib.stride_tricks.sliding_window_view(fhat, 2 * r + 1).max(axis=1)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("r1,r2", [(1, 2), (3, 5), (16, 16)])
def test_sweeps_compose_into_a_wider_window(r1, r2):
    rng = np.random.default_rng(8)
    data = rng.standard_normal(777)
    two = oracle.maxfilter1d(oracle.maxfilter1d(data, r1), r2)
    assert np.array_equal(two, oracle.maxfilter1d(data, r1 + r2))
    assert np.array_equal(oracle.maxfilter1d(data, r1, sweeps=2), oracle.maxfilter1d(data, 2 * r1))
