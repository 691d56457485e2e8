"""Pins of the oracle's cross-correlation (Eq. 3) and periodic padding (Eq. 2).

None of these checks use the oracle's arithmetic: they compare with Python integers masked
to 32 bits, numpy/scipy library routines, and special cases with known results.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from paper_2406_08923_gb300 import synth


def _brute_u32(data, g, sweeps):
    n, r = len(data), (len(g) - 1) // 2
    cur = [int(v) & 0xFFFFFFFF for v in data]
    for _ in range(sweeps):
        cur = [sum(int(g[j + r]) * cur[(i + j) % n] for j in range(-r, r + 1)) & 0xFFFFFFFF
               for i in range(n)]
    return np.array(cur, dtype=np.uint64).astype(np.uint32).view(np.int32)


@pytest.mark.parametrize("n,sweeps", [(16, 10), (7, 3), (31, 1)])
def test_int32_matches_python_ints_mod_2_32(n, sweeps):
    data, g = synth.xcorr_int32(n, seed=11 + n)
    assert np.array_equal(oracle.xcorr1d(data, g, sweeps), _brute_u32(data, g, sweeps))


def test_int32_wraps_like_twos_complement():
    # values large enough to overflow int32 within one sweep
    data = np.array([2**31 - 1, -2**31, 123456789, -987654321, 7, 2**30, -5], dtype=np.int32)
    g = np.array([8, -8, 7, 5, -3, 2, -1], dtype=np.int32)
    assert np.array_equal(oracle.xcorr1d(data, g, 4), _brute_u32(data, g, 4))


def test_int32_box_sweep_with_caller_halo_wraps_like_twos_complement():
    # one sweep over a caller-filled int32 box (no periodic wrap): negative and extreme values
    fhat = np.array([-2**31, 2**31 - 1, -1, 5, -77777777, 2**30 + 3, -6, 99, -2**29, 12], dtype=np.int32)
    g = np.array([-8, 7, 5, -3, 2], dtype=np.int32)
    r, n = 2, len(fhat) - 4
    exp = [sum(int(g[j + r]) * int(fhat[i + r + j]) for j in range(-r, r + 1)) & 0xFFFFFFFF for i in range(n)]
    exp = np.array(exp, dtype=np.uint64).astype(np.uint32).view(np.int32)
    assert np.array_equal(oracle.xcorr1d_box(fhat, g), exp)


def test_f64_matches_scipy_correlate1d_wrap():
    x = synth.xcorr_f64(257, seed=5)
    g = np.array([1 / 90, -3 / 20, 3 / 2, -49 / 18, 3 / 2, -3 / 20, 1 / 90])
    ref = x.copy()
    for _ in range(3):
        ref = ndi.correlate1d(ref, g, mode="wrap")
    np.testing.assert_allclose(oracle.xcorr1d(x, g, 3), ref, rtol=1e-12, atol=1e-12)


def test_asymmetric_weights_orientation():
    # Eq. 3 is a correlation, not a convolution: weight index j multiplies f[i + j]
    x = np.zeros(11)
    x[5] = 1.0
    g = np.arange(1.0, 8.0)  # g_{-3..3} = 1..7
    out = oracle.xcorr1d(x, g, 1)
    # out[i] = g[5 - i] where 5 - i in [-3, 3]  ->  out[2] = g_{+3} = 7, out[8] = g_{-3} = 1
    assert out[2] == 7.0 and out[8] == 1.0 and out[5] == 4.0


def test_identity_and_shift():
    x = synth.xcorr_f64(64, seed=9)
    ident = np.array([0, 0, 0, 1.0, 0, 0, 0])
    np.testing.assert_array_equal(oracle.xcorr1d(x, ident, 5), x)
    shift = np.array([0, 0, 0, 0, 0, 0, 1.0])  # g_{+3} = 1: out[i] = x[i + 3]
    np.testing.assert_array_equal(oracle.xcorr1d(x, shift, 2), np.roll(x, -6))


def test_box_sweep_is_valid_correlation():
    # caller-filled (non-periodic) halo: one sweep equals numpy's 'valid' correlation
    rng = synth.uniform(3, 1, 40, -1, 1)
    g = synth.uniform(3, 2, 7, -1, 1)
    np.testing.assert_allclose(oracle.xcorr1d_box(rng, g), np.correlate(rng, g, "valid"),
                               rtol=1e-13, atol=1e-15)


def test_pad_periodic_3d_matches_numpy_wrap():
    f = synth.uniform(4, 1, 5 * 7 * 8).reshape(5, 7, 8)
    np.testing.assert_array_equal(oracle.pad_periodic(f), np.pad(f, 3, mode="wrap"))
    f1 = synth.uniform(4, 2, 9)
    np.testing.assert_array_equal(oracle.pad_periodic(f1), np.pad(f1, 3, mode="wrap"))


def test_pad_periodic_leaves_unit_axes_unpadded():
    # an axis of extent 1 carries no halo (a 2D field stored as a 3D array)
    f = synth.uniform(4, 3, 6 * 8).reshape(1, 6, 8)
    np.testing.assert_array_equal(oracle.pad_periodic(f), np.pad(f, ((0, 0), (3, 3), (3, 3)), mode="wrap"))
    g = synth.uniform(4, 4, 5 * 7).reshape(5, 1, 7)
    np.testing.assert_array_equal(oracle.pad_periodic(g, 2), np.pad(g, ((2, 2), (0, 0), (2, 2)), mode="wrap"))
