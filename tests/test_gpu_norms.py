"""GPU FP64 norm reductions (sum, sum of squares, max |f|, MHD mass) against the oracle's
norms and mass (long-double accumulation; pinned against math.fsum in test_oracle_norms.py)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import heat_plan, mhd_plan
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth

pytestmark = pytest.mark.gpu


def _ref(x):
    return oracle.norms(np.asarray(x, np.float64))


@pytest.mark.parametrize("dtype", (L.STENCIL_F64, L.STENCIL_F32))
def test_heat_field_norms(cuda_lib, dtype):
    shape = (37, 41, 29)
    f0 = synth.heat_field(shape, seed=2)
    p, _ = heat_plan(shape, dtype)
    a = p.alloc(fill=1e6)  # halo garbage must not leak into interior reductions
    p.upload(a, [f0])
    got = p.norms(a)
    ref = _ref(p.download(a)[0])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_int32_norms(cuda_lib):
    n = (1 << 20) + 5
    data, g = synth.xcorr_int32(n)
    p = L.Plan(1, (n,), 3, 1, L.STENCIL_BC_PERIODIC, L.STENCIL_XCORR, L.STENCIL_I32, L.STENCIL_I32, coeffs=g)
    a = p.alloc(fill=123456)
    p.upload(a, [data])
    np.testing.assert_allclose(p.norms(a), _ref(data), rtol=1e-15)


@pytest.mark.parametrize("storage", (L.STENCIL_F64, L.STENCIL_BF16))
def test_mhd_norms_and_mass(cuda_lib, storage):
    shape = (20, 24, 28)
    f8 = synth.mhd_fields(shape, seed=4)
    p, par = mhd_plan(shape, storage)
    a = p.alloc()
    p.upload(a, f8)
    got = p.norms(a)
    stored = p.download(a)
    for q in range(8):
        # sums of pure sine modes are ~0: compare them against the rounding scale sum |f|
        atol = 1e-14 * np.abs(stored[q]).sum()
        np.testing.assert_allclose(got[3 * q:3 * q + 3], _ref(stored[q]), rtol=1e-12, atol=atol)
    mass = oracle.mass(stored[0]) * par.dx[0] * par.dx[1] * par.dx[2]
    assert abs(got[-1] - mass) <= 1e-13 * abs(mass)


def test_norms_are_deterministic(cuda_lib):
    shape = (64, 64, 64)
    p, _ = heat_plan(shape, L.STENCIL_F64)
    a = p.alloc()
    p.upload(a, [synth.heat_field(shape, seed=9)])
    r = [p.norms(a) for _ in range(3)]
    assert all(np.array_equal(r[0], x) for x in r[1:])


@pytest.mark.parametrize("storage", (L.STENCIL_F64, L.STENCIL_F32, L.STENCIL_BF16))
def test_a_nan_cell_makes_the_max_nan(cuda_lib, storage):
    # max |f| must not drop a NaN (fmax would): a field that has blown up reports NaN
    shape = (20, 24, 28)
    p, _ = mhd_plan(shape, storage)
    a = p.alloc()
    f8 = synth.mhd_fields(shape, seed=4)
    f8[3][7, 11, 13] = np.nan
    p.upload(a, f8)
    got = p.norms(a)
    for q in range(8):
        s, s2, mx = got[3 * q:3 * q + 3]
        if q == 3:
            assert np.isnan(s) and np.isnan(s2) and np.isnan(mx), got[9:12]
        else:
            assert np.isfinite([s, s2, mx]).all(), (q, got[3 * q:3 * q + 3])


@pytest.mark.parametrize("shape", [(40, 70, 33), (7, 7, (1 << 17) + 5)])
def test_norms_when_warps_take_several_pieces(cuda_lib, shape):
    # More pieces than the pass's warps (304 x 8), so each warp walks on from its first piece:
    # (40, 70, 33) has 2800 one-segment rows; (7, 7, 2^17 + 5) has 49 rows of 65 segments each
    # (3185 pieces), whose walk carries from segment to row and from row to plane.
    nz, ny, nx = shape
    f = synth.uniform(2406089241, 3, nz * ny * nx, -1.0, 1.0).reshape(shape)
    p = L.Plan(3, (nx, ny, nz), 3, 1, L.STENCIL_BC_PERIODIC, L.STENCIL_DIFFUSION, L.STENCIL_F64, L.STENCIL_F64,
               params=L.heat_params(shape))
    a = p.alloc(fill=1e6)
    p.upload(a, [f])
    np.testing.assert_allclose(p.norms(a), _ref(f), rtol=1e-12, atol=1e-12)
    p.close()
