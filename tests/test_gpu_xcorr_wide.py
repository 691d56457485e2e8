"""GPU parity of the large-radius 1D stencils, through the C ABI:

* the cross-correlation of Eq. 3 at radius 5..1024 (the radius sweep of Sec. 5.2), FP64 and
  FP32, against the FP64 oracle (FP64 <= 1e-12, FP32 <= 1e-5, relative L2 and L-infinity);
* the max filter f'_i = max_{j=-r..r} f^_{i+j} (Sec. 2.1) for int32, FP32 and FP64 at radius
  0..1024: bit-exact against the oracle's plain window maximum.
"""
import numpy as np
import pytest

import oracle
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth

from gpu_util import assert_close

pytestmark = pytest.mark.gpu

SEED = 2406089238
TOL = {L.STENCIL_F64: 1e-12, L.STENCIL_F32: 1e-5}


def _run(kind, storage, n, r, data, coeffs=None, sweeps=1, bc=L.STENCIL_BC_PERIODIC):
    p = L.Plan(1, (n,), r, 1, bc, kind, storage, storage, coeffs=coeffs)
    a, b = p.alloc(), p.alloc()
    p.upload(a, [data])
    p.step(a, b, sweeps)
    p.sync()
    return p, a, b


def _weights(r, signed):
    w = synth.uniform(SEED, 100 + r, 2 * r + 1, -1.0 if signed else 0.0, 1.0)
    return w / np.abs(w).sum()


@pytest.mark.parametrize("storage", [L.STENCIL_F64, L.STENCIL_F32])
# radii cover every compiled register-block size V (FP32 9/11/13/15, FP64 5/7/9), and the
# sizes both the bulk-copied interior chunks and the staged edge chunks
@pytest.mark.parametrize("r,n,sweeps", [(5, 3001, 1), (8, 20001, 2), (16, 70001, 3), (32, 50003, 1), (100, 4097, 2),
                                        (128, 300007, 1), (1024, 5000, 1), (1024, (1 << 20) + 3, 2)])
def test_wide_xcorr_matches_oracle(cuda_lib, storage, r, n, sweeps):
    signed = storage == L.STENCIL_F64  # FP32 sums of 2r+1 terms: keep them well conditioned
    g = _weights(r, signed)
    data = synth.uniform(SEED, 200 + r, n, -1.0 if signed else 0.0, 1.0)
    if storage == L.STENCIL_F32:
        data = data.astype(np.float32).astype(np.float64)
        g = g.astype(np.float32).astype(np.float64)
    p, a, b = _run(L.STENCIL_XCORR, storage, n, r, data, coeffs=g, sweeps=sweeps)
    # FP32 up to radius 32 runs the temporally blocked kernel, the rest the wide one
    blocked = storage == L.STENCIL_F32 and r <= 32
    assert (p.variant()[2] == "wide_register_blocked") != blocked, p.variant()[2]
    got = p.download(b)[0]
    ref = oracle.xcorr1d(data, g, sweeps)
    assert_close(got, ref, TOL[storage], f"xcorr r={r} n={n}")
    # periodic images in the output halo; input interior untouched
    full = p.view3(b[0])[0, 0].double().cpu().numpy()
    o = p.origin[0]
    np.testing.assert_array_equal(full[o - r:o], full[o + n - r:o + n])
    np.testing.assert_array_equal(full[o + n:o + n + r], full[o:o + r])
    np.testing.assert_array_equal(p.download(a)[0], data)
    p.close()


def test_wide_xcorr_caller_halo(cuda_lib):
    r, n = 64, 9000
    g = _weights(r, True)
    p = L.Plan(1, (n,), r, 1, L.STENCIL_BC_CALLER, L.STENCIL_XCORR, L.STENCIL_F64, L.STENCIL_F64, coeffs=g)
    a, b = p.alloc(), p.alloc()
    fhat = synth.uniform(SEED, 7, n + 2 * r, -1.0, 1.0)
    import torch
    o = p.origin[0]
    p.view3(a[0])[0, 0, o - r:o + n + r] = torch.from_numpy(fhat).to(a[0].device)
    p.step(a, b, 1)
    p.sync()
    assert_close(p.download(b)[0], oracle.xcorr1d_box(fhat, g), 1e-12, "caller halo")
    p.close()


@pytest.mark.parametrize("storage", [L.STENCIL_I32, L.STENCIL_F32, L.STENCIL_F64])
@pytest.mark.parametrize("r,n,sweeps", [(0, 100, 1), (1, 4099, 3), (5, 70001, 2), (64, 9001, 1), (1024, 5000, 2),
                                        (1024, (1 << 20) + 1, 1)])
def test_maxfilter_is_exact(cuda_lib, storage, r, n, sweeps):
    if storage == L.STENCIL_I32:
        data = synth.integers(SEED, 300 + r, n, -2 ** 31, 2 ** 31 - 1).astype(np.int32)
    else:
        data = synth.normal(SEED, 300 + r, n)
        if storage == L.STENCIL_F32:
            data = data.astype(np.float32).astype(np.float64)
    p, a, b = _run(L.STENCIL_MAXFILTER, storage, n, r, data, sweeps=sweeps)
    got = p.download(b, dtype=None)[0] if storage == L.STENCIL_I32 else p.download(b)[0]
    ref = oracle.maxfilter1d(data, r, sweeps)
    assert np.array_equal(np.asarray(got).astype(ref.dtype), ref)
    full = p.view3(b[0])[0, 0].cpu().numpy()
    o = p.origin[0]
    if r:
        np.testing.assert_array_equal(full[o - r:o], full[o + n - r:o + n])
        np.testing.assert_array_equal(full[o + n:o + n + r], full[o:o + r])
    p.close()


def test_maxfilter_caller_halo(cuda_lib):
    r, n = 300, 20000
    p = L.Plan(1, (n,), r, 1, L.STENCIL_BC_CALLER, L.STENCIL_MAXFILTER, L.STENCIL_F32, L.STENCIL_F32)
    a, b = p.alloc(), p.alloc()
    fhat = synth.normal(SEED, 8, n + 2 * r).astype(np.float32)
    import torch
    o = p.origin[0]
    p.view3(a[0])[0, 0, o - r:o + n + r] = torch.from_numpy(fhat).to(a[0].device)
    p.step(a, b, 1)
    p.sync()
    assert np.array_equal(p.download(b)[0], oracle.maxfilter1d_box(fhat.astype(np.float64), r))
    p.close()


@pytest.mark.parametrize("r,n,sweeps", [(5, 9001, 14), (9, 4099, 8), (12, 70001, 13), (16, 2187, 5),
                                        (20, 5003, 7), (30, 4405, 4), (32, 50003, 3)])
def test_blocked_fp32_mid_radius(cuda_lib, r, n, sweeps):
    # FP32 radius 5..32 through the temporally blocked kernel: up to 1 + 60 / r sweeps per
    # launch, so these sweep counts need several launches; ragged chunks and short arrays
    g = _weights(r, False)
    data = synth.uniform(SEED, 400 + r, n, 0.0, 1.0).astype(np.float32).astype(np.float64)
    g = g.astype(np.float32).astype(np.float64)
    p, a, b = _run(L.STENCIL_XCORR, L.STENCIL_F32, n, r, data, coeffs=g, sweeps=sweeps)
    assert p.variant()[2] != "wide_register_blocked"
    assert_close(p.download(b)[0], oracle.xcorr1d(data, g, sweeps), 1e-5, f"r={r} sweeps={sweeps}")
    full = p.view3(b[0])[0, 0].double().cpu().numpy()
    o = p.origin[0]
    np.testing.assert_array_equal(full[o - r:o], full[o + n - r:o + n])
    np.testing.assert_array_equal(full[o + n:o + n + r], full[o:o + r])
    p.close()
    # caller-filled halo, one sweep
    p = L.Plan(1, (n,), r, 1, L.STENCIL_BC_CALLER, L.STENCIL_XCORR, L.STENCIL_F32, L.STENCIL_F32, coeffs=g)
    a, b = p.alloc(), p.alloc()
    fhat = synth.uniform(SEED, 500 + r, n + 2 * r, 0.0, 1.0).astype(np.float32)
    import torch
    o = p.origin[0]
    p.view3(a[0])[0, 0, o - r:o + n + r] = torch.from_numpy(fhat).to(a[0].device)
    p.step(a, b, 1)
    p.sync()
    assert_close(p.download(b)[0], oracle.xcorr1d_box(fhat.astype(np.float64), g), 1e-5, "caller halo")
    p.close()
