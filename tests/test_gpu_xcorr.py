"""GPU parity of the 1D cross-correlation (Eq. 3) against the oracle.

int32 is compared bit for bit (arithmetic modulo 2^32); FP64/FP32 within 1e-12 / 1e-5
relative.  Covers the full benchmark size (2^20 cells, 10 sweeps), ragged tails, the minimum
periodic extent, radius 0..4, caller-filled halos, zero steps and multi-launch sweeps.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_close
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth

pytestmark = pytest.mark.gpu

D2 = np.array([1 / 90, -3 / 20, 3 / 2, -49 / 18, 3 / 2, -3 / 20, 1 / 90])


def _run(data, g, sweeps, dtype, bc=L.STENCIL_BC_PERIODIC, halo=None):
    n = len(data)
    r = (len(g) - 1) // 2
    p = L.Plan(1, (n,), r, 1, bc, L.STENCIL_XCORR, dtype, dtype, coeffs=g)
    a, b = p.alloc(), p.alloc(fill=7)
    p.upload(a, [data])
    if halo is not None:  # caller-filled halo: write f^ around the interior
        ox = p.origin[0]
        full = p.view3(a[0])[0, 0]
        import torch
        full[ox - r:ox].copy_(torch.from_numpy(halo[0]).to(full.dtype))
        full[ox + n:ox + n + r].copy_(torch.from_numpy(halo[1]).to(full.dtype))
    p.step(a, b, sweeps)
    p.sync()
    out = p.interior(b[0]).cpu().numpy()
    whole = p.view3(b[0])[0, 0].cpu().numpy()
    return out, whole, p, p.interior(a[0]).cpu().numpy()


@pytest.mark.parametrize("n", [1 << 20, 4099, 2048, 7, 2053])
def test_int32_bit_exact(cuda_lib, n):
    data, g = synth.xcorr_int32(n)
    out, whole, p, kept = _run(data, g, 10, L.STENCIL_I32)
    assert np.array_equal(out, oracle.xcorr1d(data, g, 10))
    # the input interior is untouched and the output halo holds the periodic image (Eq. 2)
    assert np.array_equal(kept, data)
    ox = p.origin[0]
    assert np.array_equal(whole[ox - 3:ox], out[-3:]) and np.array_equal(whole[ox + n:ox + n + 3], out[:3])


@pytest.mark.parametrize("r", [0, 1, 2, 3, 4])
def test_int32_all_radii(cuda_lib, r):
    data, _ = synth.xcorr_int32(3001, seed=r + 1)
    g = synth.integers(99, r, 2 * r + 1, -8, 8).astype(np.int32)
    out, *_ = _run(data, g, 5, L.STENCIL_I32)
    assert np.array_equal(out, oracle.xcorr1d(data, g, 5))


@pytest.mark.parametrize("sweeps", [0, 1, 16, 17, 35])
def test_int32_sweep_counts(cuda_lib, sweeps):
    data, g = synth.xcorr_int32(5000, seed=3)
    out, *_ = _run(data, g, sweeps, L.STENCIL_I32)
    ref = data if sweeps == 0 else oracle.xcorr1d(data, g, sweeps)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("n", [1 << 20, 3333])
def test_f64_second_derivative_weights(cuda_lib, n):
    x = synth.xcorr_f64(n)
    out, *_ = _run(x, D2, 10, L.STENCIL_F64)
    assert_close(out, oracle.xcorr1d(x, D2, 10), 1e-12, "xcorr f64")


def test_f32(cuda_lib):
    x = synth.xcorr_f64(100003).astype(np.float32)
    g = np.array([0.1, -0.2, 0.3, 0.5, 0.3, -0.2, 0.1])
    out, *_ = _run(x, g, 10, L.STENCIL_F32)
    assert_close(out, oracle.xcorr1d(x.astype(np.float64), g, 10), 1e-5, "xcorr f32")


def test_caller_halo_single_sweep(cuda_lib):
    n = 2500
    x = synth.xcorr_f64(n, seed=4)
    halo = (synth.uniform(8, 1, 3, -5, 5), synth.uniform(8, 2, 3, -5, 5))
    out, *_ = _run(x, D2, 1, L.STENCIL_F64, bc=L.STENCIL_BC_CALLER, halo=halo)
    fhat = np.concatenate([halo[0], x, halo[1]])
    assert_close(out, oracle.xcorr1d_box(fhat, D2), 1e-13, "caller halo")
    with pytest.raises(L.StencilError):
        _run(x, D2, 2, L.STENCIL_F64, bc=L.STENCIL_BC_CALLER, halo=halo)


def test_minimum_extent_wraps_several_times(cuda_lib):
    data, g = synth.xcorr_int32(7, seed=9)
    out, *_ = _run(data, g, 16, L.STENCIL_I32)
    assert np.array_equal(out, oracle.xcorr1d(data, g, 16))


@pytest.mark.parametrize("dtype", [L.STENCIL_I32, L.STENCIL_F32, L.STENCIL_F64])
def test_large_grid_full_blocks(cuda_lib, dtype):
    # 2^21 + 5 cells: many chunks and a ragged tail (FP64: two whole waves of 512-thread CTAs
    # with 3450-cell chunks).  16 + 3 sweeps: two launches.
    n = (1 << 21) + 5
    if dtype == L.STENCIL_I32:
        data, g = synth.xcorr_int32(n)
    else:
        data = synth.uniform(2406089231, 9, n, -1.0, 1.0)
        g = D2
        if dtype == L.STENCIL_F32:
            data = data.astype(np.float32).astype(np.float64)
            g = D2.astype(np.float32).astype(np.float64)
    out, whole, p, _ = _run(data, g, 19, dtype)
    ref = oracle.xcorr1d(data, g, 19)
    if dtype == L.STENCIL_I32:
        assert np.array_equal(out, ref)
    else:
        assert_close(out, ref, 1e-12 if dtype == L.STENCIL_F64 else 1e-5, "2^21 + 5")
    ox = p.origin[0]
    np.testing.assert_array_equal(whole[ox - 3:ox], whole[ox + n - 3:ox + n])
    np.testing.assert_array_equal(whole[ox + n:ox + n + 3], whole[ox:ox + 3])
    p.close()


def test_f64_past_l2_runs_the_256_thread_chunks(cuda_lib):
    # 2^23 + 3 FP64 cells: input and output (134 MB) exceed 7/8 of L2, so the launches take
    # 2048-cell chunks in 256-thread CTAs instead of whole waves of 512-thread CTAs.  Ragged
    # tail, 16 + 3 sweeps in two launches, and the periodic images of both ends.
    n = (1 << 23) + 3
    data = synth.uniform(2406089233, 9, n, -1.0, 1.0)
    out, whole, p, _ = _run(data, D2, 19, L.STENCIL_F64)
    assert_close(out, oracle.xcorr1d(data, D2, 19), 1e-12, "2^23 + 3")
    ox = p.origin[0]
    np.testing.assert_array_equal(whole[ox - 3:ox], whole[ox + n - 3:ox + n])
    np.testing.assert_array_equal(whole[ox + n:ox + n + 3], whole[ox:ox + 3])
    p.close()
