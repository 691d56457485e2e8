"""Edge cases of the step entry point, against the oracle.

* Zero steps: stencil_step copies the input and fills the periodic halo (Eq. 2), so the
  output is the input's augmented array, for every kind.
* The minimum periodic extent 2r + 1 = 7 on every axis (the halo then wraps almost the whole
  interior): 3D heat for every kernel variant, and the 8-field MHD system (Eqs. A1-A4, RK3).
* Arrays beyond 4 GiB, where a 32-bit byte offset would overflow: a heat field of 1024^3 FP32
  (4.4 GB padded), and the MHD RK register and Kahan terms at 512^3 FP32 (4.3 GB each).  The input is a product of three 1D sines, an exact eigenfunction
  of the discrete operator of Eq. 7.  It is built on the device as the product of three FP32
  vectors that the host computed.  The host forms the same FP32 products for the boxes around
  sampled cells, and the oracle steps them (box evaluation).  The discrete closed form is a
  second, independent check.  The MHD fields are products of 1D factors too, advanced by the
  oracle's box RK3 around sampled cells.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL, assert_close, heat_plan, mhd_plan, oracle_mhd_params, sample_cells
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth
from symbols import lam2

pytestmark = pytest.mark.gpu


def _whole(p, fields):
    return [p.view3(t).double().cpu().numpy() for t in fields]


def _box(p, arr, shape, r=3):
    ox, oy, oz = p.origin
    nz, ny, nx = shape
    return arr[oz - r:oz + nz + r, oy - r:oy + ny + r, ox - r:ox + nx + r]


@pytest.mark.parametrize("dtype", (L.STENCIL_F64, L.STENCIL_F32))
def test_zero_steps_heat_copies_and_fills_halo(cuda_lib, dtype):
    shape = (20, 21, 22)
    f0 = synth.heat_field(shape, seed=8)
    if dtype == L.STENCIL_F32:
        f0 = f0.astype(np.float32).astype(np.float64)
    p, _ = heat_plan(shape, dtype)
    a, b = p.alloc(), p.alloc(fill=7.0)
    p.upload(a, [f0])
    p.step(a, b, 0)
    p.sync()
    np.testing.assert_array_equal(_box(p, _whole(p, b)[0], shape), oracle.pad_periodic(f0))


def test_zero_steps_mhd_copies_and_fills_halo(cuda_lib):
    shape = (9, 10, 11)
    p, _ = mhd_plan(shape, L.STENCIL_F32)
    f8 = synth.mhd_fields(shape, seed=12).astype(np.float32).astype(np.float64)
    a, b = p.alloc(), p.alloc(fill=-3.0)
    p.upload(a, f8)
    p.step(a, b, 0)
    p.sync()
    got = _whole(p, b)
    for q in range(8):
        np.testing.assert_array_equal(_box(p, got[q], shape), oracle.pad_periodic(f8[q]), err_msg=f"field {q}")


@pytest.mark.parametrize("dtype", (L.STENCIL_F64, L.STENCIL_F32))
def test_minimum_extent_heat_every_variant(cuda_lib, dtype):
    shape = (7, 7, 7)
    f0 = synth.heat_field(shape, seed=21)
    if dtype == L.STENCIL_F32:
        f0 = f0.astype(np.float32).astype(np.float64)
    p, par = heat_plan(shape, dtype)
    ref = oracle.diffusion(f0, par.dt, par.alpha, (par.dx[0], par.dx[1], par.dx[2]), 3)
    for v in range(p.variant()[1]):
        p.set_variant(v)
        a, b = p.alloc(), p.alloc()
        p.upload(a, [f0])
        p.step(a, b, 3)
        p.sync()
        assert_close(p.download(b)[0], ref, TOL[dtype], f"variant {p.variant()[2]}")


@pytest.mark.parametrize("storage", (L.STENCIL_F64, L.STENCIL_F32))
def test_minimum_extent_mhd_every_variant(cuda_lib, storage):
    shape = (7, 7, 7)
    p, par = mhd_plan(shape, storage)
    f8 = synth.mhd_fields(shape, seed=23)
    if storage != L.STENCIL_F64:
        f8 = f8.astype(np.float32).astype(np.float64)
    ref = oracle.mhd_rk3(f8, oracle_mhd_params(par), par.dt, 1)
    for v in range(p.variant()[1]):
        p.set_variant(v)
        a, b = p.alloc(), p.alloc()
        p.upload(a, f8)
        p.step(a, b, 1)
        p.sync()
        got = p.download(b)
        for q in range(8):
            assert_close(got[q], ref[q], TOL[storage], f"variant {p.variant()[2]} field {q}")


@pytest.mark.slow
def test_heat_1024_fp32_beyond_4_gib(cuda_lib):
    n, steps = 1024, 2
    p, par = heat_plan((n, n, n), L.STENCIL_F32)
    h = (par.dx[0], par.dx[1], par.dx[2])
    k = (5, 3, 7)  # wavenumbers along x, y, z
    phase = (0.3, 0.1, 0.2)
    vec = [np.sin(k[a] * h[a] * np.arange(n) + phase[a]).astype(np.float32) for a in range(3)]
    vx, vy, vz = vec
    a, b = p.alloc(), p.alloc()
    ox, oy, oz = p.origin
    dev = [torch.from_numpy(v).cuda() for v in vec]
    p.view3(a[0])[oz:oz + n, oy:oy + n, ox:ox + n] = dev[2][:, None, None] * dev[1][None, :, None] * dev[0][None, None, :]
    del dev
    p.step(a, b, steps)
    p.sync()
    out = p.view3(b[0])
    amp = (1 + par.dt * par.alpha * sum(lam2(kk, hh) for kk, hh in zip(k, h))) ** steps
    assert amp < 0.9999
    # the oracle steps a box around each sampled cell; the last step keeps a 3^3 interior (an
    # axis of extent 1 would count as absent there), whose centre is the cell
    half = 3 * steps + 1
    for cell in sample_cells((n, n, n), extra=[(n - 1, 511, 512), (700, n - 2, 1)]):
        z, y, x = cell
        iz, iy, ix = [np.arange(c - half, c + half + 1) % n for c in cell]
        # the device's FP32 products, formed the same way on the host: (vz * vy) * vx
        box = ((vz[iz][:, None, None] * vy[iy][None, :, None]) * vx[ix][None, None, :]).astype(np.float64)
        ref = box
        for s in range(steps):
            m = 2 * half + 1 - 6 * (s + 1)
            ref = oracle.diffusion_box(ref, par.dt, par.alpha, h, (m, m, m))
        got = float(out[oz + z, oy + y, ox + x])
        assert abs(got - ref[1, 1, 1]) <= TOL[L.STENCIL_F32], (cell, got, ref[1, 1, 1])
        exact = amp * float(vz[z]) * float(vy[y]) * float(vx[x])
        assert abs(got - exact) <= 2 * TOL[L.STENCIL_F32], (cell, got, exact)


@pytest.mark.slow
def test_mhd_512_fp32_rk_scratch_beyond_4_gib(cuda_lib):
    # 512^3 with FP32 storage: the RK register and the Kahan terms (8 values per cell, one array
    # each) are 4.3 GB, so their offsets 8 cell + q pass 2^32.  Every field is a product of three
    # 1D factors built on the device; the oracle advances boxes around sampled cells (three RK3
    # substeps shrink a 21^3 box to its central 3^3).
    n = 512
    p, par = mhd_plan((n, n, n), L.STENCIL_F32)
    h = par.dx[0]
    i = np.arange(n)
    # (offset, amplitude) per field: lnrho and s near 1, velocity ~ 0.2^3, vector potential ~ 0.1^3
    scale = [(1.0, 0.05), (0.2, 0.06), (0.2, 0.06), (0.2, 0.06), (0.1, 0.03), (0.1, 0.03), (0.1, 0.03),
             (1.0, 0.05)]
    fac = [[(c + s * np.sin((q + ax + 1) * h * i + 0.1 * (q + 3 * ax))).astype(np.float32) for ax in range(3)]
           for q, (c, s) in enumerate(scale)]  # fac[q] = [x factor, y factor, z factor]
    a, b = p.alloc(), p.alloc()
    ox, oy, oz = p.origin
    for q in range(8):
        fx, fy, fz = [torch.from_numpy(v).cuda() for v in fac[q]]
        p.view3(a[q])[oz:oz + n, oy:oy + n, ox:ox + n] = (fz[:, None, None] * fy[None, :, None]) * fx[None, None, :]
        del fx, fy, fz
    p.step(a, b, 1)
    p.sync()
    opar = oracle_mhd_params(par)
    half = 3 * 3 + 1
    for cell in sample_cells((n, n, n), extra=[(n - 1, 255, 256), (300, n - 2, 1)]):
        z, y, x = cell
        iz, iy, ix = [np.arange(c - half, c + half + 1) % n for c in cell]
        box8 = np.stack([((fz[iz][:, None, None] * fy[iy][None, :, None]) * fx[ix][None, None, :]).astype(np.float64)
                         for fx, fy, fz in fac])
        ref = oracle.mhd_rk3_box(box8, opar, par.dt, 3)[:, half, half, half]
        for q in range(8):
            got = float(p.view3(b[q])[oz + z, oy + y, ox + x])
            tol = TOL[L.STENCIL_F32] * np.abs(box8[q]).max()
            assert abs(got - ref[q]) <= tol, (cell, q, got, ref[q])
