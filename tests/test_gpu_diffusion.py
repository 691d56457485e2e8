"""GPU parity of the 3D heat-equation step (Eqs. 4-7) against the oracle.

Small and ragged grids: full comparison with the oracle after several steps, for every
kernel variant.  Full size (256^3, 100 steps, the benchmark's launch configuration): the
discrete single-mode closed form (holds at any size), the conservation of sum f and decay
of sum f^2 on the seeded field, and one step on sampled cells against the oracle's box
evaluation.
"""
import numpy as np
import pytest

import oracle
from gpu_util import TOL, assert_close, heat_plan, periodic_box, sample_cells
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth
from symbols import lam2

pytestmark = pytest.mark.gpu

DT = (L.STENCIL_F64, L.STENCIL_F32)


def _steps(shape, dtype, nsteps, f0, variant=None):
    p, par = heat_plan(shape, dtype)
    if variant is not None:
        p.set_variant(variant)
    a, b = p.alloc(), p.alloc()
    p.upload(a, [f0])
    p.step(a, b, nsteps)
    p.sync()
    return p.download(b)[0], p, par, (a, b)


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("shape", [(32, 32, 32), (70, 19, 67), (7, 9, 8)])
def test_against_oracle(cuda_lib, dtype, shape):
    f0 = synth.heat_field(shape, seed=11)
    if dtype == L.STENCIL_F32:
        f0 = f0.astype(np.float32).astype(np.float64)
    p, par = heat_plan(shape, dtype)
    nv = p.variant()[1]
    h = (par.dx[0], par.dx[1], par.dx[2])
    ref = oracle.diffusion(f0, par.dt, par.alpha, h, 5)
    for v in range(nv):
        got, *_ = _steps(shape, dtype, 5, f0, variant=v)
        assert_close(got, ref, TOL[dtype], f"variant {v} shape {shape}")


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("shape", [(20, 21, 22), (40, 48, 128), (7, 16, 64)])
def test_halo_images_and_input_untouched(cuda_lib, dtype, shape):
    f0 = synth.heat_field(shape, seed=3)
    got, p, par, (a, b) = _steps(shape, dtype, 1, f0)
    whole = p.view3(b[0]).double().cpu().numpy()
    ox, oy, oz = p.origin
    nz, ny, nx = shape
    box = whole[oz - 3:oz + nz + 3, oy - 3:oy + ny + 3, ox - 3:ox + nx + 3]
    np.testing.assert_array_equal(box, np.pad(got, 3, mode="wrap"))
    kept = p.download(a)[0]
    ref = f0 if dtype == L.STENCIL_F64 else f0.astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(kept, ref)


def test_caller_halo_quadratic_exact(cuda_lib):
    # lap(x^2 + 2 y^2 - z^2 + xy) = 4; the caller fills the halo with the polynomial itself
    n, h = 12, 0.25
    par = L.heat_params(n)
    par.dx[0] = par.dx[1] = par.dx[2] = h
    par.dt, par.alpha = 0.01, 3.0
    p, _ = heat_plan((n, n, n), L.STENCIL_F64, bc=L.STENCIL_BC_CALLER, params=par)
    a, b = p.alloc(), p.alloc()
    ox, oy, oz = p.origin
    px, py, pz = p.padded
    cx = (np.arange(px) - ox) * h
    cy = (np.arange(py) - oy) * h
    cz = (np.arange(pz) - oz) * h
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    f = X ** 2 + 2 * Y ** 2 - Z ** 2 + X * Y
    import torch
    p.view3(a[0]).copy_(torch.from_numpy(f))
    p.step(a, b, 1)
    p.sync()
    got = p.download(b)[0]
    exp = f[oz:oz + n, oy:oy + n, ox:ox + n] + par.dt * par.alpha * 4.0
    np.testing.assert_allclose(got, exp, atol=1e-12)


@pytest.mark.parametrize("dtype", DT)
def test_full_size_single_mode_closed_form(cuda_lib, dtype):
    n, steps = 256, 100
    h = 2 * np.pi / n
    k = (3, 5, 2)
    c = np.arange(n) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f0 = np.sin(k[0] * X + k[1] * Y + k[2] * Z + 0.25)
    got, p, par, _ = _steps((n, n, n), dtype, steps, f0)
    amp = (1 + par.dt * par.alpha * sum(lam2(kk, h) for kk in k)) ** steps
    assert amp < 0.999
    assert_close(got, amp * f0, TOL[dtype], "single mode")


@pytest.mark.parametrize("dtype", DT)
def test_full_size_seeded_field(cuda_lib, dtype):
    n, steps = 256, 100
    f0 = synth.heat_field(n)
    p, par = heat_plan((n, n, n), dtype)
    a, b = p.alloc(), p.alloc()
    p.upload(a, [f0])
    n0 = p.norms(a)
    p.step(a, b, 1)
    one = p.download(b)[0]
    h = (par.dx[0], par.dx[1], par.dx[2])
    f0s = f0 if dtype == L.STENCIL_F64 else f0.astype(np.float32).astype(np.float64)
    for cell in sample_cells((n, n, n)):
        box = periodic_box(f0s, cell, 4)  # 9^3 box = 3^3 interior + halo 3
        ref = oracle.diffusion_box(box, par.dt, par.alpha, h, (3, 3, 3))[1, 1, 1]
        got = one[cell]
        assert abs(got - ref) <= TOL[dtype] * np.abs(f0s).max(), (cell, got, ref)
    p.step(a, b, steps)
    n1 = p.norms(b)
    # sum f conserved (weights of the 2nd derivative sum to zero), sum f^2 decays
    assert abs(n1[0] - n0[0]) <= (1e-12 if dtype == L.STENCIL_F64 else 1e-5) * n ** 3
    assert n1[1] < n0[1]
