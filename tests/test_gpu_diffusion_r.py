"""GPU parity of the diffusion radius sweep (Sec. 5.3): the forward-Euler step with the
order-2r central Laplacian, r = 1..4, in 1D, 2D and 3D, FP64 and FP32, through the C ABI,
against the FP64 oracle (`oracle.diffusion_r`).

Bars: FP64 relative L2 and L-infinity <= 1e-12; FP32 <= 1e-5 (against the FP64 oracle started
from the same FP32-rounded field).
"""
import numpy as np
import pytest

import oracle
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth

from gpu_util import assert_close

pytestmark = pytest.mark.gpu

SEED = 2406089236
TOL = {L.STENCIL_F64: 1e-12, L.STENCIL_F32: 1e-5}
SHAPES = {1: (4099,), 2: (45, 70), 3: (21, 29, 37)}  # dense (.., ny, nx), ragged against every tile


def _field(shape, storage):
    n = int(np.prod(shape))
    f = synth.uniform(SEED, len(shape), n, -1.0, 1.0).reshape(shape)
    if storage == L.STENCIL_F32:
        f = f.astype(np.float32).astype(np.float64)
    return f


def _plan(shape, r, storage, bc=L.STENCIL_BC_PERIODIC):
    dims = tuple(reversed(shape))  # (nx, ny, nz)
    return L.Plan(len(shape), dims, r, 1, bc, L.STENCIL_DIFFUSION, storage, storage, params=L.heat_params(shape))


def _h(par, ndim):
    return (par.dx[0], par.dx[1], par.dx[2])  # absent axes are never differentiated


@pytest.mark.parametrize("storage", [L.STENCIL_F64, L.STENCIL_F32])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_radius_sweep_matches_oracle(cuda_lib, ndim, r, storage):
    shape = SHAPES[ndim]
    p = _plan(shape, r, storage)
    a, b = p.alloc(), p.alloc()
    f = _field(shape, storage)
    p.upload(a, [f])
    steps = 17 if ndim == 1 else 3  # 1D: more than one temporally blocked launch
    p.step(a, b, steps)
    p.sync()
    got = p.download(b)[0]
    par = p.params
    ref = oracle.diffusion_r(f, r, par.dt, par.alpha, _h(par, ndim), steps)
    assert_close(got, ref, TOL[storage], f"{ndim}D r={r}")
    # the input interior is not modified
    np.testing.assert_array_equal(p.download(a)[0], f)
    p.close()


@pytest.mark.parametrize("storage", [L.STENCIL_F64, L.STENCIL_F32])
@pytest.mark.parametrize("r", [1, 4])
@pytest.mark.parametrize("ndim", [2, 3])
def test_output_halo_is_the_periodic_image(cuda_lib, ndim, r, storage):
    shape = SHAPES[ndim]
    p = _plan(shape, r, storage)
    a, b = p.alloc(), p.alloc()
    p.upload(a, [_field(shape, storage)])
    p.step(a, b, 2)
    p.sync()
    full = p.view3(b[0]).double().cpu().numpy()
    ox, oy, oz = p.origin
    nx, ny, nz = p.dims
    hz = r if ndim == 3 else 0
    box = full[oz - hz:oz + nz + hz, oy - r:oy + ny + r, ox - r:ox + nx + r]
    inner = box[hz:hz + nz, r:r + ny, r:r + nx]
    want = np.pad(inner, ((hz, hz), (r, r), (r, r)), mode="wrap")
    np.testing.assert_array_equal(box, want)
    p.close()


@pytest.mark.parametrize("r", [2, 4])
@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_caller_filled_halo_one_step(cuda_lib, ndim, r):
    # non-periodic: the caller fills the halo; one step reads it as given
    shape = {1: (257,), 2: (47, 70), 3: (23, 31, 37)}[ndim]
    storage = L.STENCIL_F64
    p = _plan(shape, r, storage, bc=L.STENCIL_BC_CALLER)
    a, b = p.alloc(), p.alloc()
    ox, oy, oz = p.origin
    nx, ny, nz = p.dims
    hy, hz = (r if ndim >= 2 else 0), (r if ndim == 3 else 0)
    bshape = (nz + 2 * hz, ny + 2 * hy, nx + 2 * r)
    boxv = synth.uniform(SEED, 9, int(np.prod(bshape)), -1.0, 1.0).reshape(bshape)
    import torch
    v = p.view3(a[0])
    v[oz - hz:oz + nz + hz, oy - hy:oy + ny + hy, ox - r:ox + nx + r] = torch.from_numpy(boxv).to(v.device)
    p.step(a, b, 1)
    p.sync()
    got = p.download(b)[0]
    par = p.params
    fhat = boxv.reshape(bshape[3 - ndim:]) if ndim < 3 else boxv
    ref = oracle.diffusion_r_box(fhat, r, par.dt, par.alpha, _h(par, ndim), shape)
    assert_close(got, ref, 1e-12, f"caller halo {ndim}D r={r}")
    p.close()


@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("shape,steps", [((45, 72), 9), ((37, 12), 5), ((300, 1024), 6)])
def test_2d_every_variant_matches_oracle(cuda_lib, r, shape, steps):
    # FP32 2D: the one-step tile kernel and the temporally blocked streaming kernels (2 and 4
    # steps per pass, the remainder one step at a time).  nx is a multiple of 4 so the blocked
    # variants run; the shapes overhang a strip (72, 12 < 104 cells), wrap rows more than once
    # (ny = 37 < 2 K r + chunk) and span several strips and row chunks (1024 x 300).
    storage = L.STENCIL_F32
    p = _plan(shape, r, storage)
    nv = p.variant()[1]
    assert nv == 3
    f = _field(shape, storage)
    par = p.params
    ref = oracle.diffusion_r(f, r, par.dt, par.alpha, _h(par, 2), steps)
    ox, oy, _ = p.origin
    nx, ny, _ = p.dims
    for v in range(nv):
        p.set_variant(v)
        a, b = p.alloc(), p.alloc()
        p.upload(a, [f])
        p.step(a, b, steps)
        p.sync()
        assert_close(p.download(b)[0], ref, TOL[storage], f"2D r={r} {shape} variant {p.variant()[2]}")
        full = p.view3(b[0])[0].double().cpu().numpy()
        box = full[oy - r:oy + ny + r, ox - r:ox + nx + r]
        want = np.pad(box[r:r + ny, r:r + nx], ((r, r), (r, r)), mode="wrap")
        np.testing.assert_array_equal(box, want)
        np.testing.assert_array_equal(p.download(a)[0], f)
    p.close()


@pytest.mark.parametrize("variant", [1, 2])
def test_2d_blocked_variants_fall_back(cuda_lib, variant):
    # the temporally blocked variants need periodic boundaries and nx a multiple of 4; otherwise
    # they run the one-step kernel, with the same results
    r = 3
    shape = (45, 70)  # nx = 70
    p = _plan(shape, r, L.STENCIL_F32)
    p.set_variant(variant)
    f = _field(shape, L.STENCIL_F32)
    a, b = p.alloc(), p.alloc()
    p.upload(a, [f])
    p.step(a, b, 5)
    p.sync()
    par = p.params
    assert_close(p.download(b)[0], oracle.diffusion_r(f, r, par.dt, par.alpha, _h(par, 2), 5), TOL[L.STENCIL_F32],
                 f"variant {variant}, nx = 70")
    p.close()
    # caller-filled halo, nx a multiple of 4: one step, read as given
    shape = (47, 72)
    p = _plan(shape, r, L.STENCIL_F32, bc=L.STENCIL_BC_CALLER)
    p.set_variant(variant)
    a, b = p.alloc(), p.alloc()
    ox, oy, _ = p.origin
    nx, ny, _ = p.dims
    boxv = synth.uniform(SEED, 11, (ny + 2 * r) * (nx + 2 * r), -1.0, 1.0).reshape(ny + 2 * r, nx + 2 * r)
    boxv = boxv.astype(np.float32).astype(np.float64)
    import torch
    v = p.view3(a[0])
    v[0, oy - r:oy + ny + r, ox - r:ox + nx + r] = torch.from_numpy(boxv).to(v.device, torch.float32)
    p.step(a, b, 1)
    p.sync()
    par = p.params
    ref = oracle.diffusion_r_box(boxv, r, par.dt, par.alpha, _h(par, 2), shape)
    assert_close(p.download(b)[0], ref, TOL[L.STENCIL_F32], f"variant {variant}, caller halo")
    p.close()
