"""Persistent multi-step schedule of the FP32 3D heat step (Eqs. 4-7, nsteps steps in one launch).

The persistent variants run the same per-cell arithmetic as the one-launch-per-step variants of
the same tile shape, so their results must be bit-identical to them, periodic images included;
both are checked against the oracle too.  The cases cover:
- several units per CTA (more units than resident CTAs);
- z-chunks shorter than the radius, where the cells beyond one face belong to several units;
- ragged tiles;
- repeated calls and a switch of the z-chunk mode on one plan (the sync words carry an epoch
  across calls and grow with the unit count);
- the full-size 256^3 x 100-step configuration.
"""
import numpy as np
import pytest

import oracle
from gpu_util import TOL, assert_close, heat_plan
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth

pytestmark = pytest.mark.gpu


def _variants(p):
    """(per-step variant, persistent variant) pairs of the same tile shape."""
    n = p.variant()[1]
    names = []
    for v in range(n):
        p.set_variant(v)
        names.append(p.variant()[2])
    pairs = [(names.index(nm[:-len("_persist")]), v) for v, nm in enumerate(names) if nm.endswith("_persist")]
    assert pairs, names
    return pairs


def _run(p, f0, nsteps, variant, zmode=0):
    p.set_variant(variant)
    p.set_zmode(zmode)
    a, b = p.alloc(), p.alloc()
    p.upload(a, [f0])
    p.step(a, b, nsteps)
    p.sync()
    whole = p.view3(b[0]).cpu().numpy().copy()
    kept = p.download(a)[0]
    return whole, kept


def _interior(p, whole, shape):
    ox, oy, oz = p.origin
    nz, ny, nx = shape
    return whole[oz:oz + nz, oy:oy + ny, ox:ox + nx].astype(np.float64)


@pytest.mark.parametrize("shape,nsteps,zmode", [
    ((32, 32, 32), 5, 0), ((70, 19, 67), 4, 0), ((7, 9, 8), 6, 0),
    ((7, 16, 64), 5, 1),       # one-plane z-chunks: the cells beyond a z face span three units
    ((64, 128, 512), 3, 1),    # 13 z-chunks x 64 tiles: more units than resident CTAs
])
def test_bit_identical_to_per_step_schedule(cuda_lib, shape, nsteps, zmode):
    f0 = synth.heat_field(shape, seed=5).astype(np.float32).astype(np.float64)
    p, par = heat_plan(shape, L.STENCIL_F32)
    ref = oracle.diffusion(f0, par.dt, par.alpha, (par.dx[0], par.dx[1], par.dx[2]), nsteps)
    for v_step, v_pers in _variants(p):
        w_step, _ = _run(p, f0, nsteps, v_step, zmode)
        w_pers, kept = _run(p, f0, nsteps, v_pers, zmode)
        name = p.variant()[2]
        np.testing.assert_array_equal(w_pers, w_step, err_msg=f"{name} shape {shape}")  # images too
        np.testing.assert_array_equal(kept, f0, err_msg=f"{name}: input modified")
        assert_close(_interior(p, w_pers, shape), ref, TOL[L.STENCIL_F32], f"{name} shape {shape}")


def test_repeated_calls_and_zmode_switch(cuda_lib):
    # one plan, one pair of buffers: the epoch of the sync words advances across calls, and a
    # larger unit count (z-chunk mode 1) grows them between calls
    shape = (40, 24, 130)
    f0 = synth.heat_field(shape, seed=9).astype(np.float32).astype(np.float64)
    p, par = heat_plan(shape, L.STENCIL_F32)
    v_step, v_pers = _variants(p)[0]
    a, b = p.alloc(), p.alloc()
    p.upload(a, [f0])
    h = (par.dx[0], par.dx[1], par.dx[2])
    cur = f0
    for i, (nsteps, zmode) in enumerate([(3, 0), (1, 0), (4, 1), (2, 2), (5, 0)]):
        p.set_variant(v_pers)
        p.set_zmode(zmode)
        src, dst = (a, b) if i % 2 == 0 else (b, a)
        p.step(src, dst, nsteps)
        p.sync()
        got = p.download(dst)[0]
        ref = oracle.diffusion(cur, par.dt, par.alpha, h, nsteps)
        assert_close(got, ref, TOL[L.STENCIL_F32], f"call {i}: {nsteps} steps, zmode {zmode}")
        # same call through the per-step variant on copies: bit-identical
        q, _ = heat_plan(shape, L.STENCIL_F32)
        q.set_variant(v_step)
        q.set_zmode(zmode)
        qa, qb = q.alloc(), q.alloc()
        q.upload(qa, [cur.astype(np.float32).astype(np.float64)])
        q.step(qa, qb, nsteps)
        q.sync()
        np.testing.assert_array_equal(got, q.download(qb)[0], err_msg=f"call {i}")
        cur = got


@pytest.mark.slow
def test_full_size_persistent_matches_per_step(cuda_lib):
    n, steps = 256, 100
    f0 = synth.heat_field(n).astype(np.float32).astype(np.float64)
    p, par = heat_plan((n, n, n), L.STENCIL_F32)
    v_step, v_pers = _variants(p)[0]
    w_step, _ = _run(p, f0, steps, v_step)
    w_pers, _ = _run(p, f0, steps, v_pers)
    np.testing.assert_array_equal(w_pers, w_step)
    ref = oracle.diffusion(f0, par.dt, par.alpha, (par.dx[0], par.dx[1], par.dx[2]), steps)
    assert_close(_interior(p, w_pers, (n, n, n)), ref, TOL[L.STENCIL_F32], "256^3 x 100, persistent")
