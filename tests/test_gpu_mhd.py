"""GPU parity of the fused 8-field MHD step (Eqs. A1-A4, 6th-order derivatives, RK3).

* The right-hand side alone (stencil_mhd_rhs) against the oracle on ragged multi-tile grids,
  for every storage type and kernel variant (the BF16/FP32 kernels see the same rounded
  inputs as the oracle, so the RHS must agree to FP32 accuracy).
* Whole RK3 steps against the oracle: FP64 within 1e-12; FP32 and BF16 storage with
  Kahan-compensated accumulation within 1e-5 and 1e-2 of the FP64 oracle after every one of
  20 steps.
* Full benchmark sizes (256^3 FP64, 384^3 FP32/BF16): one step on sampled cells against the
  oracle's neighbourhood-box evaluation.
* Closed form: a uniform state stays uniform (all derivatives vanish).
* The heat-conduction term of A3 (K != 0): RHS and RK3 steps against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import (TOL, assert_close, mhd_plan, oracle_mhd_params, periodic_box, rel_l2,
                      sample_cells)
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth

pytestmark = pytest.mark.gpu

STORAGE = (L.STENCIL_F64, L.STENCIL_F32, L.STENCIL_BF16)


def _rounded(f8, storage):
    """The fields as the GPU stores them (FP64 view of the rounded values)."""
    t = torch.from_numpy(f8)
    if storage == L.STENCIL_F32:
        t = t.float()
    elif storage == L.STENCIL_BF16:
        t = t.to(torch.bfloat16)
    return t.double().numpy()


@pytest.mark.parametrize("storage", STORAGE)
@pytest.mark.parametrize("shape", [(16, 16, 16), (70, 13, 45)])
def test_rhs_against_oracle(cuda_lib, storage, shape):
    f8 = synth.mhd_fields(shape, seed=21) * 20.0
    p, par = mhd_plan(shape, storage)
    a = p.alloc()
    p.upload(a, f8)
    ref = oracle.mhd_rhs(_rounded(f8, storage), oracle_mhd_params(par))
    ctype = torch.float64 if storage == L.STENCIL_F64 else torch.float32
    tol = 1e-12 if storage == L.STENCIL_F64 else 1e-5
    for v in range(p.variant()[1]):
        p.set_variant(v)
        rhs = [torch.zeros(shape, dtype=ctype, device="cuda") for _ in range(8)]
        p.mhd_rhs(a, rhs)
        p.sync()
        errs = [assert_close(rhs[q].double().cpu().numpy(), ref[q], tol, f"variant {v} field {q}")
                for q in range(8)]
        print(f"rhs {shape} storage {storage} variant {v}: worst rel L2 / Linf per field "
              + " ".join(f"{e2:.2e}/{ei:.2e}" for e2, ei in errs))


def test_uniform_state_is_stationary(cuda_lib):
    shape = (16, 16, 16)
    f8 = np.empty((8,) + shape)
    for q, v in enumerate((0.2, 0.5, -0.3, 0.1, 1.0, -2.0, 0.7, 0.4)):
        f8[q] = v
    p, par = mhd_plan(shape)
    a = p.alloc()
    p.upload(a, f8)
    rhs = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(8)]
    p.mhd_rhs(a, rhs)
    p.sync()
    assert max(float(r.abs().max()) for r in rhs) < 1e-13


@pytest.mark.parametrize("shape,steps", [((32, 32, 32), 3), ((70, 13, 45), 2)])
def test_f64_steps_against_oracle(cuda_lib, shape, steps):
    f8 = synth.mhd_fields(shape, seed=5) * 20.0
    p, par = mhd_plan(shape)
    ref = oracle.mhd_rk3(f8, oracle_mhd_params(par), par.dt, steps)
    for v in range(p.variant()[1]):
        p.set_variant(v)
        a, b = p.alloc(), p.alloc()
        p.upload(a, f8)
        p.step(a, b, steps)
        p.sync()
        got = p.download(b)
        for q in range(8):
            assert_close(got[q], ref[q], 1e-12, f"variant {v} field {q}")
            # the increment itself, a much stricter view than the state
            assert rel_l2(got[q] - f8[q], ref[q] - f8[q]) < 1e-10


@pytest.mark.parametrize("storage", (L.STENCIL_F32, L.STENCIL_BF16))
def test_low_precision_storage_every_step(cuda_lib, storage):
    shape, nsteps = (48, 48, 48), 20
    f8 = synth.mhd_fields(shape, seed=synth.SEED_MHD_LOWP)
    p, par = mhd_plan(shape, storage)
    op = oracle_mhd_params(par)
    ref = f8.copy()
    a, b = p.alloc(), p.alloc()
    p.upload(a, f8)
    worst = 0.0
    for k in range(1, nsteps + 1):
        ref = oracle.mhd_rk3(ref, op, par.dt, 1)
        p.step(a, b, k)  # from the initial state, so Kahan terms span the whole run
        got = p.download(b)
        for q in range(8):
            e2, ei = assert_close(got[q], ref[q], TOL[storage], f"step {k} field {q}")
            worst = max(worst, e2, ei)
    m0 = oracle.mass(f8[0])
    m1 = p.norms(b)[-1] / (par.dx[0] * par.dx[1] * par.dx[2])
    assert abs(m1 - m0) / m0 < 1e-3
    print(f"worst relative error over {nsteps} steps: {worst:.3e}")


@pytest.mark.parametrize("storage,n", [(L.STENCIL_F64, 256), (L.STENCIL_F32, 384), (L.STENCIL_BF16, 384)])
def test_full_size_step_sampled(cuda_lib, storage, n):
    shape = (n, n, n)
    seed = synth.SEED_MHD if storage == L.STENCIL_F64 else synth.SEED_MHD_LOWP
    f8 = synth.mhd_fields(n, seed=seed)
    p, par = mhd_plan(shape, storage)
    a, b = p.alloc(), p.alloc()
    p.upload(a, f8)
    p.step(a, b, 1)
    p.sync()
    fin = _rounded(f8, storage)
    op = oracle_mhd_params(par)
    got = [p.interior(t) for t in b]
    for cell in sample_cells(shape, extra=((n - 1, 0, 0), (0, n - 1, 33))):
        box = periodic_box(fin, cell, 9)
        ref = oracle.mhd_rk3_box(box, op, par.dt, 3)[:, 9, 9, 9]
        g = np.array([float(t[cell]) for t in got])
        scale = np.abs(fin).reshape(8, -1).max(axis=1)
        tol = TOL[storage]
        assert np.all(np.abs(g - ref) <= tol * scale + 1e-300), (cell, g, ref)


@pytest.mark.parametrize("storage", STORAGE)
def test_heat_conduction_rhs_against_oracle(cuda_lib, storage):
    shape = (20, 17, 35)
    f8 = synth.mhd_fields(shape, seed=31) * 20.0
    p, par = mhd_plan(shape, storage, K=0.05)
    a = p.alloc()
    p.upload(a, f8)
    ref = oracle.mhd_rhs(_rounded(f8, storage), oracle_mhd_params(par))
    ref0 = oracle.mhd_rhs(_rounded(f8, storage), oracle_mhd_params(L.mhd_params(shape)))
    assert rel_l2(ref[7] - ref0[7], ref0[7]) > 1e-3  # the term is not negligible in this case
    ctype = torch.float64 if storage == L.STENCIL_F64 else torch.float32
    tol = 1e-12 if storage == L.STENCIL_F64 else 1e-5
    for v in range(p.variant()[1]):
        p.set_variant(v)
        rhs = [torch.zeros(shape, dtype=ctype, device="cuda") for _ in range(8)]
        p.mhd_rhs(a, rhs)
        p.sync()
        for q in range(8):
            assert_close(rhs[q].double().cpu().numpy(), ref[q], tol, f"K, variant {v} field {q}")


def test_heat_conduction_steps_against_oracle(cuda_lib):
    shape = (24, 24, 24)
    f8 = synth.mhd_fields(shape, seed=32) * 20.0
    for storage in (L.STENCIL_F64, L.STENCIL_F32):
        p, par = mhd_plan(shape, storage, K=0.05)
        ref = oracle.mhd_rk3(_rounded(f8, storage), oracle_mhd_params(par), par.dt, 3)
        a, b = p.alloc(), p.alloc()
        p.upload(a, f8)
        p.step(a, b, 3)
        p.sync()
        got = p.download(b)
        for q in range(8):
            assert_close(got[q], ref[q], TOL[storage], f"K, storage {storage} field {q}")


@pytest.mark.parametrize("storage", (L.STENCIL_F32, L.STENCIL_BF16))
@pytest.mark.parametrize("nx", (70, 71, 72))
def test_every_variant_is_bit_identical(cuda_lib, storage, nx):
    # every variant performs the same IEEE operations per cell (only the tile shape and the ring
    # differ), so whole RK3 steps agree bit for bit, periodic images included; every width
    # (odd and even) overhangs the tiles
    shape = (40, 20, nx)
    f8 = synth.mhd_fields(shape, seed=41) * 20.0
    p, par = mhd_plan(shape, storage)
    outs = []
    for v in range(p.variant()[1]):
        p.set_variant(v)
        a, b = p.alloc(), p.alloc()
        p.upload(a, f8)
        p.step(a, b, 2)
        p.sync()
        outs.append((p.variant()[2], [t.cpu() for t in b]))
    for name, fields in outs[1:]:
        for q in range(8):
            assert torch.equal(fields[q], outs[0][1][q]), (name, q)
