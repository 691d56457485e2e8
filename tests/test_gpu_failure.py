"""Failure detection on the GPU without a fault: a bounded device wait that nothing
completes runs out, the kernel records the expiry and returns, the host reads
STENCIL_ETIMEOUT at the next sync, and the context and plan stay usable."""
import time

import numpy as np
import pytest

import oracle
from gpu_util import heat_plan
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth

pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_plan_recovers(cuda_lib):
    shape = (16, 16, 16)
    p, par = heat_plan(shape, L.STENCIL_F64)
    t0 = time.perf_counter()
    p.selftest_wait(2_000_000)  # 2 ms
    with pytest.raises(L.StencilError) as e:
        p.sync()
    assert e.value.status == L.STENCIL_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    p.sync()  # the error word was cleared
    # the plan still computes correct results afterwards
    f0 = synth.heat_field(shape, seed=1)
    a, b = p.alloc(), p.alloc()
    p.upload(a, [f0])
    p.step(a, b, 2)
    p.sync()
    h = (par.dx[0], par.dx[1], par.dx[2])
    ref = oracle.diffusion(f0, par.dt, par.alpha, h, 2)
    np.testing.assert_allclose(p.download(b)[0], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_timeout_is_also_reported_by_norms(cuda_lib):
    p, _ = heat_plan((8, 8, 8), L.STENCIL_F64)
    a = p.alloc()
    p.selftest_wait(1_000)
    with pytest.raises(L.StencilError) as e:
        p.norms(a)
    assert e.value.status == L.STENCIL_ETIMEOUT
    p.norms(a)
