"""The allocation-free norm entry point (stencil_field_norms_noalloc).

It serves callers that cannot allocate device memory, such as a serving loop whose HBM
budget is fully committed, or an application whose device memory belongs to another
allocator.  Its scratch is a fixed device array inside the library.  This file is collected
last, so a run that stops at the first failure has already run every other test.  It must
pass both alone in a fresh process and after the other tests.

Each call is checked through the C ABI against stencil_field_norms, the plan-based entry
point, within the norm tests' tolerance.  Two calls are made in a row, on different
workloads, so a stale value left in the shared array would show.
"""
import gc

import numpy as np
import pytest
import torch

from gpu_util import heat_plan, mhd_plan
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(p, fields, mass_volume, out=None):
    n = 3 * len(fields) + (1 if mass_volume > 0 else 0)
    if out is None:
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    L.stencil_field_norms_noalloc(fields, p.storage, p.dims, p.padded, p.origin, mass_volume, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_matches_plan_entry_point_two_calls_in_a_row(cuda_lib):
    # call 1: the 8-field MHD state (BF16 storage) with the mass term
    shape = (20, 24, 28)
    p1, par = mhd_plan(shape, L.STENCIL_BF16)
    f1 = p1.alloc(fill=3.0)
    p1.upload(f1, synth.mhd_fields(shape, seed=4))
    ref1 = p1.norms(f1)
    got1 = _noalloc(p1, f1, par.dx[0] * par.dx[1] * par.dx[2])
    np.testing.assert_allclose(got1, ref1, rtol=1e-12, atol=1e-14 * np.abs(ref1).max())

    # call 2: one FP64 heat field of another shape, no mass term
    shape2 = (37, 41, 29)
    p2, _ = heat_plan(shape2, L.STENCIL_F64)
    f2 = p2.alloc(fill=1e6)
    p2.upload(f2, [synth.heat_field(shape2, seed=2)])
    ref2 = p2.norms(f2)
    got2 = _noalloc(p2, f2, 0.0)
    np.testing.assert_allclose(got2, ref2, rtol=1e-12, atol=1e-14 * np.abs(ref2).max())


def test_rejects_more_fields_than_the_static_scratch_holds(cuda_lib):
    shape = (16, 16, 16)
    p, _ = heat_plan(shape, L.STENCIL_F64)
    f = p.alloc()
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(L.StencilError) as e:
        L.stencil_field_norms_noalloc(f * 9, p.storage, p.dims, p.padded, p.origin, 0.0, out)
    assert e.value.status == L.STENCIL_EINVAL
    assert "at most 8 fields" in str(e.value)


def test_a_call_allocates_no_device_memory(cuda_lib):
    # the property the entry point exists for: after a warm-up call (which loads the kernels and
    # looks up the scratch array's address), a call leaves the device's free memory and
    # PyTorch's allocator untouched
    shape = (40, 36, 44)
    p, par = mhd_plan(shape, L.STENCIL_F32)
    f = p.alloc()
    p.upload(f, synth.mhd_fields(shape, seed=6))
    vol = par.dx[0] * par.dx[1] * par.dx[2]
    out = torch.full((25,), float("nan"), dtype=torch.float64, device="cuda")
    first = _noalloc(p, f, vol, out)
    # tensors of earlier tests freed by the cyclic garbage collector inside the measured window
    # would change the counts: collect them first and keep the collector off meanwhile
    gc.collect()
    gc.disable()
    try:
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        L.stencil_field_norms_noalloc(f, p.storage, p.dims, p.padded, p.origin, vol, out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        alloc1 = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    assert alloc1 == alloc0
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    np.testing.assert_array_equal(out.cpu().numpy(), first)
