"""stencil_step_host: the step with the fields in host memory (one C-ABI call copies in, steps,
copies out and synchronises) equals stencil_step on device fields, bit for bit."""
import numpy as np
import pytest
import torch

from gpu_util import heat_plan, mhd_plan
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ("heat_f64", "heat_f32", "mhd_bf16"))
def test_host_buffers_equal_device_step(cuda_lib, kind):
    shape = (21, 18, 35)
    if kind.startswith("heat"):
        p, _ = heat_plan(shape, L.STENCIL_F64 if kind == "heat_f64" else L.STENCIL_F32)
        init = [synth.heat_field(shape, seed=71)]
    else:
        p, _ = mhd_plan(shape, L.STENCIL_BF16)
        init = synth.mhd_fields(shape, seed=71) * 20.0
    a, b = p.alloc(), p.alloc()
    p.upload(a, init)
    host_in = [t.cpu().pin_memory() for t in a]
    host_out = [torch.full_like(t, 7, device="cpu").pin_memory() for t in a]
    p.step(a, b, 3)
    p.sync()
    ref = [t.cpu() for t in b]
    d_in, d_out = p.alloc(fill=5), p.alloc(fill=5)
    p.step_host(host_in, host_out, d_in, d_out, 3)
    for q in range(p.nfields):
        got = p.interior(host_out[q])
        assert torch.equal(got, p.interior(ref[q])), q


def test_host_call_rejects_null_host_fields(cuda_lib):
    p, _ = heat_plan((12, 12, 12))
    d_in, d_out = p.alloc(), p.alloc()
    (pi, ki), (po, ko) = L._ptrs(d_in), L._ptrs(d_out)
    st = L.load().stencil_step_host(p.h, None, None, pi, po, 1, L._stream(None))
    assert st == L.STENCIL_EINVAL
    assert "NULL" in L.load().stencil_last_error_detail(p.h).decode()
