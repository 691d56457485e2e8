"""The autotuner (stencil_autotune, after the tuning protocol of Sec. 5.1): its search covers the
tile shape and, for the z-streaming 3D kernels, the z-chunk length; the winner is remembered per
problem class and GPU in the process and in the STENCIL_AUTOTUNE_CACHE file, and a remembered
choice is taken without timing anything; the serving batch takes its tile shapes from it.
Tiling never changes results: every z-chunk mode and every batched shape is bit-identical."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from gpu_util import heat_plan, mhd_plan
from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import serving, synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("kind,storage", [("heat", L.STENCIL_F64), ("heat", L.STENCIL_F32), ("mhd", L.STENCIL_F32),
                                          ("mhd", L.STENCIL_BF16)])
def test_every_zchunk_mode_is_bit_identical(cuda_lib, kind, storage):
    shape = (37, 20, 70)
    if kind == "heat":
        p, _ = heat_plan(shape, storage)
        init = [synth.heat_field(shape, seed=81)]
    else:
        p, _ = mhd_plan(shape, storage)
        init = synth.mhd_fields(shape, seed=81) * 20.0
    outs = []
    for z in range(3):
        p.set_zmode(z)
        a, b = p.alloc(), p.alloc()
        p.upload(a, init)
        p.step(a, b, 2)
        p.sync()
        outs.append([t.cpu() for t in b])
    for z in (1, 2):
        for q in range(p.nfields):
            assert torch.equal(outs[z][q], outs[0][q]), (z, q)
    with pytest.raises(L.StencilError):
        p.set_zmode(3)


def test_a_remembered_choice_is_taken_without_timing(cuda_lib, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("STENCIL_AUTOTUNE_CACHE", str(cache))
    shape = (48, 40, 64)
    p1, _ = heat_plan(shape, L.STENCIL_F32)
    a, b = p1.alloc(), p1.alloc()
    p1.upload(a, [synth.heat_field(shape, seed=82)])
    p1.autotune(a, b, nsteps=2, reps=1)
    from_cache, z1, ms1 = p1.autotune_status()
    assert not from_cache and 0 <= z1 < 3 and ms1 > 0
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split("\t")[1] == p1.variant()[2]
    # a second plan of the same class: the remembered choice, and fields_out is never written
    p2, _ = heat_plan(shape, L.STENCIL_F32)
    c, d = p2.alloc(), p2.alloc(fill=7.0)
    p2.upload(c, [synth.heat_field(shape, seed=82)])
    p2.autotune(c, d, nsteps=2, reps=1)
    assert p2.autotune_status()[:2] == (True, z1)
    assert p2.variant()[2] == p1.variant()[2]
    torch.cuda.synchronize()
    assert bool((d[0] == 7.0).all()), "a cache hit must not run the timing"
    assert len(cache.read_text().splitlines()) == 1
    # another process reads the file
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
            "from gpu_util import heat_plan\nfrom paper_2406_08923_gb300 import _lib as L\n"
            "p, _ = heat_plan((48, 40, 64), L.STENCIL_F32)\na, b = p.alloc(), p.alloc()\n"
            "p.autotune(a, b, nsteps=2, reps=1)\nprint(p.autotune_status()[0], p.variant()[2])\n"
            % (ROOT, os.path.join(ROOT, "tests")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, STENCIL_AUTOTUNE_CACHE=str(cache)))
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["True", p1.variant()[2]]


def _serve_one(kind, n, steps, templates):
    req = serving.Request(0, kind, n, steps)
    server = L.stencil_server_create(10 ** 10, 16)
    try:
        name = L.stencil_server_variant(server, kind)
    finally:
        L.stencil_server_destroy(server)
    serving.serve([req], templates, keep_outputs=True)
    return name, [t.numpy().copy() for t in req.out]


@pytest.mark.parametrize("kind,variants,names", [
    (L.STENCIL_MHD8, ("tx32_ty4_s8_b2", "tx32_ty12_s8_b1"), ("batch_tx32_ty4_s8", "batch_tx32_ty8_s8")),
    (L.STENCIL_DIFFUSION, ("f32_by4_ry2_zb2_s8_m3", "f32_by8_ry2_zb2_s8_m2"),
     ("batch_by4_ry2_zb2_s8", "batch_by8_ry2_zb2_s8"))])
def test_server_takes_the_tuned_tile_shape(cuda_lib, tmp_path, monkeypatch, kind, variants, names):
    # learn the problem-class key from one real tuning run, then offer each choice in its own file
    first = tmp_path / "first.txt"
    monkeypatch.setenv("STENCIL_AUTOTUNE_CACHE", str(first))
    shape = (24, 24, 24)
    p = mhd_plan(shape, L.STENCIL_F32)[0] if kind == L.STENCIL_MHD8 else heat_plan(shape, L.STENCIL_F32)[0]
    a, b = p.alloc(), p.alloc()
    p.autotune(a, b, nsteps=1, reps=1)
    key = first.read_text().splitlines()[-1].split("\t")[0]
    templates = serving.Templates(pinned=True)
    outs = []
    for i, (v, want) in enumerate(zip(variants, names)):
        f = tmp_path / f"c{i}.txt"
        f.write_text(f"{key}\t{v}\t0\t1.0\n")
        monkeypatch.setenv("STENCIL_AUTOTUNE_CACHE", str(f))
        name, out = _serve_one(kind, 29, 3, templates)
        assert name == want
        outs.append(out)
    for q in range(len(outs[0])):
        assert np.array_equal(outs[0][q], outs[1][q]), q
