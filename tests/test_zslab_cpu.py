"""Z-slab decomposition on CPU ranks: the host logic of paper_2406_08923_gb300/zslab.py.

Two and three gloo ranks (127.0.0.1) each own a z-slab of one periodic grid in the oracle's
padded layout.  Before every pass they exchange their z halos with DistTransport, the same
code that moves the halos between GPUs, fill their x/y images, and run the oracle's own box
evaluation on the slab: the heat step of Eq. 4 (oracle.diffusion_box) and the MHD right-hand
side of Eqs. A1-A4 (oracle.mhd_rhs_box) with the 2N-storage RK3 update.  The slabs put back
together must equal the single-domain oracle (oracle.diffusion, oracle.mhd_rk3) -- bit for
bit, since every cell sees the same values and the same arithmetic -- and the all-reduced
norms must equal the whole grid's.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R = 3
RK_A = (0.0, -5.0 / 9.0, -153.0 / 128.0)
RK_B = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fill_xy(box):
    """x/y periodic images of every plane of a padded (pz, py, px) box from its own cells."""
    inner = box[:, R:-R, R:-R].copy()
    box[:] = np.pad(inner, ((0, 0), (R, R), (R, R)), mode="wrap")


def _worker(rank, world, port, kind, shape, steps, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2406_08923_gb300 import synth
    from paper_2406_08923_gb300.zslab import DistTransport, SlabPlanes, slab_bounds

    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    nz, ny, nx = shape
    z0, z1 = slab_bounds(nz, world, rank, R)
    nzl = z1 - z0
    padded = (nx + 2 * R, ny + 2 * R, nzl + 2 * R)
    planes = SlabPlanes(padded, R, nzl, R)
    tr = DistTransport(rank, world)
    nf = 8 if kind == "mhd" else 1
    whole = synth.mhd_fields(shape, seed=51) * 20.0 if kind == "mhd" else synth.heat_field(shape, seed=52)[None]
    fields = [torch.zeros(padded[0] * padded[1] * padded[2], dtype=torch.float64) for _ in range(nf)]

    def box(t):
        return t.numpy().reshape(padded[2], padded[1], padded[0])

    for q in range(nf):
        box(fields[q])[R:R + nzl, R:-R, R:-R] = whole[q][z0:z1]
    h = (2 * np.pi / nx, 2 * np.pi / ny, 2 * np.pi / nz)
    if kind == "heat":
        dt = 0.1 * min(h) ** 2
        for _ in range(steps):
            tr.exchange(planes, fields)
            b = box(fields[0])
            _fill_xy(b)
            b[R:R + nzl, R:-R, R:-R] = oracle.diffusion_box(b, dt, 1.0, h, (nzl, ny, nx))
    else:
        par = oracle.MhdParams.for_grid(shape)
        dt = par.dt_default()
        w = np.zeros((8, nzl, ny, nx))
        for _ in range(steps):
            for s in range(3):
                tr.exchange(planes, fields)
                boxes = [box(t) for t in fields]
                for b in boxes:
                    _fill_xy(b)
                rhs = oracle.mhd_rhs_box(np.stack(boxes), par)
                w = RK_A[s] * w + dt * rhs
                for q in range(8):
                    inner = boxes[q][R:R + nzl, R:-R, R:-R]
                    inner[:] = inner + RK_B[s] * w[q]
    res = np.stack([box(t)[R:R + nzl, R:-R, R:-R].copy() for t in fields])
    local = np.concatenate([oracle.norms(res[q]) for q in range(nf)])
    norms = tr.allreduce_norms(local, nf)
    np.save(os.path.join(out_dir, f"slab{rank}.npy"), res)
    np.save(os.path.join(out_dir, f"norms{rank}.npy"), norms)
    dist.barrier()
    dist.destroy_process_group()


def _run(kind, shape, steps, world, tmp_path):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, kind, shape, steps, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    slabs = [np.load(tmp_path / f"slab{r}.npy") for r in range(world)]
    norms = [np.load(tmp_path / f"norms{r}.npy") for r in range(world)]
    return np.concatenate(slabs, axis=1), norms


def test_slab_bounds_cover_the_grid():
    from paper_2406_08923_gb300.zslab import slab_bounds
    for nz, world in ((256, 8), (20, 3), (21, 2), (9, 3), (384, 7)):
        b = [slab_bounds(nz, world, r) for r in range(world)]
        assert b[0][0] == 0 and b[-1][1] == nz
        assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
        sizes = [z1 - z0 for z0, z1 in b]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= R
    with pytest.raises(ValueError):
        slab_bounds(8, 3, 0)  # 2-plane slabs are thinner than the radius
    with pytest.raises(ValueError):
        slab_bounds(16, 2, 2)


@pytest.mark.parametrize("world", (2, 3))
def test_heat_slabs_equal_the_single_domain_oracle(tmp_path, world):
    import oracle
    from paper_2406_08923_gb300 import synth
    shape, steps = (20, 11, 13), 3
    got, norms = _run("heat", shape, steps, world, tmp_path)
    f0 = synth.heat_field(shape, seed=52)
    h = (2 * np.pi / shape[2], 2 * np.pi / shape[1], 2 * np.pi / shape[0])
    ref = oracle.diffusion(f0, 0.1 * min(h) ** 2, 1.0, h, steps)
    np.testing.assert_array_equal(got[0], ref)
    whole = oracle.norms(ref)
    for nr in norms:
        np.testing.assert_allclose(nr[:2], whole[:2], rtol=1e-13)
        assert nr[2] == whole[2]


@pytest.mark.parametrize("world", (2, 3))
def test_mhd_slabs_equal_the_single_domain_oracle(tmp_path, world):
    import oracle
    from paper_2406_08923_gb300 import synth
    shape, steps = (16, 9, 10), 2
    got, norms = _run("mhd", shape, steps, world, tmp_path)
    f8 = synth.mhd_fields(shape, seed=51) * 20.0
    par = oracle.MhdParams.for_grid(shape)
    ref = oracle.mhd_rk3(f8, par, par.dt_default(), steps)
    np.testing.assert_array_equal(got, ref)
    for nr in norms:
        for q in range(8):
            whole = oracle.norms(ref[q])
            scale = np.abs(ref[q]).sum()
            assert abs(nr[3 * q] - whole[0]) <= 1e-13 * scale
            assert nr[3 * q + 1] == pytest.approx(whole[1], rel=1e-13)
            assert nr[3 * q + 2] == whole[2]
