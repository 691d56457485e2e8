"""Helpers shared by the GPU parity tests (error metrics, plan construction, samplers)."""
import numpy as np

from paper_2406_08923_gb300 import _lib as L

# Tolerances on relative L2 and relative L-infinity error against the FP64 oracle, per
# arithmetic: FP64 <= 1e-12, FP32 <= 1e-5, BF16 storage <= 1e-2.
TOL = {L.STENCIL_F64: 1e-12, L.STENCIL_F32: 1e-5, L.STENCIL_BF16: 1e-2}


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def rel_linf(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def assert_close(a, b, tol, what=""):
    e2, ei = rel_l2(a, b), rel_linf(a, b)
    assert e2 <= tol and ei <= tol, f"{what}: rel L2 {e2:.3e}, rel Linf {ei:.3e} > {tol:.0e}"
    return e2, ei


def periodic_box(f, center, half):
    """Cut the (2 half + 1)^3 neighbourhood of `center` (z, y, x) out of periodic f[..., z, y, x]."""
    idx = [np.arange(c - half, c + half + 1) % n for c, n in zip(center, f.shape[-3:])]
    return f[..., idx[0], :, :][..., :, idx[1], :][..., :, :, idx[2]]


def sample_cells(shape, rng_seed=0, extra=()):
    """Cells at faces, tile and z-chunk boundaries, plus a few seeded interior ones."""
    nz, ny, nx = shape
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz // 2, 0, nx - 1), (63 % nz, 31 % ny, 31 % nx),
           (64 % nz, 32 % ny, 32 % nx), (2, ny - 3, 1)]
    rng = np.random.default_rng(rng_seed)
    for _ in range(4):
        pts.append(tuple(int(rng.integers(0, n)) for n in shape))
    pts.extend(extra)
    return pts


def heat_plan(shape, dtype=L.STENCIL_F64, bc=L.STENCIL_BC_PERIODIC, params=None):
    nz, ny, nx = shape
    par = params or L.heat_params(shape)
    return L.Plan(3, (nx, ny, nz), 3, 1, bc, L.STENCIL_DIFFUSION, dtype, dtype, params=par), par


def mhd_plan(shape, storage=L.STENCIL_F64, **kw):
    nz, ny, nx = shape
    par = L.mhd_params(shape, **kw)
    compute = L.STENCIL_F64 if storage == L.STENCIL_F64 else L.STENCIL_F32
    return L.Plan(3, (nx, ny, nz), 3, 8, L.STENCIL_BC_PERIODIC, L.STENCIL_MHD8, storage, compute, params=par), par


def oracle_mhd_params(par):
    import oracle
    return oracle.MhdParams(dx=par.dx[0], dy=par.dx[1], dz=par.dx[2], cs0=par.cs0, gamma=par.gamma,
                            cp=par.cp, lnrho0=par.lnrho0, nu=par.nu, eta=par.eta, zeta=par.zeta,
                            mu0=par.mu0, K=par.K)
