"""FP64 CPU oracle for the stencil engine -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline`` /
``--impl reference`` legs may import this package.  The library under
``paper_2406_08923_gb300`` never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, double precision, ``-ffp-contract=off``,
OpenMP over the outermost loop); this module compiles it with gcc on first use and marshals
numpy arrays.  Each wrapper names the passage of the paper it evaluates.  Parity of every
function is pinned in ``tests/test_oracle_*.py`` against closed forms, polynomial exactness,
library routines and brute force, never against the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

R = 3  # radius of the 6th-order central differences (Sec. 3.3)


def build(force: bool = False, src: str | None = None, lib: str | None = None) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FMA contraction, OpenMP).

    `src` / `lib` default to this package's source and library; the planted-mistake tests pass
    a mutated copy of the source and a library path in a temporary directory."""
    src = src or _SRC
    lib = lib or _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True, capture_output=True)
        os.replace(tmp, lib)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            D = ctypes.c_double
            sig = {
                "oracle_pad_periodic_f64": (None, [P, I64, I64, I64, I, P]),
                "oracle_xcorr1d_box_f64": (None, [P, I64, P, I, P]),
                "oracle_xcorr1d_box_u32": (None, [P, I64, P, I, P]),
                "oracle_xcorr1d_f64": (I, [P, I64, P, I, I, P]),
                "oracle_xcorr1d_u32": (I, [P, I64, P, I, I, P]),
                "oracle_derivs_box": (None, [P, I64, I64, I64, P, P]),
                "oracle_diffusion_box": (None, [P, I64, I64, I64, D, D, P, P]),
                "oracle_diffusion": (I, [P, I64, I64, I64, D, D, P, I, P]),
                "oracle_diffusion_r_box": (I, [P, I64, I64, I64, I, D, D, P, P]),
                "oracle_maxfilter1d_box_f64": (None, [P, I64, I, P]),
                "oracle_maxfilter1d_box_i32": (None, [P, I64, I, P]),
                "oracle_maxfilter1d_f64": (I, [P, I64, I, I, P]),
                "oracle_maxfilter1d_i32": (I, [P, I64, I, I, P]),
                "oracle_diffusion_r": (I, [P, I64, I64, I64, I, D, D, P, I, P]),
                "oracle_mhd_rhs_box": (None, [P, I64, I64, I64, P, P]),
                "oracle_mhd_rk3": (I, [P, I64, I64, I64, P, D, I]),
                "oracle_mhd_rk3_box": (I, [P, I64, I64, I64, P, D, I]),
                "oracle_norms": (None, [P, I64, P]),
                "oracle_mass": (D, [P, I64]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _dims3(shape):
    """(nx, ny, nz) of a dense (nz, ny, nx) / (ny, nx) / (nx,) array."""
    s = tuple(shape)
    s = (1,) * (3 - len(s)) + s
    return s[2], s[1], s[0]


# ----------------------------------------------------------------- Eq. 2 (padding)


def pad_periodic(f: np.ndarray, r: int = R) -> np.ndarray:
    """f^ of Eq. 2 with the periodic boundary function (axes of extent 1 get no halo)."""
    f = _c(f, np.float64)
    nx, ny, nz = _dims3(f.shape)
    h = lambda n: n + 2 * r if n > 1 else 1
    out = np.empty(tuple(h(n) for n in (nz, ny, nx))[3 - f.ndim:], dtype=np.float64)
    _load().oracle_pad_periodic_f64(_p(f), nx, ny, nz, r, _p(out))
    return out


# ------------------------------------------------------ Eq. 3 (cross-correlation)


def xcorr1d_box(fhat: np.ndarray, g: np.ndarray) -> np.ndarray:
    """One sweep of Eq. 3 over a padded 1D array (caller-filled halo of width r)."""
    g = np.asarray(g)
    r = (len(g) - 1) // 2
    n = len(fhat) - 2 * r
    if np.asarray(fhat).dtype.kind in "iu":
        fh = _c(np.asarray(fhat).astype(np.int64) & 0xFFFFFFFF, np.uint32)
        out = np.empty(n, dtype=np.uint32)
        _load().oracle_xcorr1d_box_u32(_p(fh), n, _p(_c(g, np.int32)), r, _p(out))
        return out.view(np.int32)
    fh = _c(fhat, np.float64)
    out = np.empty(n, dtype=np.float64)
    _load().oracle_xcorr1d_box_f64(_p(fh), n, _p(_c(g, np.float64)), r, _p(out))
    return out


def xcorr1d(data: np.ndarray, g: np.ndarray, sweeps: int = 1) -> np.ndarray:
    """`sweeps` periodic sweeps of Eq. 3.  int32 data use arithmetic modulo 2**32."""
    g = np.asarray(g)
    r = (len(g) - 1) // 2
    n = len(data)
    lib = _load()
    if np.asarray(data).dtype.kind in "iu":
        d = _c(np.asarray(data).astype(np.int64) & 0xFFFFFFFF, np.uint32)
        out = np.empty(n, dtype=np.uint32)
        rc = lib.oracle_xcorr1d_u32(_p(d), n, _p(_c(g, np.int32)), r, sweeps, _p(out))
        assert rc == 0
        return out.view(np.int32)
    d = _c(data, np.float64)
    out = np.empty(n, dtype=np.float64)
    rc = lib.oracle_xcorr1d_f64(_p(d), n, _p(_c(g, np.float64)), r, sweeps, _p(out))
    assert rc == 0
    return out


# -------------------------------------------------- Sec. 3.3 (central differences)


def maxfilter1d_box(fhat: np.ndarray, r: int) -> np.ndarray:
    """One max-filter sweep f'_i = max_{j=-r..r} f^_{i+j} over a padded 1D array (caller halo of
    width r).  int32 data stay int32; anything else is evaluated in FP64."""
    fhat = np.asarray(fhat)
    n = len(fhat) - 2 * r
    if fhat.dtype.kind in "iu":
        fh = _c(fhat, np.int32)
        out = np.empty(n, dtype=np.int32)
        _load().oracle_maxfilter1d_box_i32(_p(fh), n, r, _p(out))
        return out
    fh = _c(fhat, np.float64)
    out = np.empty(n, dtype=np.float64)
    _load().oracle_maxfilter1d_box_f64(_p(fh), n, r, _p(out))
    return out


def maxfilter1d(data: np.ndarray, r: int, sweeps: int = 1) -> np.ndarray:
    """`sweeps` periodic max-filter sweeps (the nonlinear stencil of Sec. 2.1)."""
    data = np.asarray(data)
    n = len(data)
    if data.dtype.kind in "iu":
        d = _c(data, np.int32)
        out = np.empty(n, dtype=np.int32)
        assert _load().oracle_maxfilter1d_i32(_p(d), n, r, sweeps, _p(out)) == 0
        return out
    d = _c(data, np.float64)
    out = np.empty(n, dtype=np.float64)
    assert _load().oracle_maxfilter1d_f64(_p(d), n, r, sweeps, _p(out)) == 0
    return out


def derivs_box(fhat: np.ndarray, h) -> np.ndarray:
    """9 derivative fields (dx, dy, dz, dxx, dyy, dzz, dxy, dxz, dyz) at the interior of a
    padded 3D box with halo 3 on every axis; h = (dx, dy, dz)."""
    fhat = _c(fhat, np.float64)
    pz, py, px = fhat.shape
    nx, ny, nz = px - 2 * R, py - 2 * R, pz - 2 * R
    out = np.empty((9, nz, ny, nx), dtype=np.float64)
    _load().oracle_derivs_box(_p(fhat), nx, ny, nz, _p(_c(h, np.float64)), _p(out))
    return out


# ----------------------------------------------------------- Eq. 4 (diffusion)


def diffusion_box(fhat: np.ndarray, dt: float, alpha: float, h, interior_shape) -> np.ndarray:
    """One Euler step of Eq. 4 on a padded box; returns the interior."""
    fhat = _c(fhat, np.float64)
    nx, ny, nz = _dims3(interior_shape)
    out = np.empty(tuple(interior_shape), dtype=np.float64)
    _load().oracle_diffusion_box(_p(fhat), nx, ny, nz, dt, alpha, _p(_c(h, np.float64)), _p(out))
    return out


def diffusion_r_box(fhat: np.ndarray, r: int, dt: float, alpha: float, h, interior_shape) -> np.ndarray:
    """One Euler step with the radius-r (order 2r) Laplacian on a padded box (halo r on every
    axis of extent > 1); returns the interior."""
    fhat = _c(fhat, np.float64)
    nx, ny, nz = _dims3(interior_shape)
    out = np.empty(tuple(interior_shape), dtype=np.float64)
    rc = _load().oracle_diffusion_r_box(_p(fhat), nx, ny, nz, r, dt, alpha, _p(_c(h, np.float64)), _p(out))
    assert rc == 0, "radius must be 1..4"
    return out


def diffusion_r(f: np.ndarray, r: int, dt: float, alpha: float, h, steps: int) -> np.ndarray:
    """`steps` periodic forward-Euler steps with the radius-r Laplacian (radius sweep of the
    diffusion equation, Sec. 5.3), in 1, 2 or 3 dimensions."""
    f = _c(f, np.float64)
    nx, ny, nz = _dims3(f.shape)
    out = np.empty_like(f)
    rc = _load().oracle_diffusion_r(_p(f), nx, ny, nz, r, dt, alpha, _p(_c(h, np.float64)), steps, _p(out))
    assert rc == 0, "radius must be 1..4"
    return out


def diffusion(f: np.ndarray, dt: float, alpha: float, h, steps: int) -> np.ndarray:
    """`steps` periodic forward-Euler steps of the diffusion equation (Eq. 4)."""
    f = _c(f, np.float64)
    nx, ny, nz = _dims3(f.shape)
    out = np.empty_like(f)
    rc = _load().oracle_diffusion(_p(f), nx, ny, nz, dt, alpha, _p(_c(h, np.float64)), steps,
                                  _p(out))
    assert rc == 0
    return out


# --------------------------------------------------- Appendix A (MHD) + RK3


@dataclass
class MhdParams:
    """Constants of Eqs. A1-A4.  The paper prints none of them; these are the readings."""
    dx: float
    dy: float
    dz: float
    cs0: float = 1.0
    gamma: float = 5.0 / 3.0
    cp: float = 1.0
    lnrho0: float = 0.0
    nu: float = 5e-3
    eta: float = 5e-3
    zeta: float = 0.0
    mu0: float = 1.0
    K: float = 0.0  # heat conductivity of A3 (0: the benchmark configuration)

    @classmethod
    def for_grid(cls, n, **kw):
        nz, ny, nx = (n, n, n) if np.isscalar(n) else tuple(n)
        tau = 2.0 * np.pi
        return cls(dx=tau / nx, dy=tau / ny, dz=tau / nz, **kw)

    def array(self) -> np.ndarray:
        return np.array([self.dx, self.dy, self.dz, self.cs0, self.gamma, self.cp, self.lnrho0,
                         self.nu, self.eta, self.zeta, self.mu0, self.K], dtype=np.float64)

    def dt_default(self) -> float:
        """dt = 0.1 * min grid spacing (Table B2, PyTorch MHD row)."""
        return 0.1 * min(self.dx, self.dy, self.dz)


def mhd_rhs_box(fhat8: np.ndarray, par: MhdParams) -> np.ndarray:
    """RHS of Eqs. A1-A4 at the interior of 8 padded boxes (8, nz+6, ny+6, nx+6)."""
    fhat8 = _c(fhat8, np.float64)
    _, pz, py, px = fhat8.shape
    nx, ny, nz = px - 2 * R, py - 2 * R, pz - 2 * R
    out = np.empty((8, nz, ny, nx), dtype=np.float64)
    fp = (ctypes.c_void_p * 8)(*[fhat8[q].ctypes.data for q in range(8)])
    op = (ctypes.c_void_p * 8)(*[out[q].ctypes.data for q in range(8)])
    _load().oracle_mhd_rhs_box(ctypes.cast(fp, ctypes.c_void_p), nx, ny, nz,
                               _p(par.array()), ctypes.cast(op, ctypes.c_void_p))
    return out


def mhd_rhs(f8: np.ndarray, par: MhdParams) -> np.ndarray:
    """RHS of Eqs. A1-A4 on the periodic grid."""
    return mhd_rhs_box(np.stack([pad_periodic(f8[q]) for q in range(8)]), par)


def mhd_rk3(f8: np.ndarray, par: MhdParams, dt: float, steps: int) -> np.ndarray:
    """`steps` periodic RK3 steps (3 substeps each) of the MHD system; returns a new array."""
    f = _c(f8, np.float64).copy()
    nz, ny, nx = f.shape[1:]
    rc = _load().oracle_mhd_rk3(_p(f), nx, ny, nz, _p(par.array()), dt, steps)
    assert rc == 0
    return f


def mhd_rk3_box(box8: np.ndarray, par: MhdParams, dt: float, nsub: int = 3) -> np.ndarray:
    """`nsub` RK3 substeps on a non-periodic neighbourhood box (8, mz, my, mx); only the box
    shrunk by 3*nsub cells on every side holds advanced values on return."""
    f = _c(box8, np.float64).copy()
    mz, my, mx = f.shape[1:]
    rc = _load().oracle_mhd_rk3_box(_p(f), mx, my, mz, _p(par.array()), dt, nsub)
    assert rc == 0
    return f


# ----------------------------------------------------------------------- norms


def norms(f: np.ndarray) -> np.ndarray:
    """(sum f, sum f^2, max |f|) accumulated in long double."""
    f = _c(f, np.float64).ravel()
    out = np.empty(3, dtype=np.float64)
    _load().oracle_norms(_p(f), f.size, _p(out))
    return out


def mass(lnrho: np.ndarray) -> float:
    """sum exp(lnrho) (multiply by the cell volume for the physical mass)."""
    f = _c(lnrho, np.float64).ravel()
    return float(_load().oracle_mass(_p(f), f.size))
