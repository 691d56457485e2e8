"""ctypes binding of libstencil.so (include/stencil.h).

Argument marshalling only: every step of the stencil path runs in the library's CUDA
kernels.  The functions keep the C names (stencil_create, stencil_step, ...); ``Plan`` is a
small convenience wrapper that owns a handle and allocates fields with PyTorch according to
``stencil_layout``.  PyTorch provides device memory and streams, nothing else.

There is no fallback: if libstencil.so is missing or fails to load, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstencil.so")

# enums (include/stencil.h)
STENCIL_OK, STENCIL_EINVAL, STENCIL_ENOMEM, STENCIL_ECUDA, STENCIL_EUNSUPPORTED, STENCIL_ETIMEOUT = range(6)
STENCIL_I32, STENCIL_F64, STENCIL_F32, STENCIL_BF16 = range(4)
STENCIL_BC_PERIODIC, STENCIL_BC_CALLER, STENCIL_BC_PERIODIC_XY = range(3)
STENCIL_XCORR, STENCIL_DIFFUSION, STENCIL_MHD8, STENCIL_MAXFILTER = range(4)

EXPORTED = (
    "stencil_create", "stencil_destroy", "stencil_layout", "stencil_step", "stencil_halo_fill",
    "stencil_mhd_rhs", "stencil_field_norms", "stencil_sync", "stencil_strerror",
    "stencil_last_error_detail", "stencil_abi_version", "stencil_get_variant",
    "stencil_set_variant", "stencil_autotune", "stencil_field_norms_noalloc", "stencil_selftest_wait",
    "stencil_server_create", "stencil_server_destroy", "stencil_server_submit", "stencil_server_progress",
    "stencil_server_poll", "stencil_server_stats", "stencil_server_sync", "stencil_server_last_error_detail",
    "stencil_server_cancel", "stencil_substep", "stencil_step_host", "stencil_autotune_status",
    "stencil_server_variant", "stencil_set_zmode",
)

STENCIL_REQ_PENDING, STENCIL_REQ_ACTIVE, STENCIL_REQ_COMPLETING, STENCIL_REQ_DONE, STENCIL_REQ_CANCELLED = range(5)


class stencil_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("alpha", ctypes.c_double), ("dx", ctypes.c_double * 3),
                ("cs0", ctypes.c_double), ("gamma", ctypes.c_double), ("cp", ctypes.c_double),
                ("lnrho0", ctypes.c_double), ("nu", ctypes.c_double), ("eta", ctypes.c_double),
                ("zeta", ctypes.c_double), ("mu0", ctypes.c_double), ("K", ctypes.c_double)]


class stencil_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dims", ctypes.c_int64 * 3), ("nsteps", ctypes.c_int),
                ("coeffs", ctypes.c_double * 7), ("params", stencil_params)]


class StencilError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({_strerror(status)}): {detail}")


_lock = threading.Lock()
_lib = None


def load():
    """Load libstencil.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libstencil.so not built ({LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        sigs = {
            "stencil_create": (I, [I, ctypes.POINTER(I64), I, P, I, I, I, I, I, I,
                                   ctypes.POINTER(stencil_params), ctypes.POINTER(P)]),
            "stencil_destroy": (None, [P]),
            "stencil_layout": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                   ctypes.POINTER(I64)]),
            "stencil_step": (I, [P, PP, PP, I, P]),
            "stencil_halo_fill": (I, [P, PP, P]),
            "stencil_substep": (I, [P, PP, PP, I, P]),
            "stencil_step_host": (I, [P, PP, PP, PP, PP, I, P]),
            "stencil_mhd_rhs": (I, [P, PP, PP, P]),
            "stencil_field_norms": (I, [P, PP, ctypes.POINTER(D), P]),
            "stencil_sync": (I, [P, P]),
            "stencil_strerror": (ctypes.c_char_p, [I]),
            "stencil_last_error_detail": (ctypes.c_char_p, [P]),
            "stencil_abi_version": (I, []),
            "stencil_get_variant": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_char_p)]),
            "stencil_set_variant": (I, [P, I]),
            "stencil_set_zmode": (I, [P, I]),
            "stencil_autotune": (I, [P, PP, PP, I, I, P]),
            "stencil_autotune_status": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float)]),
            "stencil_selftest_wait": (I, [P, I64, P]),
            "stencil_server_create": (I, [I64, I, P, ctypes.POINTER(P)]),
            "stencil_server_destroy": (None, [P]),
            "stencil_server_submit": (I, [P, ctypes.POINTER(stencil_request), PP, PP, ctypes.POINTER(I64)]),
            "stencil_server_progress": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
            "stencil_server_poll": (I, [P, I64, ctypes.POINTER(I)]),
            "stencil_server_cancel": (I, [P, I64]),
            "stencil_server_stats": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]),
            "stencil_server_sync": (I, [P]),
            "stencil_server_last_error_detail": (ctypes.c_char_p, [P]),
            "stencil_server_variant": (ctypes.c_char_p, [P, I]),
            "stencil_field_norms_noalloc": (I, [PP, I, I, ctypes.POINTER(I64), ctypes.POINTER(I64),
                                                ctypes.POINTER(I64), D, P, P]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _strerror(status: int) -> str:
    try:
        return load().stencil_strerror(status).decode()
    except Exception:  # noqa: BLE001 -- only used to format an error message
        return "?"


def _check(status: int, where: str, handle=None):
    if status != STENCIL_OK:
        detail = load().stencil_last_error_detail(handle).decode()
        raise StencilError(status, where, detail)


def _ptrs(tensors):
    arr = (ctypes.c_void_p * len(tensors))(*[int(t.data_ptr()) for t in tensors])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


# ----------------------------------------------------------------- raw C-named calls


def stencil_create(ndim, dims, radius, coeffs, nfields, bc, kind, storage, compute, params=None):
    lib = load()
    d = (ctypes.c_int64 * 3)(*(list(dims) + [1, 1, 1])[:3])
    keep = None
    cptr, ncoeffs = None, 0
    if coeffs is not None:
        keep = np.ascontiguousarray(coeffs, dtype=np.int32 if storage == STENCIL_I32 else np.float64)
        cptr, ncoeffs = keep.ctypes.data_as(ctypes.c_void_p), keep.size
    h = ctypes.c_void_p()
    st = lib.stencil_create(ndim, d, radius, cptr, ncoeffs, nfields, bc, kind, storage, compute,
                            ctypes.byref(params) if params is not None else None, ctypes.byref(h))
    _check(st, "stencil_create", None)
    return h


def stencil_layout(h):
    pad, pitch, origin = (ctypes.c_int64 * 3)(), (ctypes.c_int64 * 3)(), (ctypes.c_int64 * 3)()
    nbytes = ctypes.c_int64()
    _check(load().stencil_layout(h, pad, pitch, origin, ctypes.byref(nbytes)), "stencil_layout", h)
    return tuple(pad), tuple(pitch), tuple(origin), nbytes.value


def stencil_step(h, fields_in, fields_out, nsteps, stream=None):
    pi, ki = _ptrs(fields_in)
    po, ko = _ptrs(fields_out)
    _check(load().stencil_step(h, pi, po, nsteps, _stream(stream)), "stencil_step", h)


def stencil_step_host(h, host_in, host_out, dev_in, dev_out, nsteps, stream=None):
    """host_in / host_out: host tensors (page-locked for asynchronous copies) in the padded layout."""
    hi, khi = _ptrs(host_in)
    ho, kho = _ptrs(host_out)
    di, kdi = _ptrs(dev_in)
    do, kdo = _ptrs(dev_out)
    _check(load().stencil_step_host(h, hi, ho, di, do, nsteps, _stream(stream)), "stencil_step_host", h)


def stencil_substep(h, fields_in, fields_out, substep, stream=None):
    pi, ki = _ptrs(fields_in)
    po, ko = _ptrs(fields_out)
    _check(load().stencil_substep(h, pi, po, int(substep), _stream(stream)), "stencil_substep", h)


def stencil_halo_fill(h, fields, stream=None):
    p, k = _ptrs(fields)
    _check(load().stencil_halo_fill(h, p, _stream(stream)), "stencil_halo_fill", h)


def stencil_mhd_rhs(h, fields, rhs, stream=None):
    p, k = _ptrs(fields)
    r, kr = _ptrs(rhs)
    _check(load().stencil_mhd_rhs(h, p, r, _stream(stream)), "stencil_mhd_rhs", h)


def stencil_field_norms(h, fields, nvalues, stream=None):
    p, k = _ptrs(fields)
    out = (ctypes.c_double * nvalues)()
    _check(load().stencil_field_norms(h, p, out, _stream(stream)), "stencil_field_norms", h)
    return np.array(out[:], dtype=np.float64)


def stencil_sync(h, stream=None):
    _check(load().stencil_sync(h, _stream(stream)), "stencil_sync", h)


def stencil_get_variant(h):
    v, n, name = ctypes.c_int(), ctypes.c_int(), ctypes.c_char_p()
    _check(load().stencil_get_variant(h, ctypes.byref(v), ctypes.byref(n), ctypes.byref(name)),
           "stencil_get_variant", h)
    return v.value, n.value, name.value.decode()


def stencil_set_variant(h, variant):
    _check(load().stencil_set_variant(h, variant), "stencil_set_variant", h)


def stencil_autotune(h, fields_in, fields_out, nsteps=1, reps=3, stream=None):
    pi, ki = _ptrs(fields_in)
    po, ko = _ptrs(fields_out)
    _check(load().stencil_autotune(h, pi, po, nsteps, reps, _stream(stream)), "stencil_autotune", h)


def stencil_autotune_status(h):
    """(from_cache, zmode, ms) of the plan's current tuned choice."""
    c, z, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(load().stencil_autotune_status(h, ctypes.byref(c), ctypes.byref(z), ctypes.byref(ms)),
           "stencil_autotune_status", h)
    return bool(c.value), z.value, ms.value


def stencil_selftest_wait(h, limit_ns, stream=None):
    _check(load().stencil_selftest_wait(h, int(limit_ns), _stream(stream)), "stencil_selftest_wait", h)


_ESIZE = {STENCIL_I32: 4, STENCIL_F64: 8, STENCIL_F32: 4, STENCIL_BF16: 2}


def _einval(where, msg):
    raise StencilError(STENCIL_EINVAL, where, msg)


def stencil_field_norms_noalloc(fields, storage, dims, padded, origin, mass_volume, out_dev, stream=None):
    """Allocation-free norms: results written to the device tensor out_dev (float64).

    The C entry point only sees addresses, so the tensors are checked here first: out_dev
    must be a CUDA float64 tensor with room for every result, and each field a CUDA tensor
    of the storage element size holding at least the whole padded array."""
    where = "stencil_field_norms_noalloc"
    need = 3 * len(fields) + (1 if mass_volume > 0 else 0)
    if str(out_dev.dtype) != "torch.float64":
        _einval(where, f"out_dev must be float64, not {out_dev.dtype}")
    if out_dev.numel() < need:
        _einval(where, f"out_dev holds {out_dev.numel()} elements, {need} needed")
    npad = int(padded[0]) * int(padded[1]) * int(padded[2])
    for i, t in enumerate(fields):
        if storage in _ESIZE and t.element_size() != _ESIZE[storage]:
            _einval(where, f"fields[{i}] element size {t.element_size()} does not match the storage "
                           f"type ({_ESIZE[storage]} bytes)")
        if t.numel() < npad:
            _einval(where, f"fields[{i}] holds {t.numel()} elements, fewer than the padded array's {npad}")
    for i, t in enumerate(list(fields) + [out_dev]):
        if not t.is_cuda:
            _einval(where, ("out_dev" if i == len(fields) else f"fields[{i}]") + " is not a CUDA tensor")
    p, k = _ptrs(fields)
    d = (ctypes.c_int64 * 3)(*dims)
    pd = (ctypes.c_int64 * 3)(*padded)
    o = (ctypes.c_int64 * 3)(*origin)
    st = load().stencil_field_norms_noalloc(p, len(fields), storage, d, pd, o, float(mass_volume),
                                            ctypes.c_void_p(int(out_dev.data_ptr())), _stream(stream))
    _check(st, "stencil_field_norms_noalloc", None)


def _scheck(status, where, server):
    if status != STENCIL_OK:
        detail = load().stencil_server_last_error_detail(server).decode()
        raise StencilError(status, where, detail)


def stencil_server_create(hbm_budget_bytes, max_active, stream=None):
    h = ctypes.c_void_p()
    _scheck(load().stencil_server_create(int(hbm_budget_bytes), int(max_active), _stream(stream), ctypes.byref(h)),
            "stencil_server_create", None)
    return h


def stencil_server_destroy(h):
    if h:
        load().stencil_server_destroy(h)


def stencil_server_submit(h, req, host_in_ptrs, host_out_ptrs):
    """host_in_ptrs / host_out_ptrs: lists of integer host addresses (float32 arrays)."""
    pi = (ctypes.c_void_p * len(host_in_ptrs))(*host_in_ptrs)
    po = (ctypes.c_void_p * len(host_out_ptrs))(*host_out_ptrs)
    t = ctypes.c_int64()
    _scheck(load().stencil_server_submit(h, ctypes.byref(req), ctypes.cast(pi, ctypes.POINTER(ctypes.c_void_p)),
                                         ctypes.cast(po, ctypes.POINTER(ctypes.c_void_p)), ctypes.byref(t)),
            "stencil_server_submit", h)
    return t.value


def stencil_server_progress(h):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _scheck(load().stencil_server_progress(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
            "stencil_server_progress", h)
    return a.value, b.value, c.value


def stencil_server_poll(h, ticket):
    st = ctypes.c_int()
    _scheck(load().stencil_server_poll(h, int(ticket), ctypes.byref(st)), "stencil_server_poll", h)
    return st.value


def stencil_server_cancel(h, ticket):
    _scheck(load().stencil_server_cancel(h, int(ticket)), "stencil_server_cancel", h)


def stencil_server_stats(h):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _scheck(load().stencil_server_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
            "stencil_server_stats", h)
    return a.value, b.value, c.value


def stencil_server_variant(h, kind):
    return load().stencil_server_variant(h, int(kind)).decode()


def stencil_server_sync(h):
    _scheck(load().stencil_server_sync(h), "stencil_server_sync", h)


def stencil_destroy(h):
    if h:
        load().stencil_destroy(h)


# ----------------------------------------------------------------- convenience wrapper

_TORCH_DT = {STENCIL_I32: "int32", STENCIL_F64: "float64", STENCIL_F32: "float32", STENCIL_BF16: "bfloat16"}
_NP_DT = {STENCIL_I32: np.int32, STENCIL_F64: np.float64, STENCIL_F32: np.float32}


class Plan:
    """Owns one stencil plan; allocates fields in its padded layout with PyTorch."""

    def __init__(self, ndim, dims, radius, nfields, bc, kind, storage, compute, coeffs=None,
                 params=None):
        self.ndim, self.radius, self.nfields = ndim, radius, nfields
        self.dims = tuple(dims) + (1,) * (3 - len(dims))
        self.kind, self.storage, self.compute, self.bc = kind, storage, compute, bc
        self.params = params
        self.h = stencil_create(ndim, self.dims, radius, coeffs, nfields, bc, kind, storage,
                                compute, params)
        self.padded, self.pitch, self.origin, self.bytes_per_field = stencil_layout(self.h)

    def close(self):
        if self.h:
            stencil_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 -- interpreter shutdown
            pass

    # -- memory
    @property
    def torch_dtype(self):
        import torch
        return getattr(torch, _TORCH_DT[self.storage])

    def alloc(self, device="cuda", fill=0):
        """nfields flat tensors of padded[0]*padded[1]*padded[2] elements."""
        import torch
        n = self.padded[0] * self.padded[1] * self.padded[2]
        return [torch.full((n,), fill, dtype=self.torch_dtype, device=device) for _ in range(self.nfields)]

    def view3(self, t):
        """(z, y, x) view of a whole padded field."""
        return t.view(self.padded[2], self.padded[1], self.padded[0])

    def interior(self, t):
        """(nz, ny, nx) view of the interior (2D: (ny, nx); 1D: (nx,))."""
        v = self.view3(t)
        ox, oy, oz = self.origin
        nx, ny, nz = self.dims
        v = v[oz:oz + nz, oy:oy + ny, ox:ox + nx]
        return v[0, 0] if self.ndim == 1 else (v[0] if self.ndim == 2 else v)

    def upload(self, fields, arrays):
        """Copy host arrays (interior shape) into the interior of device fields."""
        import torch
        for t, a in zip(fields, arrays):
            src = torch.from_numpy(np.ascontiguousarray(a))
            self.interior(t).copy_(src.to(self.torch_dtype))

    def download(self, fields, dtype=np.float64):
        """Interiors of device fields as one host array (nfields, ...)."""
        import torch
        out = [self.interior(t).to(torch.float64 if dtype == np.float64 else self.torch_dtype).cpu().numpy()
               for t in fields]
        return np.stack(out)

    # -- calls
    def step(self, fin, fout, nsteps=1, stream=None):
        stencil_step(self.h, fin, fout, nsteps, stream)

    def step_host(self, host_in, host_out, dev_in, dev_out, nsteps=1, stream=None):
        stencil_step_host(self.h, host_in, host_out, dev_in, dev_out, nsteps, stream)

    def substep(self, fin, fout, substep, stream=None):
        stencil_substep(self.h, fin, fout, substep, stream)

    def halo_fill(self, fields, stream=None):
        stencil_halo_fill(self.h, fields, stream)

    def mhd_rhs(self, fields, rhs, stream=None):
        stencil_mhd_rhs(self.h, fields, rhs, stream)

    def norms(self, fields, stream=None):
        n = 3 * self.nfields + (1 if self.kind == STENCIL_MHD8 else 0)
        return stencil_field_norms(self.h, fields, n, stream)

    def sync(self, stream=None):
        stencil_sync(self.h, stream)

    def variant(self):
        return stencil_get_variant(self.h)

    def set_variant(self, v):
        stencil_set_variant(self.h, v)

    def selftest_wait(self, limit_ns, stream=None):
        stencil_selftest_wait(self.h, limit_ns, stream)

    def autotune(self, fin, fout, nsteps=1, reps=3, stream=None):
        stencil_autotune(self.h, fin, fout, nsteps, reps, stream)
        return self.variant()

    def autotune_status(self):
        return stencil_autotune_status(self.h)

    def set_zmode(self, zmode):
        _check(load().stencil_set_zmode(self.h, int(zmode)), "stencil_set_zmode", self.h)


def mhd_params(n, dt=None, **kw) -> stencil_params:
    """stencil_params for the 8-field system on a periodic (2 pi)^3 box of n^3 (or (nz,ny,nx))."""
    nz, ny, nx = (n, n, n) if np.isscalar(n) else tuple(n)
    p = stencil_params()
    tau = 2.0 * np.pi
    p.dx[0], p.dx[1], p.dx[2] = tau / nx, tau / ny, tau / nz
    vals = dict(cs0=1.0, gamma=5.0 / 3.0, cp=1.0, lnrho0=0.0, nu=5e-3, eta=5e-3, zeta=0.0, mu0=1.0, K=0.0)
    vals.update(kw)
    for k, v in vals.items():
        setattr(p, k, v)
    p.dt = 0.1 * min(p.dx[0], p.dx[1], p.dx[2]) if dt is None else dt
    return p


def heat_params(n, alpha=1.0, dt=None) -> stencil_params:
    """stencil_params for the heat equation on a periodic (2 pi)^d box; dt = 0.1 dx^2.  n is the
    edge of a cube or the dense shape ((nz, ny, nx), (ny, nx) or (nx,)); absent axes get dx = 2 pi."""
    nz, ny, nx = (n, n, n) if np.isscalar(n) else (1,) * (3 - len(tuple(n))) + tuple(n)
    p = stencil_params()
    tau = 2.0 * np.pi
    p.dx[0], p.dx[1], p.dx[2] = tau / nx, tau / ny, tau / nz
    p.alpha = alpha
    used = [d for d, m in zip((p.dx[0], p.dx[1], p.dx[2]), (nx, ny, nz)) if m > 1] or [p.dx[0]]
    p.dt = 0.1 * min(used) ** 2 if dt is None else dt
    return p
