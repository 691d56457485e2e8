"""Host-side checks of the C ABI: the library loads without a GPU, exports every symbol that
include/stencil.h declares, and rejects invalid arguments before touching the device.  The
ctypes binding agrees with the header: argument counts, result kinds, enumerator values, and
the size and field offsets of the structs (as gcc lays them out)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2406_08923_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stencil.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2406_08923_gb300 import build
        build.build()
    return _lib.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stencil_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (stencil_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)
    assert set(_lib.EXPORTED) == set(names)


def test_abi_version_and_strerror(lib):
    assert lib.stencil_abi_version() == 1
    for s in range(6):
        assert lib.stencil_strerror(s).decode().startswith("STENCIL_")
    assert b"unknown" in lib.stencil_strerror(99)


def _create(lib, ndim=3, dims=(16, 16, 16), radius=3, coeffs=None, nfields=1, bc=0, kind=1, storage=1,
            compute=1, params=True):
    d = (ctypes.c_int64 * 3)(*dims)
    keep = None
    cp, nc = None, 0
    if coeffs is not None:
        keep = np.ascontiguousarray(coeffs, dtype=np.int32 if storage == 0 else np.float64)
        cp, nc = keep.ctypes.data_as(ctypes.c_void_p), keep.size
    p = (_lib.mhd_params(16) if kind == 2 else _lib.heat_params(16)) if params else None
    h = ctypes.c_void_p()
    st = lib.stencil_create(ndim, d, radius, cp, nc, nfields, bc, kind, storage, compute,
                            ctypes.byref(p) if p is not None else None, ctypes.byref(h))
    return st, h, lib.stencil_last_error_detail(None).decode()


@pytest.mark.parametrize("kw,expect", [
    (dict(ndim=0), _lib.STENCIL_EINVAL),
    (dict(ndim=4), _lib.STENCIL_EINVAL),
    (dict(dims=(0, 16, 16)), _lib.STENCIL_EINVAL),
    (dict(radius=-1), _lib.STENCIL_EINVAL),
    (dict(radius=5), _lib.STENCIL_EUNSUPPORTED),                # diffusion radius 1..4
    (dict(radius=0), _lib.STENCIL_EUNSUPPORTED),
    (dict(kind=2, nfields=8, radius=2), _lib.STENCIL_EINVAL),   # MHD8 is radius 3
    (dict(dims=(6, 16, 16)), _lib.STENCIL_EINVAL),              # periodic extent < 2r+1
    (dict(params=False), _lib.STENCIL_EINVAL),
    (dict(nfields=2), _lib.STENCIL_EINVAL),
    (dict(kind=7), _lib.STENCIL_EINVAL),
    (dict(storage=9), _lib.STENCIL_EINVAL),
    (dict(storage=3, compute=2), _lib.STENCIL_EUNSUPPORTED),    # BF16 diffusion
    (dict(kind=2, nfields=8, ndim=2, dims=(16, 16, 1)), _lib.STENCIL_EUNSUPPORTED),  # MHD8 is 3D
    (dict(ndim=2, dims=(16, 6, 1), radius=3), _lib.STENCIL_EINVAL),  # periodic extent < 2r+1
    (dict(kind=2, nfields=8, bc=1), _lib.STENCIL_EUNSUPPORTED),  # MHD8 needs periodic
    (dict(bc=3), _lib.STENCIL_EINVAL),                           # unknown boundary mode
    (dict(bc=2, ndim=2, dims=(16, 16, 1)), _lib.STENCIL_EUNSUPPORTED),  # z-slabs are 3D
    (dict(bc=2, kind=0, ndim=1, dims=(64, 1, 1), coeffs=[1.0, 2.0, 1.0], radius=1), _lib.STENCIL_EUNSUPPORTED),
    (dict(bc=2, dims=(16, 16, 2)), _lib.STENCIL_EINVAL),          # slab thinner than the radius
    (dict(bc=2, dims=(6, 16, 16)), _lib.STENCIL_EINVAL),          # periodic x extent < 2r+1
    (dict(kind=2, nfields=8, storage=0, compute=0), _lib.STENCIL_EUNSUPPORTED),
    (dict(kind=0, ndim=1, dims=(64, 1, 1), radius=3, nfields=1, coeffs=[1] * 6, storage=0, compute=0), _lib.STENCIL_EINVAL),
    (dict(kind=0, ndim=1, dims=(64, 1, 1), radius=5, nfields=1, coeffs=[1] * 11, storage=0, compute=0), _lib.STENCIL_EUNSUPPORTED),
    (dict(kind=0, ndim=3, radius=1, coeffs=[1, 2, 3], storage=0, compute=0), _lib.STENCIL_EUNSUPPORTED),
    (dict(kind=0, ndim=1, dims=(4096, 1, 1), radius=1025, coeffs=[1.0] * 2051), _lib.STENCIL_EUNSUPPORTED),
    (dict(kind=3, ndim=1, dims=(4096, 1, 1), radius=1025, params=False), _lib.STENCIL_EUNSUPPORTED),
    (dict(kind=3, ndim=1, dims=(64, 1, 1), radius=2, coeffs=[1.0] * 5, params=False), _lib.STENCIL_EINVAL),
    (dict(kind=3, ndim=2, dims=(64, 64, 1), radius=2, params=False), _lib.STENCIL_EUNSUPPORTED),
    (dict(kind=3, ndim=1, dims=(64, 1, 1), radius=2, storage=3, compute=3, params=False), _lib.STENCIL_EUNSUPPORTED),
    (dict(kind=3, ndim=1, dims=(8, 1, 1), radius=4, params=False), _lib.STENCIL_EINVAL),  # n < 2r+1
    (dict(kind=0, ndim=1, dims=(64, 1, 1), radius=1, coeffs=[1, 2, 3], storage=1, compute=2), _lib.STENCIL_EUNSUPPORTED),
])
def test_create_rejects_invalid_arguments(lib, kw, expect):
    st, h, detail = _create(lib, **kw)
    assert st == expect, (st, detail)
    assert not h.value
    assert detail


@pytest.mark.parametrize("kw", [dict(bc=2, dims=(16, 16, 3)), dict(bc=2, kind=2, nfields=8, dims=(16, 16, 5))])
def test_z_slab_plans_are_accepted(lib, kw):
    st, plan, detail = _create(lib, **kw)
    assert st in (0, _lib.STENCIL_ECUDA), detail
    if st == 0:
        lib.stencil_destroy(plan)


def test_null_plan_calls_are_rejected(lib):
    assert lib.stencil_layout(None, None, None, None, None) == _lib.STENCIL_EINVAL
    assert lib.stencil_step(None, None, None, 1, None) == _lib.STENCIL_EINVAL
    assert lib.stencil_sync(None, None) == _lib.STENCIL_EINVAL
    assert lib.stencil_set_variant(None, 0) == _lib.STENCIL_EINVAL
    assert lib.stencil_substep(None, None, None, 0, None) == _lib.STENCIL_EINVAL
    lib.stencil_destroy(None)


@pytest.mark.parametrize("ndim,dims,radius", [(1, (64, 1, 1), 1), (1, (9, 1, 1), 4), (2, (16, 9, 1), 4),
                                              (2, (32, 32, 1), 2), (3, (16, 16, 16), 1), (3, (9, 9, 9), 4)])
def test_diffusion_radius_sweep_plans_are_accepted(lib, ndim, dims, radius):
    for storage in (1, 2):
        st, plan, detail = _create(lib, ndim=ndim, dims=dims, radius=radius, storage=storage, compute=storage)
        # argument validation accepts the plan; without a GPU the device allocation then fails
        assert st in (0, _lib.STENCIL_ECUDA), detail
        if st == 0:
            lib.stencil_destroy(plan)


@pytest.mark.parametrize("kw", [dict(kind=0, ndim=1, dims=(2049, 1, 1), radius=1024, coeffs=[0.5] * 2049, storage=2,
                                     compute=2, params=False),
                                dict(kind=0, ndim=1, dims=(99, 1, 1), radius=17, coeffs=[0.5] * 35, params=False),
                                dict(kind=3, ndim=1, dims=(2049, 1, 1), radius=1024, storage=0, compute=0, params=False),
                                dict(kind=3, ndim=1, dims=(5, 1, 1), radius=0, params=False)])
def test_wide_xcorr_and_maxfilter_plans_are_accepted(lib, kw):
    st, plan, detail = _create(lib, **kw)
    assert st in (0, _lib.STENCIL_ECUDA), detail
    if st == 0:
        lib.stencil_destroy(plan)


def test_create_null_out_and_dims(lib):
    p = _lib.heat_params(16)
    d = (ctypes.c_int64 * 3)(16, 16, 16)
    assert lib.stencil_create(3, d, 3, None, 0, 1, 0, 1, 1, 1, ctypes.byref(p), None) == _lib.STENCIL_EINVAL
    h = ctypes.c_void_p()
    assert lib.stencil_create(3, None, 3, None, 0, 1, 0, 1, 1, 1, ctypes.byref(p), ctypes.byref(h)) == _lib.STENCIL_EINVAL


def test_python_binding_raises_with_detail(lib):
    with pytest.raises(_lib.StencilError) as e:
        _lib.stencil_create(3, (5, 16, 16), 3, None, 1, 0, 1, 1, 1, _lib.heat_params(16))
    assert e.value.status == _lib.STENCIL_EINVAL
    assert "2*radius+1" in str(e.value)


def _prototypes():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = {}
    for m in re.finditer(r"([\w\s\*]+?)\b(stencil_\w+)\s*\(([^;{}]*?)\)\s*;", src):
        params = m.group(3).strip()
        out[m.group(2)] = (" ".join(m.group(1).split()), 0 if params in ("", "void") else params.count(",") + 1)
    return src, out


def test_binding_signatures_match_the_header(lib):
    # every bound function takes as many arguments as its prototype, with a matching result kind
    src, protos = _prototypes()
    assert set(protos) == set(_declared())
    for name, (ret, nargs) in protos.items():
        fn = getattr(lib, name)
        assert len(fn.argtypes) == nargs, (name, len(fn.argtypes), nargs)
        if ret.endswith("void") and "*" not in ret:
            assert fn.restype is None, name
        elif "char" in ret:
            assert fn.restype is ctypes.c_char_p, name
        else:
            assert fn.restype is ctypes.c_int, name
    # enumerators the binding re-declares carry the header's values
    for k, v in re.findall(r"\b(STENCIL_[A-Z0-9_]+)\s*=\s*(\d+)", src):
        if hasattr(_lib, k):
            assert getattr(_lib, k) == int(v), k


def test_binding_structs_match_the_c_layout(tmp_path):
    # sizes and field offsets of the two structs the ABI passes by pointer, as gcc lays them out
    fields = {"stencil_params": [f for f, _ in _lib.stencil_params._fields_],
              "stencil_request": [f for f, _ in _lib.stencil_request._fields_]}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "stencil.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'printf("%zu\\n", sizeof({st}));')
        lines += [f'printf("%zu\\n", offsetof({st}, {f}));' for f in fs]
    lines.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    k = 0
    for st, fs in fields.items():
        cls = getattr(_lib, st)
        assert vals[k] == ctypes.sizeof(cls), st
        k += 1
        for f in fs:
            assert vals[k] == getattr(cls, f).offset, (st, f)
            k += 1


def _noalloc_call(lib, field_addrs, storage, out_addr, dims=(16, 16, 16), padded=(24, 22, 22), origin=(4, 3, 3)):
    arr = (ctypes.c_void_p * len(field_addrs))(*field_addrs)
    d, pd, o = (ctypes.c_int64 * 3)(*dims), (ctypes.c_int64 * 3)(*padded), (ctypes.c_int64 * 3)(*origin)
    st = lib.stencil_field_norms_noalloc(ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), len(field_addrs),
                                         storage, d, pd, o, 0.0, ctypes.c_void_p(out_addr), None)
    return st, lib.stencil_last_error_detail(None).decode()


@pytest.mark.parametrize("storage,addr", [(_lib.STENCIL_F64, 0x10004), (_lib.STENCIL_F32, 0x10002),
                                          (_lib.STENCIL_I32, 0x10001), (_lib.STENCIL_BF16, 0x10001)])
def test_noalloc_norms_rejects_misaligned_fields(lib, storage, addr):
    # rejected on the host before any launch: a misaligned element address would fault in pass 1
    st, detail = _noalloc_call(lib, [0x20000, addr], storage, 0x30000)
    assert st == _lib.STENCIL_EINVAL, detail
    assert "fields[1] is not aligned" in detail


def test_noalloc_norms_rejects_misaligned_output(lib):
    st, detail = _noalloc_call(lib, [0x20000], _lib.STENCIL_F64, 0x30004)
    assert st == _lib.STENCIL_EINVAL, detail
    assert "out_dev is not 8-byte aligned" in detail


def test_noalloc_binding_checks_its_tensors():
    # the Python binding refuses tensors that the kernels would read or write out of bounds
    torch = pytest.importorskip("torch")
    dims, padded, origin = (16, 16, 16), (24, 22, 22), (4, 3, 3)
    n = padded[0] * padded[1] * padded[2]
    good_f = [torch.zeros(n, dtype=torch.float64)]
    good_out = torch.zeros(3, dtype=torch.float64)
    cases = [
        (good_f, torch.zeros(3, dtype=torch.float32), "float64"),                 # FP32 result buffer
        (good_f, torch.zeros(2, dtype=torch.float64), "elements"),                # too short
        ([torch.zeros(n, dtype=torch.float32)], good_out, "element size"),        # dtype vs storage
        ([torch.zeros(n - 1, dtype=torch.float64)], good_out, "padded"),          # field too small
        (good_f, good_out, "CUDA"),                                               # host tensors
    ]
    for fields, out, words in cases:
        with pytest.raises(_lib.StencilError) as e:
            _lib.stencil_field_norms_noalloc(fields, _lib.STENCIL_F64, dims, padded, origin, 0.0, out)
        assert e.value.status == _lib.STENCIL_EINVAL
        assert words in str(e.value), (words, str(e.value))
    # the mass slot needs one more double
    with pytest.raises(_lib.StencilError) as e:
        _lib.stencil_field_norms_noalloc(good_f, _lib.STENCIL_F64, dims, padded, origin, 1.0, good_out)
    assert "elements" in str(e.value)
