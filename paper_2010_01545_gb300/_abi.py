"""ctypes binding of the C ABI in ``include/advect.h`` (same names).

Argument marshalling only: every step of the computation runs in the CUDA
library.  There is no fallback: if ``_build/libadvect.so`` is missing the
first call raises.  Device buffers are passed as integer addresses.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libadvect.so")

ADVECT_F64, ADVECT_F32, ADVECT_F16S, ADVECT_F64_FF = 0, 1, 2, 3
STATUS_NAMES = {0: "ADVECT_OK", 1: "ADVECT_EINVAL", 2: "ADVECT_ENOMEM", 3: "ADVECT_ECUDA",
                4: "ADVECT_EUNSUPPORTED", 5: "ADVECT_ETIMEOUT"}

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class AdvectError(RuntimeError):
    """A non-OK advect_status, with the library's message."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class advect_grid(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("z", _dp), ("zn", _dp), ("rho", _dp), ("rhon", _dp)]


class advect_coeffs(ctypes.Structure):
    _fields_ = [("tcx", ctypes.c_double), ("tcy", ctypes.c_double),
                ("tzc1", _dp), ("tzc2", _dp), ("tzd1", _dp), ("tzd2", _dp)]


EXPORTS = (
    "advect_coeffs_from_grid", "advect_create", "advect_forward", "advect_adjoint",
    "advect_forward_host", "advect_f16s_output_scales", "advect_set_f64_levels",
    "advect_ensemble_create", "advect_ensemble_forward", "advect_ensemble_adjoint",
    "advect_sync", "advect_kernel_name", "advect_destroy", "advect_last_error",
    "advect_autotune", "advect_tuned_config", "advect_forward_noalloc",
    "advect_forward_integrate",
)

NOALLOC_MAX_NZ = 512  # ADVECT_NOALLOC_MAX_NZ

_lib = None


def library_path() -> str:
    return LIB_PATH


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_2010_01545_gb300.build.build())")
    L = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    L.advect_coeffs_from_grid.argtypes = [ctypes.POINTER(advect_grid), _dp, _dp, _dp, _dp, _dp, _dp]
    L.advect_coeffs_from_grid.restype = st
    L.advect_create.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(advect_coeffs), ctypes.c_int,
                                                     ctypes.POINTER(_vp)]
    L.advect_create.restype = st
    L.advect_forward.argtypes = [_vp] * 7 + [ctypes.POINTER(ctypes.c_float), _vp]
    L.advect_forward.restype = st
    L.advect_forward_integrate.argtypes = ([_vp] * 7 + [ctypes.c_double] + [_vp] * 3
                                           + [ctypes.POINTER(ctypes.c_float), _vp])
    L.advect_forward_integrate.restype = st
    L.advect_adjoint.argtypes = [_vp] * 10 + [_vp]
    L.advect_adjoint.restype = st
    L.advect_forward_host.argtypes = [_vp] * 7 + [ctypes.POINTER(ctypes.c_float)]
    L.advect_forward_host.restype = st
    L.advect_f16s_output_scales.argtypes = [_vp, ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_float)]
    L.advect_f16s_output_scales.restype = st
    L.advect_set_f64_levels.argtypes = [_vp, ctypes.c_int]
    L.advect_set_f64_levels.restype = st
    ip = ctypes.POINTER(ctypes.c_int)
    L.advect_ensemble_create.argtypes = [ctypes.c_int, ip, ip, ip, ctypes.POINTER(advect_coeffs),
                                         ctypes.c_int, ctypes.POINTER(_vp)]
    L.advect_ensemble_create.restype = st
    pp = ctypes.POINTER(_vp)
    L.advect_ensemble_forward.argtypes = [_vp] + [pp] * 6 + [_vp]
    L.advect_ensemble_forward.restype = st
    L.advect_ensemble_adjoint.argtypes = [_vp] + [pp] * 9 + [_vp]
    L.advect_ensemble_adjoint.restype = st
    L.advect_sync.argtypes = [_vp, _vp]
    L.advect_sync.restype = st
    L.advect_kernel_name.argtypes = [_vp, ctypes.c_int]
    L.advect_kernel_name.restype = ctypes.c_char_p
    L.advect_autotune.argtypes = [_vp, ctypes.c_int]
    L.advect_autotune.restype = st
    L.advect_tuned_config.argtypes = [_vp, ctypes.c_int]
    L.advect_tuned_config.restype = ctypes.c_char_p
    L.advect_forward_noalloc.argtypes = ([ctypes.c_int] * 3 + [ctypes.POINTER(advect_coeffs), ctypes.c_int]
                                         + [_vp] * 6 + [ctypes.POINTER(ctypes.c_float), _vp])
    L.advect_forward_noalloc.restype = st
    L.advect_destroy.argtypes = [_vp]
    L.advect_destroy.restype = None
    L.advect_last_error.argtypes = []
    L.advect_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status: int) -> None:
    if status != 0:
        raise AdvectError(status, lib().advect_last_error().decode())


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def advect_coeffs_from_grid(nz, dx, dy, z, zn, rho, rhon):
    """(tcx, tcy, tzc1, tzc2, tzd1, tzd2) computed by the library."""
    arrs = [_f64(a) for a in (z, zn, rho, rhon)]
    if any(a.shape != (nz,) for a in arrs):
        raise ValueError("level arrays must have shape (nz,)")
    g = advect_grid(int(nz), float(dx), float(dy), *(_ptr(a) for a in arrs))
    tcx, tcy = ctypes.c_double(), ctypes.c_double()
    tabs = [np.zeros(nz) for _ in range(4)]
    _check(lib().advect_coeffs_from_grid(ctypes.byref(g), ctypes.byref(tcx), ctypes.byref(tcy),
                                         *(_ptr(t) for t in tabs)))
    return tcx.value, tcy.value, *tabs


def _coeffs_struct(tcx, tcy, tzc1, tzc2, tzd1, tzd2):
    keep = [_f64(t) for t in (tzc1, tzc2, tzd1, tzd2)]
    return advect_coeffs(float(tcx), float(tcy), *(_ptr(t) for t in keep)), keep


def advect_create(nx, ny, nz, coeffs, dtype) -> int:
    """coeffs: (tcx, tcy, tzc1, tzc2, tzd1, tzd2); returns the context handle."""
    c, keep = _coeffs_struct(*coeffs)
    out = _vp()
    _check(lib().advect_create(int(nx), int(ny), int(nz), ctypes.byref(c), int(dtype), ctypes.byref(out)))
    del keep
    return out.value


def _scales(scales):
    if scales is None:
        return None
    arr = (ctypes.c_float * len(scales))(*[float(s) for s in scales])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_float))


def advect_forward(ctx, u, v, w, su, sv, sw, scales=None, stream=0) -> None:
    _check(lib().advect_forward(ctx, u, v, w, su, sv, sw, _scales(scales), stream))


def advect_forward_integrate(ctx, u, v, w, u_base, v_base, w_base, dt, u_out, v_out, w_out,
                             scales=None, stream=0) -> None:
    _check(lib().advect_forward_integrate(ctx, u, v, w, u_base, v_base, w_base, float(dt),
                                          u_out, v_out, w_out, _scales(scales), stream))


def advect_adjoint(ctx, u, v, w, dsu, dsv, dsw, du, dv, dw, stream=0) -> None:
    _check(lib().advect_adjoint(ctx, u, v, w, dsu, dsv, dsw, du, dv, dw, stream))


def advect_forward_host(ctx, u, v, w, su, sv, sw, scales=None) -> None:
    _check(lib().advect_forward_host(ctx, u, v, w, su, sv, sw, _scales(scales)))


def advect_f16s_output_scales(ctx, scales_in):
    a = (ctypes.c_float * 3)(*[float(s) for s in scales_in])
    b = (ctypes.c_float * 3)()
    _check(lib().advect_f16s_output_scales(ctx, a, b))
    return [b[0], b[1], b[2]]


def advect_set_f64_levels(ctx, n) -> None:
    _check(lib().advect_set_f64_levels(ctx, int(n)))


def advect_ensemble_create(shapes, coeffs_list, dtype) -> int:
    n = len(shapes)
    nx = (ctypes.c_int * n)(*[s[0] for s in shapes])
    ny = (ctypes.c_int * n)(*[s[1] for s in shapes])
    nz = (ctypes.c_int * n)(*[s[2] for s in shapes])
    structs, keep = [], []
    for c in coeffs_list:
        s, k = _coeffs_struct(*c)
        structs.append(s)
        keep.append(k)
    arr = (advect_coeffs * n)(*structs)
    out = _vp()
    _check(lib().advect_ensemble_create(n, nx, ny, nz, arr, int(dtype), ctypes.byref(out)))
    del keep
    return out.value


def _ptr_array(ptrs):
    return (_vp * len(ptrs))(*ptrs)


def advect_ensemble_forward(ctx, u, v, w, su, sv, sw, stream=0) -> None:
    _check(lib().advect_ensemble_forward(ctx, *(_ptr_array(p) for p in (u, v, w, su, sv, sw)), stream))


def advect_ensemble_adjoint(ctx, u, v, w, dsu, dsv, dsw, du, dv, dw, stream=0) -> None:
    _check(lib().advect_ensemble_adjoint(
        ctx, *(_ptr_array(p) for p in (u, v, w, dsu, dsv, dsw, du, dv, dw)), stream))


def advect_sync(ctx, stream=0) -> None:
    _check(lib().advect_sync(ctx, stream))


def advect_kernel_name(ctx, adjoint=False) -> str:
    return lib().advect_kernel_name(ctx, 1 if adjoint else 0).decode()


def advect_autotune(ctx, enable=True) -> None:
    _check(lib().advect_autotune(ctx, 1 if enable else 0))


def advect_tuned_config(ctx, adjoint=False) -> str:
    return lib().advect_tuned_config(ctx, 1 if adjoint else 0).decode()


def advect_forward_noalloc(nx, ny, nz, coeffs, dtype, u, v, w, su, sv, sw, scales=None,
                           stream=0) -> None:
    """Context-free forward that allocates no device memory (see include/advect.h)."""
    c, keep = _coeffs_struct(*coeffs)
    _check(lib().advect_forward_noalloc(int(nx), int(ny), int(nz), ctypes.byref(c), int(dtype),
                                        u, v, w, su, sv, sw, _scales(scales), stream))
    del keep


def advect_destroy(ctx) -> None:
    if ctx:
        lib().advect_destroy(ctx)


def advect_last_error() -> str:
    return lib().advect_last_error().decode()
