"""Host-side checks of the C ABI that need no GPU.

The library must build for sm_103a, load, and export every function that
include/advect.h declares.  Coefficient setup (host code in the library) is
compared with the oracle's, and argument validation that happens before any
CUDA call is exercised with bad inputs (host-side fault injection).
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import workload
from paper_2010_01545_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.lib()


def declared_functions():
    with open(os.path.join(ROOT, "include", "advect.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(advect_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("advect_create", "advect_forward", "advect_adjoint", "advect_destroy",
                 "advect_ensemble_create", "advect_ensemble_forward", "advect_ensemble_adjoint",
                 "advect_last_error", "advect_coeffs_from_grid"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/advect.h but not exported"
        assert name in _abi.EXPORTS, f"{name} has no binding of the same name"


def test_oracle_is_not_linked_into_the_library():
    out = os.popen(f"nm -D --defined-only {_abi.LIB_PATH}").read()
    assert "oracle_" not in out


@pytest.mark.parametrize("nz", [3, 4, 64, 128])
def test_library_coefficients_match_oracle(lib, nz):
    g = workload.vertical_grid(nz)
    mine = _abi.advect_coeffs_from_grid(g.nz, g.dx, g.dy, g.z, g.zn, g.rho, g.rhon)
    ref = oracle.coefficients(g)
    assert mine[0] == ref.tcx and mine[1] == ref.tcy
    for a, b in zip(mine[2:], (ref.tzc1, ref.tzc2, ref.tzd1, ref.tzd2)):
        np.testing.assert_allclose(a, b, rtol=1e-15, atol=0)


def test_coefficients_reject_bad_grids(lib):
    g = workload.vertical_grid(8)
    bad_z = g.z.copy()
    bad_z[3] = bad_z[2]
    with pytest.raises(_abi.AdvectError) as e:
        _abi.advect_coeffs_from_grid(8, g.dx, g.dy, bad_z, g.zn, g.rho, g.rhon)
    assert e.value.status == 1 and "z must increase" in str(e.value)
    with pytest.raises(_abi.AdvectError):
        _abi.advect_coeffs_from_grid(8, -1.0, g.dy, g.z, g.zn, g.rho, g.rhon)
    with pytest.raises(_abi.AdvectError):
        _abi.advect_coeffs_from_grid(8, g.dx, g.dy, g.z, g.zn, -g.rho, g.rhon)
    with pytest.raises(_abi.AdvectError):
        _abi.advect_coeffs_from_grid(2, g.dx, g.dy, g.z[:2], g.zn[:2], g.rho[:2], g.rhon[:2])


def _coeffs(nz):
    g = workload.vertical_grid(nz)
    return _abi.advect_coeffs_from_grid(g.nz, g.dx, g.dy, g.z, g.zn, g.rho, g.rhon)


@pytest.mark.parametrize("shape", [(0, 4, 8), (4, 0, 8), (4, 4, 2), (-1, 4, 8)])
def test_create_rejects_bad_shapes_before_touching_the_gpu(lib, shape):
    c = _coeffs(8)
    with pytest.raises(_abi.AdvectError) as e:
        _abi.advect_create(*shape, c, _abi.ADVECT_F64)
    assert e.value.status == 1


def test_create_rejects_bad_dtype_and_coefficients(lib):
    c = _coeffs(8)
    with pytest.raises(_abi.AdvectError) as e:
        _abi.advect_create(4, 4, 8, c, 7)
    assert e.value.status == 1
    bad = list(c)
    bad[2] = bad[2].copy()
    bad[2][3] = np.nan
    with pytest.raises(_abi.AdvectError) as e:
        _abi.advect_create(4, 4, 8, bad, _abi.ADVECT_F64)
    assert "not finite" in str(e.value)


def test_null_context_and_null_out_are_errors(lib):
    L = lib
    assert L.advect_forward(None, None, None, None, None, None, None, None, None) == 1
    assert "NULL" in _abi.advect_last_error()
    assert L.advect_adjoint(*([None] * 11)) == 1
    assert L.advect_forward_integrate(*([None] * 7), 0.5, *([None] * 5)) == 1
    assert L.advect_sync(None, None) == 1
    assert L.advect_create(4, 4, 8, None, 0, None) == 1
    L.advect_destroy(None)          # NULL-safe
    assert L.advect_kernel_name(None, 0) == b""


def test_last_error_is_per_thread(lib):
    import threading
    with pytest.raises(_abi.AdvectError):
        _abi.advect_create(0, 4, 8, _coeffs(8), 0)
    seen = []
    t = threading.Thread(target=lambda: seen.append(_abi.advect_last_error()))
    t.start()
    t.join()
    assert seen == [""]
    assert "invalid shape" in _abi.advect_last_error()


def test_ensemble_create_validates_on_the_host(lib):
    c8 = _coeffs(8)
    with pytest.raises(_abi.AdvectError) as e:
        _abi.advect_ensemble_create([], [], _abi.ADVECT_F32)
    assert e.value.status == 1
    with pytest.raises(_abi.AdvectError) as e:
        _abi.advect_ensemble_create([(8, 8, 8)], [c8], _abi.ADVECT_F16S)
    assert e.value.status == 4
    c6 = _coeffs(6)
    with pytest.raises(_abi.AdvectError) as e:   # nz * 4 bytes not a multiple of 16
        _abi.advect_ensemble_create([(8, 8, 8), (8, 8, 6)], [c8, c6], _abi.ADVECT_F32)
    assert e.value.status == 4 and "member 1" in str(e.value)
    with pytest.raises(_abi.AdvectError) as e:
        _abi.advect_ensemble_create([(8, 0, 8)], [c8], _abi.ADVECT_F32)
    assert e.value.status == 1 and "member 0" in str(e.value)
    assert lib.advect_ensemble_forward(None, *([None] * 6), None) == 1
    assert lib.advect_autotune(None, 1) == 1
    assert lib.advect_tuned_config(None, 0) == b""


@pytest.mark.parametrize("bad", [3.0, 0.75, 0.0, -2.0, float("inf"), float("nan")])
def test_f16s_scales_must_be_powers_of_two(lib, bad):
    """The F16S sweep folds the input scales into the constants, which is
    exact only for powers of two: any other scale is rejected (checked before
    any CUDA call, so no GPU is needed)."""
    c = _coeffs(8)
    scales = [16.0, 16.0, 8.0, 64.0, 64.0, 32.0]
    for q in (0, 4):
        s = list(scales)
        s[q] = bad
        with pytest.raises(_abi.AdvectError) as e:
            _abi.advect_forward_noalloc(4, 4, 8, c, _abi.ADVECT_F16S, 16, 16, 16, 16, 16, 16, s)
        assert e.value.status == 1 and "power of two" in str(e.value)
