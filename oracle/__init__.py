"""CPU oracle for the PW momentum-advection source terms (Sec. 2.1, Listing 1).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the library and its Python
binding never import it.  The arithmetic lives in ``advect_oracle.c`` (plain
FP64 triple loop, ``-O2 -ffp-contract=off``); this module only compiles it
with gcc and marshals numpy arrays.

Parity status of each function (what pins it; the pins live in ``tests/``):

* ``coefficients``   -- closed forms (uniform grid), the flux-telescoping
  identity ``tzc1(k+1) rho_n(k+1) dz(k+1) = tzc2(k) rho_n(k) dz(k) = rho_w(k)/4``,
  and the linear-gradient consistency of ``tcx``.
* ``forward``        -- exact agreement with an independently written
  skew-symmetric (half flux form + half advective form) evaluator in rational
  arithmetic, impulse responses, zero tendency, reflection antisymmetry,
  periodic shift equivariance, power-of-two scaling, the su/sv transpose
  symmetry and discrete kinetic-energy conservation.
* ``integrate``      -- exact agreement with the rational skew-symmetric
  tendencies added to the base fields, the zero-step identity, and the
  forward-Euler energy budget E(u + dt S) - E(u) = dt^2 <S, S> that the
  scheme's energy conservation implies.
* ``adjoint``        -- exact dot-product identity against the forward's
  tangent ``F(x+d) - F(x) - F(d)`` and exact central differences (the map is
  quadratic), both on dyadic inputs where FP64 is exact.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "advect_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC", "-shared"]

OPENMP_CFLAGS = ["-fopenmp"]

_lib_handles = {}


def _lib_path(openmp: bool = False) -> str:
    flags = CFLAGS + (OPENMP_CFLAGS if openmp else [])
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read() + " ".join(flags).encode()).hexdigest()[:12]
    kind = "_omp" if openmp else ""
    return os.path.join(_BUILD, f"liboracle{kind}_{platform.machine()}_{tag}.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (idempotent); returns the .so path.  With
    ``openmp`` the same source is built with -fopenmp, which shares the
    forward's x-planes among all host cores (same results, bit for bit)."""
    path = _lib_path(openmp)
    if force or not os.path.exists(path):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        flags = CFLAGS + (OPENMP_CFLAGS if openmp else [])
        subprocess.run(["gcc", *flags, "-o", tmp, _SRC], check=True)
        os.replace(tmp, path)
    return path


def _lib(openmp: bool = False):
    if openmp not in _lib_handles:
        lib = ctypes.CDLL(build(openmp=openmp))
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_coefficients.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            dp, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.oracle_coefficients.restype = ctypes.c_int
        lib.oracle_forward.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [dp] * 4
                                       + [dp] * 6 + [ctypes.c_int] * 2)
        lib.oracle_forward.restype = ctypes.c_int
        lib.oracle_adjoint.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [dp] * 4
                                       + [dp] * 9)
        lib.oracle_adjoint.restype = ctypes.c_int
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        _lib_handles[openmp] = lib
    return _lib_handles[openmp]


def threads(openmp: bool = False) -> int:
    """Threads ``forward`` runs on (1 for the plain build)."""
    return int(_lib(openmp).oracle_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


@dataclass(frozen=True)
class Coefficients:
    """tcx, tcy and the four per-level tables (0-based: paper level k at [k-1])."""

    tcx: float
    tcy: float
    tzc1: np.ndarray
    tzc2: np.ndarray
    tzd1: np.ndarray
    tzd2: np.ndarray

    @property
    def nz(self) -> int:
        return int(self.tzc1.shape[0])


def coefficients(grid) -> Coefficients:
    """Advection coefficients from a ``workload.VerticalGrid``."""
    nz = grid.nz
    z, zn, rho, rhon = (_f64(a) for a in (grid.z, grid.zn, grid.rho, grid.rhon))
    tc = np.zeros(2)
    tabs = [np.zeros(nz) for _ in range(4)]
    rc = _lib().oracle_coefficients(nz, grid.dx, grid.dy, _p(z), _p(zn), _p(rho), _p(rhon),
                                    _p(tc), *(_p(t) for t in tabs))
    if rc != 0:
        raise ValueError("oracle_coefficients: invalid grid")
    return Coefficients(float(tc[0]), float(tc[1]), *tabs)


def coefficients_from_tables(tcx, tcy, tzc1, tzc2, tzd1, tzd2) -> Coefficients:
    return Coefficients(float(tcx), float(tcy), *(_f64(t) for t in (tzc1, tzc2, tzd1, tzd2)))


def _check_fields(*fields):
    shape = fields[0].shape
    if len(shape) != 3 or any(f.shape != shape for f in fields):
        raise ValueError("fields must share one (nx, ny, nz) shape")
    return shape


def forward(u, v, w, c: Coefficients, i_range=None, openmp=False):
    """(su, sv, sw) for x-planes in ``i_range`` (default: all; others stay 0).
    ``openmp`` runs the same loop on all host cores (the -fopenmp build)."""
    u, v, w = _f64(u), _f64(v), _f64(w)
    nx, ny, nz = _check_fields(u, v, w)
    if nz != c.nz:
        raise ValueError("coefficient tables do not match nz")
    i0, i1 = (0, nx) if i_range is None else i_range
    su, sv, sw = (np.zeros((nx, ny, nz)) for _ in range(3))
    rc = _lib(openmp).oracle_forward(nx, ny, nz, c.tcx, c.tcy, _p(c.tzc1), _p(c.tzc2), _p(c.tzd1),
                               _p(c.tzd2), _p(u), _p(v), _p(w), _p(su), _p(sv), _p(sw), i0, i1)
    if rc != 0:
        raise ValueError("oracle_forward: invalid arguments")
    return su, sv, sw


def adjoint(u, v, w, dsu, dsv, dsw, c: Coefficients):
    """(du, dv, dw) = J(u,v,w)^T (dsu, dsv, dsw)."""
    fields = [_f64(a) for a in (u, v, w, dsu, dsv, dsw)]
    nx, ny, nz = _check_fields(*fields)
    outs = [np.zeros((nx, ny, nz)) for _ in range(3)]
    rc = _lib().oracle_adjoint(nx, ny, nz, c.tcx, c.tcy, _p(c.tzc1), _p(c.tzc2), _p(c.tzd1),
                               _p(c.tzd2), *(_p(a) for a in fields), *(_p(o) for o in outs))
    if rc != 0:
        raise ValueError("oracle_adjoint: invalid arguments")
    return tuple(outs)


def integrate(u, v, w, c: Coefficients, dt, base=None):
    """The source terms integrated into the flow fields (Sec. 2.1: later in
    the timestep the source terms are added to the prognostic fields):
    out_f = base_f + dt * s_f for f in u, v, w, with (su, sv, sw) from
    ``forward`` and base = (u, v, w) unless given (one explicit step; a
    leapfrog step passes the previous time level as base and 2 dt).  Returns
    (u_out, v_out, w_out)."""
    su, sv, sw = forward(u, v, w, c)
    if base is None:
        base = (u, v, w)
    b = [_f64(x) for x in base]
    _check_fields(su, *b)
    dt = float(dt)
    return tuple(bf + dt * s for bf, s in zip(b, (su, sv, sw)))
