"""Seeded synthetic workloads for the momentum-advection stencil.

This module only *draws inputs*: wind fields, cotangents, the vertical grid
(level heights and reference densities) and ensemble member shapes.  It holds
none of the advection arithmetic (no coefficients, no stencil), so both the
CPU oracle and the CUDA path can be fed from it without sharing any of the
method's code.

Recipe (stand-in for the MONC stratus-cloud test case of the paper's Sec. 5,
which is not available here):

* layout ``[nx][ny][nz]`` with z contiguous (the Fortran ``u(k,j,i)`` order of
  Listing 1), C-contiguous numpy arrays;
* ``u, v, w = U(-10, 10) + 2 sin(2 pi i / nx) cos(2 pi j / ny)`` m/s; the
  uniform part comes from raw PCG64 words (``SeedSequence([seed, member,
  field])``) mapped as ``-10 + 20 * (bits >> 11) * 2**-53``;
* vertical grid: ``z(1) = 0``, ``z(k) = z(k-1) + dz1 * r**(k-2)`` with
  ``dz1 = 10 m``, ``r = 1.05``; ``zn(k) = (z(k-1) + z(k)) / 2`` for ``k >= 2``
  (``zn(1) = -dz1 / 2``, a mirror level that no formula reads);
  ``rho(z) = exp(-z / 8000)`` on both level sets;
* horizontal spacing ``dx = dy = 50 m``;
* cotangents ``N(0, 1)`` by Box-Muller on raw PCG64 words.

Arrays are 0-based: level ``k`` (1-based in the paper) is stored at ``[k-1]``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DEFAULT_SEED = 1545
DX = 50.0
DY = 50.0
DZ1 = 10.0
STRETCH = 1.05
SCALE_HEIGHT = 8000.0

FIELD_U, FIELD_V, FIELD_W, FIELD_DSU, FIELD_DSV, FIELD_DSW = range(6)


@dataclass(frozen=True)
class VerticalGrid:
    """Heights and reference densities of the two staggered level sets."""

    z: np.ndarray     # w-levels (cell tops), length nz
    zn: np.ndarray    # u/v-levels (cell centres), length nz
    rho: np.ndarray   # density on w-levels
    rhon: np.ndarray  # density on u/v-levels
    dx: float
    dy: float

    @property
    def nz(self) -> int:
        return int(self.z.shape[0])


def vertical_grid(nz: int, dz1: float = DZ1, ratio: float = STRETCH,
                  scale_height: float = SCALE_HEIGHT, dx: float = DX,
                  dy: float = DY) -> VerticalGrid:
    """Stretched vertical grid with an exponential reference density."""
    if nz < 1:
        raise ValueError("nz must be >= 1")
    z = np.zeros(nz, dtype=np.float64)
    for k in range(1, nz):
        z[k] = z[k - 1] + dz1 * ratio ** (k - 1)
    zn = np.empty(nz, dtype=np.float64)
    zn[0] = -0.5 * dz1
    zn[1:] = 0.5 * (z[:-1] + z[1:])
    rho = np.exp(-z / scale_height)
    rhon = np.exp(-zn / scale_height)
    return VerticalGrid(z=z, zn=zn, rho=rho, rhon=rhon, dx=float(dx), dy=float(dy))


def custom_grid(z, zn, rho, rhon, dx: float, dy: float) -> VerticalGrid:
    """A grid from explicit level arrays (used by tests with dyadic values)."""
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (z, zn, rho, rhon)]
    n = arrs[0].shape[0]
    if any(a.shape != (n,) for a in arrs):
        raise ValueError("level arrays must all have shape (nz,)")
    return VerticalGrid(*arrs, dx=float(dx), dy=float(dy))


def _raw_words(n: int, seed: int, member: int, field: int) -> np.ndarray:
    bg = np.random.PCG64(np.random.SeedSequence([int(seed), int(member), int(field)]))
    return bg.random_raw(n).astype(np.uint64, copy=False)


def _unit_uniform(n: int, seed: int, member: int, field: int) -> np.ndarray:
    """U[0,1) doubles from raw words: (bits >> 11) * 2**-53."""
    w = _raw_words(n, seed, member, field)
    return (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def wind_field(nx: int, ny: int, nz: int, field: int, seed: int = DEFAULT_SEED,
               member: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """One wind component, shape (nx, ny, nz), float64."""
    n = nx * ny * nz
    a = _unit_uniform(n, seed, member, field)
    a *= 20.0
    a -= 10.0
    a = a.reshape(nx, ny, nz)
    sx = np.sin(2.0 * math.pi * np.arange(nx, dtype=np.float64) / nx)
    cy = np.cos(2.0 * math.pi * np.arange(ny, dtype=np.float64) / ny)
    pert = 2.0 * sx[:, None] * cy[None, :]
    a += pert[:, :, None]
    if out is not None:
        out[...] = a
        return out
    return a


def winds(nx: int, ny: int, nz: int, seed: int = DEFAULT_SEED, member: int = 0):
    """(u, v, w) for one grid."""
    return tuple(wind_field(nx, ny, nz, f, seed, member) for f in (FIELD_U, FIELD_V, FIELD_W))


def cotangent_field(nx: int, ny: int, nz: int, field: int, seed: int = DEFAULT_SEED,
                    member: int = 0) -> np.ndarray:
    """Standard-normal field via Box-Muller on two uniform streams."""
    n = nx * ny * nz
    u1 = _unit_uniform(n, seed, member, 16 + 2 * field)
    u2 = _unit_uniform(n, seed, member, 17 + 2 * field)
    r = np.sqrt(-2.0 * np.log1p(-u1))          # 1 - u1 in (0, 1]
    return (r * np.cos(2.0 * math.pi * u2)).reshape(nx, ny, nz)


def cotangents(nx: int, ny: int, nz: int, seed: int = DEFAULT_SEED, member: int = 0):
    return tuple(cotangent_field(nx, ny, nz, f, seed, member)
                 for f in (FIELD_DSU, FIELD_DSV, FIELD_DSW))


def small_int_field(shape, lo: int, hi: int, seed: int, field: int) -> np.ndarray:
    """Integers in [lo, hi] stored as float64 (exact-arithmetic test inputs)."""
    n = int(np.prod(shape))
    w = _raw_words(n, seed, 0, 100 + field)
    span = np.uint64(hi - lo + 1)
    return ((w % span).astype(np.int64) + lo).astype(np.float64).reshape(shape)


ENSEMBLE_NXY = tuple(range(96, 768 + 1, 32))
ENSEMBLE_NZ = (32, 64, 128)


def ensemble_shapes(n_members: int = 48, seed: int = DEFAULT_SEED):
    """Uneven member shapes: nx, ny from {96..768 step 32}, nz from {32, 64, 128}."""
    w = _raw_words(3 * n_members, seed, 0, 200).reshape(n_members, 3)
    out = []
    for m in range(n_members):
        nx = ENSEMBLE_NXY[int(w[m, 0] % np.uint64(len(ENSEMBLE_NXY)))]
        ny = ENSEMBLE_NXY[int(w[m, 1] % np.uint64(len(ENSEMBLE_NXY)))]
        nz = ENSEMBLE_NZ[int(w[m, 2] % np.uint64(len(ENSEMBLE_NZ)))]
        out.append((nx, ny, nz))
    return out
