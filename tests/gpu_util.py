"""Helpers shared by the GPU parity tests (inputs, tolerances, the library)."""
import numpy as np
import torch

import oracle
import workload
from paper_2010_01545_gb300 import build, torch_api

_built = False


def ensure_built():
    global _built
    if not _built:
        build.build()
        _built = True


def lib_coeffs(grid):
    return torch_api.coefficients_from_grid(grid)


def make_op(shape, dtype="f64", grid=None, **kw):
    ensure_built()
    grid = grid or workload.vertical_grid(shape[2])
    return torch_api.Advect(*shape, lib_coeffs(grid), dtype, **kw), grid


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().to("cpu", torch.float64).numpy()


def normwise(a, ref):
    m = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(a - ref))) / (m if m > 0 else 1.0)


def oracle_forward(u, v, w, grid, i_range=None):
    return oracle.forward(u, v, w, oracle.coefficients(grid), i_range=i_range)


def oracle_adjoint(u, v, w, dsu, dsv, dsw, grid):
    return oracle.adjoint(u, v, w, dsu, dsv, dsw, oracle.coefficients(grid))
