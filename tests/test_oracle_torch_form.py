"""The oracle against a second, whole-array formulation in FP64 torch ops
(``torch_form``), and the oracle's adjoint against torch autograd of it.

These are cross-checks between two independently written implementations:
the pins in test_oracle_pins.py are what fix the oracle to the paper; here a
mistake in either formulation's indexing would show as a disagreement far
above rounding.
"""
import numpy as np
import pytest
import torch

import oracle
import torch_form
import workload

SHAPES = [(5, 4, 6), (8, 8, 16), (1, 1, 3), (3, 5, 4), (16, 12, 64)]


def _coeffs(grid):
    c = oracle.coefficients(grid)
    return c, (c.tcx, c.tcy, c.tzc1, c.tzc2, c.tzd1, c.tzd2)


def _normwise(a, ref):
    return float(np.max(np.abs(a - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("shape", SHAPES)
def test_torch_form_matches_oracle(shape):
    grid = workload.vertical_grid(shape[2])
    c, tabs = _coeffs(grid)
    x = workload.winds(*shape, seed=61)
    ref = oracle.forward(*x, c)
    got = torch_form.source_terms(*(torch.from_numpy(a) for a in x), *tabs)
    for g, r, name in zip(got, ref, ("su", "sv", "sw")):
        assert _normwise(g.numpy(), r) <= 1e-14, name


@pytest.mark.parametrize("shape", SHAPES)
def test_torch_autograd_matches_oracle_adjoint(shape):
    grid = workload.vertical_grid(shape[2])
    c, tabs = _coeffs(grid)
    x = workload.winds(*shape, seed=62)
    lam = workload.cotangents(*shape, seed=63)
    ref = oracle.adjoint(*x, *lam, c)
    got = torch_form.adjoint_by_autograd(*x, *lam, tabs)
    for g, r, name in zip(got, ref, ("du", "dv", "dw")):
        assert _normwise(g, r) <= 1e-13, name
