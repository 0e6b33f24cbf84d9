"""Pins for ``oracle.integrate``: the source terms added into the flow fields.

What fixes the result independently of the oracle: the exact rational
skew-symmetric tendencies (``skew_form``) added to the base fields, the
zero-step identity, and the energy budget of one explicit step.  Because the
scheme conserves kinetic energy (sum of m u*su + ... = 0), one forward-Euler
step changes the energy by exactly dt^2 times the weighted squared norm of
the tendencies.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import skew_form
import workload
from test_oracle_pins import as_obj, dyadic_grid, exact, int_fields


def _coeffs(grid):
    return oracle.coefficients(grid)


@pytest.mark.parametrize("separate_base", [False, True])
def test_integrate_zero_step_returns_base_bitwise(separate_base):
    shape = (6, 5, 8)
    grid = workload.vertical_grid(8)
    u, v, w = workload.winds(*shape, seed=31)
    base = workload.winds(*shape, seed=32) if separate_base else None
    out = oracle.integrate(u, v, w, _coeffs(grid), 0.0, base)
    for o, b in zip(out, base if separate_base else (u, v, w)):
        assert np.array_equal(o, b)


@pytest.mark.parametrize("separate_base,dt", [(False, 0.125), (True, 0.25), (True, -0.5)])
def test_integrate_equals_base_plus_exact_tendency(separate_base, dt):
    shape = (4, 5, 6)
    grid = dyadic_grid(6, seed=33)
    u, v, w = int_fields(shape, 33)
    base = tuple(workload.small_int_field(shape, -5, 5, 34, f) for f in range(3)) if separate_base else None
    out = oracle.integrate(u, v, w, _coeffs(grid), dt, base)
    ref = skew_form.tendencies(u, v, w, grid.dx, grid.dy, grid.z, grid.zn, grid.rho, grid.rhon)
    for o, b, r in zip(out, base if separate_base else (u, v, w), ref):
        assert (exact(o) == exact(b) + Fr(dt) * as_obj(r)).all()


def test_integrate_forward_euler_energy_budget():
    shape = (8, 6, 16)
    grid = workload.vertical_grid(16)
    u, v, w = workload.winds(*shape, seed=35)
    w[..., 0] = 0.0
    w[..., -1] = 0.0
    c = _coeffs(grid)
    dt = 3.0
    su, sv, sw = oracle.forward(u, v, w, c)
    uo, vo, wo = oracle.integrate(u, v, w, c, dt)
    dz = np.zeros(grid.nz)
    dz[1:] = np.diff(grid.z)
    dzn_up = np.zeros(grid.nz)
    dzn_up[:-1] = np.diff(grid.zn)
    mu = (grid.rhon * dz)[None, None, :]
    mw = (grid.rho * dzn_up)[None, None, :]

    def energy(a, b, c_):
        return float(np.sum(mu * (a * a + b * b)) + np.sum(mw * c_ * c_))

    growth = energy(uo, vo, wo) - energy(u, v, w)
    expect = dt * dt * energy(su, sv, sw)
    assert expect > 0
    assert abs(growth - expect) <= 1e-9 * energy(u, v, w)
    # the cross term 2 dt <u, S> vanishes; a step of -dt grows the energy equally
    back = oracle.integrate(u, v, w, c, -dt)
    assert abs((energy(*back) - energy(u, v, w)) - expect) <= 1e-9 * energy(u, v, w)


def test_integrate_rejects_mismatched_base():
    shape = (4, 4, 5)
    grid = workload.vertical_grid(5)
    u, v, w = workload.winds(*shape, seed=36)
    bad = (u, v, w[:, :, :4])
    with pytest.raises(ValueError):
        oracle.integrate(u, v, w, _coeffs(grid), 1.0, bad)
