"""Pins for the CPU oracle's forward pass and coefficients.

Each test checks the oracle against something other than itself: the
skew-symmetric definition of the Piacsek-Williams scheme (Sec. 2.1) evaluated
exactly, closed-form impulse and gradient responses, exact symmetries of
Listing 1, and discrete kinetic-energy conservation.  Inputs are small
integers with dyadic grid data wherever exactness is claimed, so every FP64
operation in the oracle is exact there and comparisons are bitwise.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import skew_form
import workload


# ---------------------------------------------------------------- helpers
def dyadic_grid(nz, dx=1.0, dy=2.0, seed=0):
    """Uniform dz = 1 with power-of-two densities: all coefficients dyadic."""
    z = np.arange(nz, dtype=np.float64)
    zn = z - 0.5
    rng = np.random.default_rng(seed)
    rho = 2.0 ** (-rng.integers(0, 3, nz)).astype(np.float64)
    rhon = 2.0 ** (-rng.integers(0, 3, nz)).astype(np.float64)
    return workload.custom_grid(z, zn, rho, rhon, dx, dy)


def int_fields(shape, seed, lo=-3, hi=3):
    return tuple(workload.small_int_field(shape, lo, hi, seed, f) for f in range(3))


def exact(a):
    return np.array([[[Fr(float(x)) for x in col] for col in pl] for pl in a], dtype=object)


def as_obj(nested):
    return np.array(nested, dtype=object)


def normwise(a, ref):
    return float(np.max(np.abs(a - ref)) / max(np.max(np.abs(ref)), 1e-300))


def run(u, v, w, grid):
    return oracle.forward(u, v, w, oracle.coefficients(grid))


# ---------------------------------------------------------------- coefficients
def test_coefficients_uniform_closed_form():
    nz, dz = 7, 25.0
    z = dz * np.arange(nz)
    zn = z - dz / 2
    g = workload.custom_grid(z, zn, np.ones(nz), np.ones(nz), 50.0, 40.0)
    c = oracle.coefficients(g)
    assert c.tcx == 1.0 / 200.0 and c.tcy == 1.0 / 160.0
    q = 1.0 / (4.0 * dz)
    assert np.all(c.tzc1[1:] == q) and np.all(c.tzc2[1:] == q)
    assert np.all(c.tzd1[1:-1] == q) and np.all(c.tzd2[1:-1] == q)
    # levels no formula reads are zero
    assert c.tzc1[0] == 0 and c.tzc2[0] == 0
    assert c.tzd1[0] == c.tzd1[-1] == c.tzd2[0] == c.tzd2[-1] == 0


def test_coefficients_flux_telescoping_stretched():
    """tzc1(k+1) rho_n(k+1) dz(k+1) = tzc2(k) rho_n(k) dz(k) = rho_w(k)/4, and the
    analogue for tzd on the w cells: the identities that make the scheme's
    vertical fluxes telescope."""
    g = workload.vertical_grid(64)
    c = oracle.coefficients(g)
    dz = np.diff(g.z)                      # dz[k-1] = z[k] - z[k-1]
    k = np.arange(1, 63)
    lhs = c.tzc1[k + 1] * g.rhon[k + 1] * dz[k]
    mid = c.tzc2[k] * g.rhon[k] * dz[k - 1]
    np.testing.assert_allclose(lhs, g.rho[k] / 4, rtol=1e-15, atol=0)
    np.testing.assert_allclose(mid, g.rho[k] / 4, rtol=1e-15, atol=0)
    dzn = np.diff(g.zn)                    # dzn[k-1] = zn[k] - zn[k-1]
    k = np.arange(2, 62)
    a = c.tzd1[k + 1] * g.rho[k + 1] * dzn[k + 1]
    b = c.tzd2[k] * g.rho[k] * dzn[k]
    np.testing.assert_allclose(a, g.rhon[k + 1] / 4, rtol=1e-15, atol=0)
    np.testing.assert_allclose(b, g.rhon[k + 1] / 4, rtol=1e-15, atol=0)


# ---------------------------------------------------------------- definition
@pytest.mark.parametrize("shape,seed", [((4, 4, 4), 1), ((5, 3, 4), 2), ((3, 5, 6), 3),
                                        ((2, 2, 3), 4), ((1, 3, 5), 5)])
def test_forward_equals_skew_symmetric_definition_exactly(shape, seed):
    grid = dyadic_grid(shape[2], seed=seed)
    u, v, w = int_fields(shape, seed)
    got = run(u, v, w, grid)
    ref = skew_form.tendencies(u, v, w, grid.dx, grid.dy, grid.z, grid.zn, grid.rho, grid.rhon)
    for g, r in zip(got, ref):
        assert (exact(g) == as_obj(r)).all()


def test_forward_matches_definition_on_stretched_grid():
    grid = workload.vertical_grid(6)
    u, v, w = workload.winds(4, 5, 6, seed=7)
    got = run(u, v, w, grid)
    ref = skew_form.tendencies(u, v, w, grid.dx, grid.dy, grid.z, grid.zn, grid.rho, grid.rhon)
    for g, r in zip(got, ref):
        r = np.array([[[float(x) for x in col] for col in pl] for pl in r])
        assert normwise(g, r) < 1e-14


# ---------------------------------------------------------------- closed forms
def _impulse(shape, where, field):
    f = [np.zeros(shape) for _ in range(3)]
    f[field][where] = 1.0
    return f


def test_impulse_u_alone():
    shape, q = (5, 6, 5), (2, 3, 2)
    grid = workload.vertical_grid(5)
    c = oracle.coefficients(grid)
    su, sv, sw = run(*_impulse(shape, q, 0), grid)
    exp = np.zeros(shape)
    exp[3, 3, 2], exp[1, 3, 2] = c.tcx, -c.tcx
    assert np.array_equal(su, exp)
    assert not sv.any() and not sw.any()


def test_impulse_v_alone():
    shape, q = (5, 6, 5), (2, 3, 3)
    grid = workload.vertical_grid(5)
    c = oracle.coefficients(grid)
    su, sv, sw = run(*_impulse(shape, q, 1), grid)
    exp = np.zeros(shape)
    exp[2, 4, 3], exp[2, 2, 3] = c.tcy, -c.tcy
    assert np.array_equal(sv, exp)
    assert not su.any() and not sw.any()


def test_impulse_w_alone():
    shape, q = (4, 4, 7), (1, 2, 3)
    grid = workload.vertical_grid(7)
    c = oracle.coefficients(grid)
    su, sv, sw = run(*_impulse(shape, q, 2), grid)
    exp = np.zeros(shape)
    exp[1, 2, 4], exp[1, 2, 2] = c.tzd1[4], -c.tzd2[2]
    assert np.array_equal(sw, exp)
    assert not su.any() and not sv.any()


def test_impulse_u_in_uniform_v():
    """u = delta_q, v = 1: su gets +-tcx along x and +-2 tcy along y; sv sees the
    u impulse through the two x-faces it touches."""
    shape, (i, j, k) = (6, 5, 4), (2, 2, 1)
    grid = workload.vertical_grid(4)
    c = oracle.coefficients(grid)
    u, v, w = _impulse(shape, (i, j, k), 0)
    v[:] = 1.0
    su, sv, sw = run(u, v, w, grid)
    e_su = np.zeros(shape)
    e_su[i + 1, j, k], e_su[i - 1, j, k] = c.tcx, -c.tcx
    e_su[i, j + 1, k], e_su[i, j - 1, k] = 2 * c.tcy, -2 * c.tcy
    e_sv = np.zeros(shape)
    e_sv[i + 1, j, k] = e_sv[i + 1, j - 1, k] = c.tcx
    e_sv[i, j, k] = e_sv[i, j - 1, k] = -c.tcx
    assert np.array_equal(su, e_su)
    assert np.array_equal(sv, e_sv)
    assert not sw.any()


def test_impulse_w_in_uniform_u():
    """w = delta_q, u = 1: su feels the w impulse through the top face of the
    cell below and the bottom face of the cell above; sw gets the x-advection
    by the uniform u plus the vertical self-interaction."""
    shape, (i, j, k) = (5, 4, 7), (2, 1, 3)
    grid = workload.vertical_grid(7)
    c = oracle.coefficients(grid)
    u, v, w = _impulse(shape, (i, j, k), 2)
    u[:] = 1.0
    su, sv, sw = run(u, v, w, grid)
    e_su = np.zeros(shape)
    e_su[i, j, k + 1] = e_su[i - 1, j, k + 1] = c.tzc1[k + 1]
    e_su[i, j, k] = e_su[i - 1, j, k] = -c.tzc2[k]
    e_sw = np.zeros(shape)
    e_sw[i + 1, j, k], e_sw[i - 1, j, k] = 2 * c.tcx, -2 * c.tcx
    e_sw[i, j, k + 1], e_sw[i, j, k - 1] = c.tzd1[k + 1], -c.tzd2[k - 1]
    assert np.array_equal(su, e_su)
    assert np.array_equal(sw, e_sw)
    assert not sv.any()


def test_zero_tendency_uniform_u():
    shape = (4, 5, 6)
    u = np.full(shape, 3.7)
    su, sv, sw = run(u, np.zeros(shape), np.zeros(shape), workload.vertical_grid(6))
    assert not su.any() and not sv.any() and not sw.any()


def test_uniform_wind_only_top_level_of_su_sv_is_nonzero():
    """Uniform (U, V, W) with constant density and uniform dz: every flux cancels
    except the omitted lid flux, leaving 2 tzc1(top) U W at the top of su."""
    nz = 6
    z = 10.0 * np.arange(nz)
    g = workload.custom_grid(z, z - 5.0, np.ones(nz), np.ones(nz), 50.0, 50.0)
    c = oracle.coefficients(g)
    U, V, W = 2.5, -1.25, 0.75
    shape = (4, 4, nz)
    su, sv, sw = run(np.full(shape, U), np.full(shape, V), np.full(shape, W), g)
    assert not su[..., :-1].any() and not sv[..., :-1].any() and not sw.any()
    np.testing.assert_allclose(su[..., -1], 2 * c.tzc1[-1] * U * W, rtol=1e-15)
    np.testing.assert_allclose(sv[..., -1], 2 * c.tzc1[-1] * V * W, rtol=1e-15)


def test_linear_gradient_gives_skew_symmetric_consistency():
    """u = U + b x along x: the x term equals -1.5 u b (half flux form -2ub,
    half advective form -ub), which fixes tcx = 1/(4 dx)."""
    nx, ny, nz = 12, 3, 3
    grid = workload.vertical_grid(nz)
    b = 0.01
    x = grid.dx * np.arange(nx)
    u = np.broadcast_to((1.5 + b * x)[:, None, None], (nx, ny, nz)).copy()
    su, _, _ = run(u, np.zeros_like(u), np.zeros_like(u), grid)
    inner = slice(1, nx - 1)
    np.testing.assert_allclose(su[inner, :, 1:], -1.5 * b * u[inner, :, 1:], rtol=1e-12)


def test_vertical_gradient_constant_density():
    """u = a + b zn(k), uniform w = W, constant density, uniform dz: the vertical
    term is -W b at interior levels."""
    nz, dz = 8, 20.0
    z = dz * np.arange(nz)
    zn = z - dz / 2
    g = workload.custom_grid(z, zn, np.ones(nz), np.ones(nz), 50.0, 50.0)
    a, b, W = 1.0, 0.02, 0.6
    shape = (3, 3, nz)
    u = np.broadcast_to(a + b * zn, shape).copy()
    su, _, _ = run(u, np.zeros(shape), np.full(shape, W), g)
    np.testing.assert_allclose(su[..., 1:-1], -W * b, rtol=1e-12)


# ---------------------------------------------------------------- symmetries
def test_x_reflection_antisymmetry_bitwise():
    shape = (6, 5, 5)
    u, v, w = workload.winds(*shape, seed=11)
    grid = workload.vertical_grid(5)
    su, sv, sw = run(u, v, w, grid)
    nx = shape[0]
    i = np.arange(nx)
    r_u = (-i - 1) % nx      # u sits at i+1/2: its mirror image is -i-1
    r_c = (-i) % nx          # v, w sit at integer x
    su2, sv2, sw2 = run(-u[r_u], v[r_c], w[r_c], grid)
    assert np.array_equal(su2, -su[r_u])
    assert np.array_equal(sv2, sv[r_c])
    assert np.array_equal(sw2, sw[r_c])


def test_y_reflection_antisymmetry_bitwise():
    shape = (5, 6, 5)
    u, v, w = workload.winds(*shape, seed=12)
    grid = workload.vertical_grid(5)
    su, sv, sw = run(u, v, w, grid)
    ny = shape[1]
    j = np.arange(ny)
    r_v = (-j - 1) % ny
    r_c = (-j) % ny
    su2, sv2, sw2 = run(u[:, r_c], -v[:, r_v], w[:, r_c], grid)
    assert np.array_equal(sv2, -sv[:, r_v])
    assert np.array_equal(su2, su[:, r_c])
    assert np.array_equal(sw2, sw[:, r_c])


def test_periodic_shift_equivariance_bitwise():
    shape = (5, 7, 4)
    u, v, w = workload.winds(*shape, seed=13)
    grid = workload.vertical_grid(4)
    out = run(u, v, w, grid)
    sh = (2, -3)
    rolled = [np.roll(f, sh, axis=(0, 1)) for f in (u, v, w)]
    out2 = run(*rolled, grid)
    for a, b in zip(out2, out):
        assert np.array_equal(a, np.roll(b, sh, axis=(0, 1)))


def test_power_of_two_scaling_bitwise():
    shape = (4, 4, 5)
    u, v, w = workload.winds(*shape, seed=14)
    grid = workload.vertical_grid(5)
    out = run(u, v, w, grid)
    out2 = run(8.0 * u, 8.0 * v, 8.0 * w, grid)
    for a, b in zip(out2, out):
        assert np.array_equal(a, 64.0 * b)


def test_su_sv_transpose_symmetry_bitwise():
    """With nx = ny and dx = dy, exchanging x<->y and u<->v maps su to sv: this
    ties the reconstructed sv to the printed su (Listing 1)."""
    shape = (5, 5, 6)
    u, v, w = workload.winds(*shape, seed=15)
    grid = workload.vertical_grid(6)
    su, sv, sw = run(u, v, w, grid)
    t = (1, 0, 2)
    su2, sv2, sw2 = run(v.transpose(t), u.transpose(t), w.transpose(t), grid)
    assert np.array_equal(sv2, su.transpose(t))
    assert np.array_equal(su2, sv.transpose(t))
    assert np.array_equal(sw2, sw.transpose(t))


# ---------------------------------------------------------------- energy
def _energy_terms(u, v, w, su, sv, sw, g):
    dz = np.zeros(g.nz)
    dz[1:] = np.diff(g.z)
    dzn_up = np.zeros(g.nz)
    dzn_up[:-1] = np.diff(g.zn)           # dzn(k+1) = zn[k+1] - zn[k]
    wu = (g.rhon * dz)[None, None, :]
    ww = (g.rho * dzn_up)[None, None, :]
    return [wu * u * su, wu * v * sv, ww * w * sw]


def test_energy_conservation_exact_dyadic():
    shape = (4, 5, 6)
    grid = dyadic_grid(6, seed=21)
    u, v, w = int_fields(shape, 21)
    w[..., 0] = 0.0
    w[..., -1] = 0.0
    su, sv, sw = run(u, v, w, grid)
    total = Fr(0)
    for t in _energy_terms(u, v, w, su, sv, sw, grid):
        total += sum(Fr(float(x)) for x in t.ravel())
    assert total == 0


def test_energy_conservation_stretched():
    shape = (8, 6, 16)
    grid = workload.vertical_grid(16)
    u, v, w = workload.winds(*shape, seed=22)
    w[..., 0] = 0.0
    w[..., -1] = 0.0
    su, sv, sw = run(u, v, w, grid)
    terms = _energy_terms(u, v, w, su, sv, sw, grid)
    s = sum(float(np.sum(t)) for t in terms)
    mag = sum(float(np.sum(np.abs(t))) for t in terms)
    assert abs(s) <= 1e-13 * mag


# ---------------------------------------------------------------- hand-worked point
def test_hand_worked_point():
    """One point of su, sv, sw on a 3x3x4 grid with dx = dy = 1 (tcx = tcy = 1/4),
    uniform dz = 1 and unit density (tzc = tzd = 1/4), evaluated by hand from
    Listing 1 and its v/w analogues; the worked arithmetic is in
    tests/golden/hand_point.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hand_point.txt")
    vals = {}
    fields = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, rest = line.split("=", 1)
            key = key.strip()
            if key in ("u", "v", "w"):
                fields[key] = np.array([float(x) for x in rest.split()]).reshape(3, 3, 4)
            else:
                vals[key] = float(Fr(rest.strip()))
    nz = 4
    z = np.arange(nz, dtype=np.float64)
    g = workload.custom_grid(z, z - 0.5, np.ones(nz), np.ones(nz), 1.0, 1.0)
    su, sv, sw = run(fields["u"], fields["v"], fields["w"], g)
    assert su[1, 1, 1] == vals["su_111"]
    assert sv[1, 1, 1] == vals["sv_111"]
    assert sw[1, 1, 1] == vals["sw_111"]
    assert su[1, 1, 3] == vals["su_113"]
