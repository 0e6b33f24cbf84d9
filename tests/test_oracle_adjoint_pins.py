"""Pins for the oracle's adjoint (transpose of the forward's Jacobian).

The forward map F(u, v, w) is quadratic (every term is coefficient * a * (b + c)
of two state values), so its tangent is exactly F(x + d) - F(x) - F(d) and a
central difference with any step is exact.  On small-integer inputs with
dyadic coefficients every FP64 operation is exact, so the dot-product identity
<J d, l> = <d, J^T l> holds with equality and is checked in rational arithmetic.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import workload


def dyadic_coeffs(nz, seed):
    z = np.arange(nz, dtype=np.float64)
    rng = np.random.default_rng(seed)
    rho = 2.0 ** (-rng.integers(0, 3, nz)).astype(np.float64)
    rhon = 2.0 ** (-rng.integers(0, 3, nz)).astype(np.float64)
    return oracle.coefficients(workload.custom_grid(z, z - 0.5, rho, rhon, 1.0, 2.0))


def ints(shape, seed, base):
    return [workload.small_int_field(shape, -3, 3, seed, base + f) for f in range(3)]


def fdot(a_list, b_list):
    s = Fr(0)
    for a, b in zip(a_list, b_list):
        for x, y in zip(a.ravel(), b.ravel()):
            if x and y:
                s += Fr(float(x)) * Fr(float(y))
    return s


@pytest.mark.parametrize("shape,seed", [((4, 4, 5), 1), ((3, 5, 4), 2), ((2, 3, 3), 3),
                                        ((1, 4, 6), 4)])
def test_dot_product_identity_exact(shape, seed):
    c = dyadic_coeffs(shape[2], seed)
    x = ints(shape, seed, 0)
    d = ints(shape, seed, 3)
    lam = ints(shape, seed, 6)
    fx = oracle.forward(*x, c)
    fd = oracle.forward(*d, c)
    fxd = oracle.forward(*[a + b for a, b in zip(x, d)], c)
    jd = [a - b - e for a, b, e in zip(fxd, fx, fd)]        # exact tangent J(x) d
    jt = oracle.adjoint(*x, *lam, c)
    assert fdot(jd, lam) == fdot(d, jt)


def test_central_difference_columns_exact():
    """(F(x + e_p) - F(x - e_p)) / 2 is column p of J(x) exactly; its dot with l
    must equal entry p of J^T l, for probes in every field and at the
    boundary levels."""
    shape = (3, 4, 5)
    c = dyadic_coeffs(5, 9)
    x = ints(shape, 9, 0)
    lam = ints(shape, 9, 6)
    jt = oracle.adjoint(*x, *lam, c)
    probes = [(0, (0, 0, 0)), (0, (1, 2, 4)), (0, (2, 3, 2)), (1, (0, 3, 1)), (1, (2, 0, 4)),
              (1, (1, 1, 0)), (2, (1, 2, 0)), (2, (0, 0, 4)), (2, (2, 1, 2)), (2, (1, 3, 3))]
    for f, p in probes:
        xp = [a.copy() for a in x]
        xm = [a.copy() for a in x]
        xp[f][p] += 1.0
        xm[f][p] -= 1.0
        col = [(a - b) / 2 for a, b in zip(oracle.forward(*xp, c), oracle.forward(*xm, c))]
        assert fdot(col, lam) == Fr(float(jt[f][p]))


def test_adjoint_is_linear_in_state_and_cotangent():
    """J^T(x) l is bilinear in (x, l): checked exactly on dyadic inputs."""
    shape = (3, 3, 4)
    c = dyadic_coeffs(4, 5)
    x1, x2 = ints(shape, 5, 0), ints(shape, 5, 3)
    l1 = ints(shape, 5, 6)
    a = oracle.adjoint(*[p + q for p, q in zip(x1, x2)], *l1, c)
    b = oracle.adjoint(*x1, *l1, c)
    e = oracle.adjoint(*x2, *l1, c)
    for r, s, t in zip(a, b, e):
        assert np.array_equal(r, s + t)


def test_adjoint_ignores_cotangents_on_unwritten_levels():
    """su, sv at the surface and sw at the surface and lid are constants (zero),
    so cotangents there contribute nothing."""
    shape = (3, 4, 5)
    c = dyadic_coeffs(5, 6)
    x = ints(shape, 6, 0)
    lam = [np.zeros(shape) for _ in range(3)]
    lam[0][..., 0] = 1.0
    lam[1][..., 0] = 1.0
    lam[2][..., 0] = 1.0
    lam[2][..., -1] = 1.0
    for g in oracle.adjoint(*x, *lam, c):
        assert not g.any()


def test_dot_product_identity_stretched_grid():
    shape = (6, 5, 12)
    c = oracle.coefficients(workload.vertical_grid(12))
    x = workload.winds(*shape, seed=31)
    d = workload.cotangents(*shape, seed=32)
    lam = workload.cotangents(*shape, seed=33)
    h = 2.0 ** -10
    fp = oracle.forward(*[a + h * b for a, b in zip(x, d)], c)
    fm = oracle.forward(*[a - h * b for a, b in zip(x, d)], c)
    jd = [(a - b) / (2 * h) for a, b in zip(fp, fm)]
    jt = oracle.adjoint(*x, *lam, c)
    lhs = sum(float(np.sum(a * b)) for a, b in zip(jd, lam))
    rhs = sum(float(np.sum(a * b)) for a, b in zip(d, jt))
    mag = sum(float(np.sum(np.abs(a * b))) for a, b in zip(d, jt))
    assert abs(lhs - rhs) <= 1e-9 * mag
