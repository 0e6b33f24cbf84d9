"""GPU parity of the gather-form adjoint and of the autograd binding.

F64: within 1e-12 of the oracle's scatter adjoint, normwise per field.  F32:
the oracle runs on the same binary32-rounded inputs.  The autograd function's
backward must be the adjoint, and the dot-product identity must hold on the
GPU (the forward is quadratic, so its central difference is exact up to
rounding).
"""
import numpy as np
import pytest
import torch

import workload
from gpu_util import dev, host, make_op, normwise, oracle_adjoint

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 64), (33, 17, 65), (5, 7, 3), (1, 1, 3), (1, 6, 9), (7, 1, 9), (130, 66, 20),
          (16, 32, 128), (20, 14, 96), (17, 9, 48)]


@pytest.mark.parametrize("shape", SHAPES)
def test_adjoint_f64_matches_oracle(shape):
    op, grid = make_op(shape, "f64")
    x = workload.winds(*shape, seed=21)
    lam = workload.cotangents(*shape, seed=22)
    got = [host(t) for t in op.adjoint(*(dev(a) for a in (*x, *lam)))]
    ref = oracle_adjoint(*x, *lam, grid)
    for g, r, name in zip(got, ref, ("du", "dv", "dw")):
        err = normwise(g, r)
        assert err <= 1e-12, f"{name} normwise error {err:.3e} ({op.kernel_name(True)})"


# (20, 14, 96) and (17, 9, 48): the binary32 sweep's rows (24 and 12 k-blocks of 4 levels)
# straddle warps, so some vertical halos come from shared memory
@pytest.mark.parametrize("shape", [(64, 64, 64), (33, 17, 65), (1, 1, 4), (20, 14, 96), (17, 9, 48),
                                   (70, 42, 128)])
def test_adjoint_f32_matches_oracle_on_rounded_inputs(shape):
    op, grid = make_op(shape, "f32")
    x = [a.astype(np.float32).astype(np.float64) for a in workload.winds(*shape, seed=23)]
    lam = [a.astype(np.float32).astype(np.float64) for a in workload.cotangents(*shape, seed=24)]
    got = [host(t) for t in op.adjoint(*(dev(a, torch.float32) for a in (*x, *lam)))]
    ref = oracle_adjoint(*x, *lam, grid)
    if shape[2] % 4 == 0:
        assert op.kernel_name(True) == "adj_sweep"
    for g, r, name in zip(got, ref, ("du", "dv", "dw")):
        err = normwise(g, r)
        assert err <= 5e-6, f"{name} normwise error {err:.3e}"


@pytest.mark.parametrize("shape", [(64, 64, 64), (33, 17, 65), (16, 32, 128)])
def test_adjoint_f64_matches_torch_autograd(shape):
    """Against reverse-mode autograd of the whole-array FP64 torch-ops
    formulation: an adjoint that owes nothing to the hand-derived gather."""
    import oracle
    import torch_form
    op, grid = make_op(shape, "f64")
    c = oracle.coefficients(grid)
    x = workload.winds(*shape, seed=26)
    lam = workload.cotangents(*shape, seed=27)
    got = [host(t) for t in op.adjoint(*(dev(a) for a in (*x, *lam)))]
    ref = torch_form.adjoint_by_autograd(*x, *lam, (c.tcx, c.tcy, c.tzc1, c.tzc2, c.tzd1, c.tzd2))
    for g, r, name in zip(got, ref, ("du", "dv", "dw")):
        err = normwise(g, r)
        assert err <= 1e-12, f"{name} normwise error {err:.3e} ({op.kernel_name(True)})"


def test_adjoint_ignores_cotangents_on_unwritten_levels():
    shape = (6, 5, 7)
    op, _ = make_op(shape, "f64")
    x = [dev(a) for a in workload.winds(*shape, seed=25)]
    lam = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    lam[0][..., 0] = 1.0
    lam[1][..., 0] = 1.0
    lam[2][..., 0] = 1.0
    lam[2][..., -1] = 1.0
    for g in op.adjoint(*x, *lam):
        assert not host(g).any()


def test_autograd_backward_is_the_adjoint():
    from paper_2010_01545_gb300 import advect
    shape = (24, 20, 32)
    op, _ = make_op(shape, "f64")
    x = [dev(a).requires_grad_(True) for a in workload.winds(*shape, seed=26)]
    lam = [dev(a) for a in workload.cotangents(*shape, seed=27)]
    out = advect(*x, op)
    torch.autograd.backward(out, lam)
    ref = op.adjoint(*(t.detach() for t in x), *lam)
    for t, r in zip(x, ref):
        assert torch.equal(t.grad, r)


def _dyadic_coeffs(nz, seed):
    """Coefficients that are powers of two (unit spacings, power-of-two
    densities): with small-integer fields every operation of the forward and
    the adjoint, in any of the three arithmetics, is exact."""
    z = np.arange(nz, dtype=np.float64)
    rng = np.random.default_rng(seed)
    rho = 2.0 ** (-rng.integers(0, 3, nz)).astype(np.float64)
    rhon = 2.0 ** (-rng.integers(0, 3, nz)).astype(np.float64)
    return workload.custom_grid(z, z - 0.5, rho, rhon, 1.0, 2.0)


def _fsum_dot(a_list, b_list):
    """sum_f <a_f, b_f> in binary64: per-plane partial sums on the device,
    then a correctly rounded sum of the partials (math.fsum)."""
    import math
    parts = []
    for a, b in zip(a_list, b_list):
        parts.extend(torch.sum(a.to(torch.float64) * b.to(torch.float64), dim=(1, 2)).tolist())
    return math.fsum(parts)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64ff"])
def test_dot_product_identity_exact_on_gpu(dtype):
    """<J d, l> = <d, J^T l> with equality: J d is the exact tangent
    F(x + d) - F(x) - F(d) of the quadratic map, formed from three library
    forwards; on small-integer inputs with power-of-two coefficients nothing
    rounds, so both sides are the same rational number (several tiles in y
    and x, a ragged tail)."""
    shape = (70, 44, 64)
    grid = _dyadic_coeffs(shape[2], 51)
    op, _ = make_op(shape, dtype, grid=grid)
    tdt = op.torch_dtype
    ints = lambda base: [dev(workload.small_int_field(shape, -3, 3, 52, base + f), tdt) for f in range(3)]  # noqa: E731
    x, d, lam = ints(0), ints(3), ints(6)
    fx = op.forward(*x)
    fd = op.forward(*d)
    fxd = op.forward(*(a + b for a, b in zip(x, d)))
    jd = [a.double() - b.double() - c.double() for a, b, c in zip(fxd, fx, fd)]
    jt = op.adjoint(*x, *lam)
    lhs = _fsum_dot(jd, lam)
    rhs = _fsum_dot(d, jt)
    assert lhs != 0.0
    assert lhs == rhs, (lhs, rhs, op.kernel_name(True))


def test_dot_product_identity_on_gpu():
    """Random winds and directions at full scale: J d = (F(x + d) - F(x - d)) / 2
    exactly for the quadratic map, so only rounding separates the two sides;
    bound 1e-12 relative to sum |d * J^T l|."""
    shape = (32, 24, 64)
    op, _ = make_op(shape, "f64")
    x = [dev(a) for a in workload.winds(*shape, seed=28)]
    d = [dev(a) for a in workload.cotangents(*shape, seed=29)]
    lam = [dev(a) for a in workload.cotangents(*shape, seed=30)]
    fp = op.forward(*(a + b for a, b in zip(x, d)))
    fm = op.forward(*(a - b for a, b in zip(x, d)))
    jd = [(a - b) * 0.5 for a, b in zip(fp, fm)]
    jt = op.adjoint(*x, *lam)
    lhs = _fsum_dot(jd, lam)
    rhs = _fsum_dot(d, jt)
    mag = _fsum_dot([a.abs() for a in d], [b.abs() for b in jt])
    assert abs(lhs - rhs) <= 1e-12 * mag, (lhs, rhs, mag)


def test_central_differences_at_probe_points():
    """64 random probes (the differentiation workload's check): the FD
    directional derivative along e_p, dotted with the cotangents, equals
    entry p of the adjoint."""
    shape = (16, 16, 32)
    op, _ = make_op(shape, "f64")
    x = [dev(a) for a in workload.winds(*shape, seed=31)]
    lam = [dev(a) for a in workload.cotangents(*shape, seed=32)]
    jt = [host(t) for t in op.adjoint(*x, *lam)]
    rng = np.random.default_rng(33)
    h = 1e-6
    for _ in range(64):
        f = int(rng.integers(3))
        p = tuple(int(rng.integers(n)) for n in shape)
        xp = [a.clone() for a in x]
        xm = [a.clone() for a in x]
        xp[f][p] += h
        xm[f][p] -= h
        fp = op.forward(*xp)
        fm = op.forward(*xm)
        fd = sum(torch.sum((a - b) * l).item() for a, b, l in zip(fp, fm, lam)) / (2 * h)
        # rounding of F(x +- h e_p) near p: ~1e-16 * |local terms| / h
        assert abs(fd - jt[f][p]) <= 1e-7 * (1 + abs(jt[f][p])), (f, p, fd, jt[f][p])
