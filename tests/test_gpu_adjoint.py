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
          (16, 32, 128)]


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


@pytest.mark.parametrize("shape", [(64, 64, 64), (33, 17, 65), (1, 1, 4)])
def test_adjoint_f32_matches_oracle_on_rounded_inputs(shape):
    op, grid = make_op(shape, "f32")
    x = [a.astype(np.float32).astype(np.float64) for a in workload.winds(*shape, seed=23)]
    lam = [a.astype(np.float32).astype(np.float64) for a in workload.cotangents(*shape, seed=24)]
    got = [host(t) for t in op.adjoint(*(dev(a, torch.float32) for a in (*x, *lam)))]
    ref = oracle_adjoint(*x, *lam, grid)
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


def test_dot_product_identity_on_gpu():
    shape = (32, 24, 64)
    op, _ = make_op(shape, "f64")
    x = [dev(a) for a in workload.winds(*shape, seed=28)]
    d = [dev(a) for a in workload.cotangents(*shape, seed=29)]
    lam = [dev(a) for a in workload.cotangents(*shape, seed=30)]
    h = 2.0 ** -10
    fp = op.forward(*(a + h * b for a, b in zip(x, d)))
    fm = op.forward(*(a - h * b for a, b in zip(x, d)))
    jd = [(a - b) / (2 * h) for a, b in zip(fp, fm)]
    jt = op.adjoint(*x, *lam)
    lhs = sum(torch.sum(a * b).item() for a, b in zip(jd, lam))
    rhs = sum(torch.sum(a * b).item() for a, b in zip(d, jt))
    mag = sum(torch.sum(torch.abs(a * b)).item() for a, b in zip(d, jt))
    assert abs(lhs - rhs) <= 1e-12 * mag * 1e3


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
