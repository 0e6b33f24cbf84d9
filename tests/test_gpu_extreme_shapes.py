"""Parity at the edges of the supported sizes.

* An x extent longer than 65535 tiles of the default length (the sweep's CTA
  grid is ceil(ny / ty) x ceil(nx / lx), and a grid's y extent is limited to
  65535, so such an extent is given longer tiles): 4,194,241 x 2 x 32.
* More than 2^31 points (element offsets past the 32-bit range):
  4096 x 4104 x 128 in binary32, 2.15 G points, forward and adjoint.

Inputs are drawn on the device; the oracle evaluates sampled columns (forward)
and 34-plane blocks (adjoint) exactly as in the full-size tests: an output
depends only on inputs within one point of it in x and y, so the interior of
a block cut around a point (periodic in the block) is the grid's own result.
"""
import numpy as np
import pytest
import torch

import oracle
import workload
from gpu_util import make_op

pytestmark = pytest.mark.gpu


def _winds_f32(shape, seed):
    """U(-10, 10) + 2 sin(2 pi i / nx) cos(2 pi j / ny) in binary32, in place."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    nx, ny, _ = shape
    i = torch.arange(nx, device="cuda", dtype=torch.float64)[:, None, None]
    j = torch.arange(ny, device="cuda", dtype=torch.float64)[None, :, None]
    pert = (2.0 * torch.sin(2 * np.pi * i / nx) * torch.cos(2 * np.pi * j / ny)).float()
    out = []
    for _ in range(3):
        a = torch.rand(shape, generator=gen, device="cuda", dtype=torch.float32)
        a.mul_(20).sub_(10).add_(pert)
        out.append(a)
    return out


def _normal_f32(shape, seed):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    return [torch.randn(shape, generator=gen, device="cuda", dtype=torch.float32) for _ in range(3)]


def _column_blocks(fields, cols):
    """(3N, 3, nz) float64: block b is the periodic 3 x 3 neighbourhood of
    column b; the oracle's value at plane 3b+1, row 1 is that column's."""
    out = []
    for t in fields:
        nx, ny, nz = t.shape
        ci = torch.tensor([c[0] for c in cols], device="cuda")
        cj = torch.tensor([c[1] for c in cols], device="cuda")
        off = torch.tensor([-1, 0, 1], device="cuda")
        ii = (ci[:, None] + off[None, :]) % nx
        jj = (cj[:, None] + off[None, :]) % ny
        out.append(t[ii[:, :, None], jj[:, None, :]].to(torch.float64).reshape(-1, 3, nz).cpu().numpy())
    return out


def _check_forward_columns(outs, x, grid, cols, tol):
    ref = oracle.forward(*_column_blocks(x, cols), oracle.coefficients(grid))
    ci = torch.tensor([c[0] for c in cols], device="cuda")
    cj = torch.tensor([c[1] for c in cols], device="cuda")
    for f in range(3):
        g = outs[f][ci, cj].to(torch.float64).cpu().numpy()
        r = ref[f][1::3, 1, :]
        err = np.max(np.abs(g - r)) / np.max(np.abs(r))
        assert err <= tol, f"field {f}: sampled normwise error {err:.3e}"


def _check_adjoint_blocks(got, x, lam, grid, centres, half=17):
    """Blocks of 2*half x-planes and rows (all rows when ny is small) around
    each centre; the interior is compared."""
    c = oracle.coefficients(grid)
    nx, ny, _ = x[0].shape
    for i0, j0 in centres:
        ii = torch.arange(i0 - half, i0 + half, device="cuda") % nx
        full_y = ny <= 2 * half
        jj = torch.arange(ny, device="cuda") if full_y else torch.arange(j0 - half, j0 + half, device="cuda") % ny
        blk = [t[ii[:, None], jj[None, :]].to(torch.float64).cpu().numpy() for t in (*x, *lam)]
        ref = oracle.adjoint(*blk, c)
        jin = jj if full_y else jj[1:-1]
        for g, r, name in zip(got, ref, ("du", "dv", "dw")):
            gi = g[ii[1:-1, None], jin[None, :]].to(torch.float64).cpu().numpy()
            ri = r[1:-1] if full_y else r[1:-1, 1:-1]
            err = float(np.max(np.abs(gi - ri)) / np.max(np.abs(ri)))
            assert err <= 5e-6, f"{name} around ({i0},{j0}): normwise error {err:.3e}"


def test_x_extent_beyond_65535_tiles():
    shape = (65535 * 64 + 1, 2, 32)
    op, grid = make_op(shape, "f32")
    assert op.kernel_name() == "fwd_sweep" and op.kernel_name(True) == "adj_sweep"
    x = _winds_f32(shape, 81)
    outs = op.forward(*x)
    torch.cuda.synchronize()
    nx = shape[0]
    cols = [(i, j) for i in (0, 1, 64 * 65535 - 1, 64 * 65535, nx - 2, nx - 1) for j in (0, 1)]
    rng = np.random.default_rng(82)
    cols += [(int(rng.integers(nx)), int(rng.integers(2))) for _ in range(200)]
    _check_forward_columns(outs, x, grid, cols, 2e-6)
    del outs
    lam = _normal_f32(shape, 83)
    got = op.adjoint(*x, *lam)
    torch.cuda.synchronize()
    _check_adjoint_blocks(got, x, lam, grid, [(0, 0), (nx - 1, 0), (64 * 65535, 0), (2_000_003, 1)])
    op.close()


def test_more_than_2_31_points_forward_and_adjoint():
    """4096 x 4104 x 128 binary32 (2.15 G points).  The adjoint takes the
    winds as its cotangents too (inputs may share memory; only outputs must
    not overlap inputs), which keeps the device footprint to six fields."""
    shape = (4096, 4104, 128)
    assert shape[0] * shape[1] * shape[2] > 2 ** 31
    torch.cuda.empty_cache()
    grid = workload.vertical_grid(shape[2])
    op, _ = make_op(shape, "f32", grid=grid)
    assert op.kernel_name() == "fwd_sweep" and op.kernel_name(True) == "adj_sweep"
    x = _winds_f32(shape, 84)
    outs = op.forward(*x)
    torch.cuda.synchronize()
    # the last planes hold the points whose flat index is past 2^31 - 1
    first_big = (2 ** 31) // (shape[1] * shape[2])
    rng = np.random.default_rng(85)
    cols = [(int(rng.integers(shape[0])), int(rng.integers(shape[1]))) for _ in range(200)]
    cols += [(int(rng.integers(first_big, shape[0])), int(rng.integers(shape[1]))) for _ in range(200)]
    cols += [(i, j) for i in (0, first_big, shape[0] - 1) for j in (0, shape[1] // 2, shape[1] - 1)]
    _check_forward_columns(outs, x, grid, cols, 2e-6)
    got = op.adjoint(*x, *x, out=outs)
    torch.cuda.synchronize()
    _check_adjoint_blocks(got, x, x, grid, [(0, 0), (shape[0] - 1, shape[1] - 1), (first_big + 1, 2049),
                                            (4090, 17)])
    del got, outs, x
    op.close()
    torch.cuda.empty_cache()
