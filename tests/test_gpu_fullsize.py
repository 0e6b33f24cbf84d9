"""Parity at the benchmark's full sizes, in the same launch configuration.

Inputs are drawn on the device (seeded torch generators, the benchmark's
distributions) so that no multi-gigabyte host arrays are made: heavy host
memory churn leaves the host's pinned copies stalling for minutes
afterwards, which would disturb a host-buffer benchmark run after the
tests.  The oracle evaluates sampled columns exactly: each column's 3 x 3 x nz
neighbourhood (periodic) is gathered from the device, the neighbourhoods are
stacked along x in blocks of three planes, and one oracle call returns every
column's values in the middle plane and row of its block (the middle of a
block sees only its own block).  The 1024 x 1024 x 128 adjoint is checked by
properties that hold at any size (dot-product identity, central differences
at 64 probes) and against the oracle on 34 x 34 x 128 periodic blocks.
"""
import numpy as np
import pytest
import torch

import oracle
import workload
from gpu_util import host, make_op

pytestmark = pytest.mark.gpu

BIG = (2048, 2048, 64)


def device_winds(shape, seed, dtype=torch.float64):
    """u, v, w ~ U(-10, 10) + 2 sin(2 pi i / nx) cos(2 pi j / ny), on the device."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    nx, ny, _ = shape
    i = torch.arange(nx, device="cuda", dtype=torch.float64)[:, None, None]
    j = torch.arange(ny, device="cuda", dtype=torch.float64)[None, :, None]
    pert = 2.0 * torch.sin(2 * np.pi * i / nx) * torch.cos(2 * np.pi * j / ny)
    out = []
    for _ in range(3):
        a = torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64) * 20 - 10
        a += pert
        out.append(a.to(dtype))
    return out


def device_normal(shape, seed, n=3, dtype=torch.float64):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    return [torch.randn(shape, generator=gen, device="cuda", dtype=torch.float64).to(dtype) for _ in range(n)]


def fsum_dot(a_list, b_list):
    """sum_f <a_f, b_f> in binary64: per-plane partial sums on the device,
    then a correctly rounded sum of the partials (math.fsum)."""
    import math
    parts = []
    for a, b in zip(a_list, b_list):
        parts.extend(torch.sum(a.to(torch.float64) * b.to(torch.float64), dim=(1, 2)).tolist())
    return math.fsum(parts)


def sample_columns(shape, n_random, seed):
    """Random columns plus every boundary class of the periodic grid."""
    nx, ny, _ = shape
    rng = np.random.default_rng(seed)
    cols = [(int(rng.integers(nx)), int(rng.integers(ny))) for _ in range(n_random)]
    cols += [(i, j) for i in (0, 1, nx - 1) for j in (0, ny // 2, ny - 1)]
    return cols


def column_blocks(fields, cols, scale=None):
    """(3N, 3, nz) float64 host arrays, block b (x-planes 3b..3b+2) the
    periodic 3 x 3 neighbourhood of column b; the oracle's result in plane
    3b+1, row 1 is that column's."""
    out = []
    for f, t in enumerate(fields):
        nx, ny, nz = t.shape
        ci = torch.tensor([c[0] for c in cols], device="cuda")
        cj = torch.tensor([c[1] for c in cols], device="cuda")
        off = torch.tensor([-1, 0, 1], device="cuda")
        ii = (ci[:, None] + off[None, :]) % nx
        jj = (cj[:, None] + off[None, :]) % ny
        blk = t[ii[:, :, None], jj[:, None, :]].to(torch.float64)  # (N, 3, 3, nz)
        if scale is not None:
            blk = blk * scale[f]
        out.append(blk.reshape(-1, 3, nz).cpu().numpy())
    return out


def column_values(t, cols):
    ci = torch.tensor([c[0] for c in cols], device="cuda")
    cj = torch.tensor([c[1] for c in cols], device="cuda")
    return t[ci, cj].to(torch.float64).cpu().numpy()  # (N, nz)


def middles(a):
    return a[1::3, 1, :]


def _check_forward(outs, inputs, grid, cols, tol):
    ref = oracle.forward(*column_blocks(inputs, cols), oracle.coefficients(grid))
    for f in range(3):
        g = column_values(outs[f], cols)
        r = middles(ref[f])
        err = np.max(np.abs(g - r)) / np.max(np.abs(r))
        assert err <= tol, f"field {f}: sampled normwise error {err:.3e}"


def test_forward_f64_2048x2048x64_sampled():
    op, grid = make_op(BIG, "f64")
    assert op.kernel_name() == "fwd_sweep"
    x = device_winds(BIG, workload.DEFAULT_SEED)
    outs = op.forward(*x)
    torch.cuda.synchronize()
    _check_forward(outs, x, grid, sample_columns(BIG, 400, 1), 1e-12)


@pytest.mark.parametrize("shape", [(512, 512, 64), (1024, 1024, 64)])
def test_forward_f64_sweep_sizes_sampled(shape):
    """The smaller grids of the very-large-grid sweep."""
    op, grid = make_op(shape, "f64")
    x = device_winds(shape, workload.DEFAULT_SEED + 11)
    outs = op.forward(*x)
    torch.cuda.synchronize()
    _check_forward(outs, x, grid, sample_columns(shape, 400, 9), 1e-12)


def test_forward_f32_2048x2048x64_sampled():
    op, grid = make_op(BIG, "f32")
    x = device_winds(BIG, workload.DEFAULT_SEED, torch.float32)
    outs = op.forward(*x)
    torch.cuda.synchronize()
    _check_forward(outs, x, grid, sample_columns(BIG, 400, 2), 2e-6)


def test_forward_f64ff_2048x2048x64_sampled():
    op, grid = make_op(BIG, "f64ff")
    x = device_winds(BIG, workload.DEFAULT_SEED + 1)
    outs = op.forward(*x)
    torch.cuda.synchronize()
    _check_forward(outs, x, grid, sample_columns(BIG, 400, 4), 1e-12)


def test_forward_f16s_2048x2048x64_sampled():
    op, grid = make_op(BIG, "f16s")
    x = device_winds(BIG, workload.DEFAULT_SEED + 2)
    s_in = [float(2.0 ** np.ceil(np.log2(torch.max(torch.abs(a)).item()))) for a in x]
    s_out = op.output_scales(s_in)
    h = [(a / s).to(torch.float16) for a, s in zip(x, s_in)]
    del x
    outs = op.forward(*h, scales=s_in + s_out)
    torch.cuda.synchronize()
    cols = sample_columns(BIG, 400, 5)
    ref = oracle.forward(*column_blocks(h, cols, s_in), oracle.coefficients(grid))
    for f in range(3):
        g = column_values(outs[f], cols) * s_out[f]
        r = middles(ref[f])
        bound = 2.0 ** -11 * s_out[f] + 2e-6 * np.max(np.abs(r))
        assert np.max(np.abs(g - r)) <= bound, f"field {f}"


def test_integrate_f64_2048x2048x64_in_place_sampled():
    """The fused step, in place on a separate base, at the benchmark size."""
    op, grid = make_op(BIG, "f64")
    x = device_winds(BIG, workload.DEFAULT_SEED)
    b = device_winds(BIG, workload.DEFAULT_SEED + 7)
    cols = sample_columns(BIG, 400, 3)
    bblk = column_blocks(b, cols)
    dt = 0.37
    out = op.integrate(*x, dt, base=b, out=b)
    torch.cuda.synchronize()
    c = oracle.coefficients(grid)
    xblk = column_blocks(x, cols)
    ref = oracle.integrate(*xblk, c, dt, base=bblk)
    s = oracle.forward(*xblk, c)
    for f in range(3):
        g = column_values(out[f], cols)
        r = middles(ref[f])
        bound = 1e-12 * dt * np.max(np.abs(middles(s[f]))) + 2.0 ** -51 * np.max(np.abs(r))
        assert np.max(np.abs(g - r)) <= bound, f"field {f}"


def test_integrate_f32_2048x2048x64_in_place_sampled():
    """The binary32 step as the benchmark runs it: a separate base (a copy of
    the winds) updated in place, dt = 0.5."""
    op, grid = make_op(BIG, "f32")
    x = device_winds(BIG, workload.DEFAULT_SEED + 8, torch.float32)
    b = [t.clone() for t in x]
    cols = sample_columns(BIG, 400, 6)
    bblk = column_blocks(b, cols)
    dt = 0.5
    op.integrate(*x, dt, base=b, out=b)
    torch.cuda.synchronize()
    c = oracle.coefficients(grid)
    xblk = column_blocks(x, cols)
    ref = oracle.integrate(*xblk, c, dt, base=bblk)
    s = oracle.forward(*xblk, c)
    for f in range(3):
        g = column_values(b[f], cols)
        r = middles(ref[f])
        bound = 2e-6 * dt * np.max(np.abs(middles(s[f]))) + 2.0 ** -22 * np.max(np.abs(r))
        assert np.max(np.abs(g - r)) <= bound, f"field {f}"


def _adjoint_blocks(op, grid, x, lam, got, tol):
    """The adjoint against the FP64 oracle adjoint on 34 x 34 x nz blocks cut
    (periodically) around chosen points, seams included; an output depends
    only on inputs within one point in x and y, so each block's interior
    32 x 32 columns are the grid's own."""
    shape = tuple(x[0].shape)
    c = oracle.coefficients(grid)
    for i0, j0 in ((0, 0), (shape[0] - 1, shape[1] // 2), (shape[0] // 2, shape[1] - 1), (257, 33)):
        ii = torch.arange(i0 - 17, i0 + 17, device="cuda") % shape[0]
        jj = torch.arange(j0 - 17, j0 + 17, device="cuda") % shape[1]
        blk = [t[ii[:, None], jj[None, :]].to(torch.float64).cpu().numpy() for t in (*x, *lam)]
        ref = oracle.adjoint(*blk, c)
        for g, r, name in zip(got, ref, ("du", "dv", "dw")):
            gi = g[ii[1:-1, None], jj[None, 1:-1]].to(torch.float64).cpu().numpy()
            ri = r[1:-1, 1:-1]
            err = float(np.max(np.abs(gi - ri)) / np.max(np.abs(ri)))
            assert err <= tol, f"{name} at ({i0},{j0}): normwise error {err:.3e} ({op.kernel_name(True)})"


@pytest.mark.parametrize("dtype", ["f64", "f64ff"])
def test_adjoint_binary64_1024x1024x128_against_oracle_on_blocks(dtype):
    """The binary64-storage adjoints at the differentiation workload's size,
    in the benchmark's launch configuration, within the 1e-12 bar."""
    shape = (1024, 1024, 128)
    op, grid = make_op(shape, dtype)
    x = device_winds(shape, 47)
    lam = device_normal(shape, 48)
    got = op.adjoint(*x, *lam)
    torch.cuda.synchronize()
    _adjoint_blocks(op, grid, x, lam, got, 1e-12)


def test_adjoint_f64_1024x1024x128_dot_product_and_probes():
    shape = (1024, 1024, 128)
    op, _ = make_op(shape, "f64")
    x = device_winds(shape, 41)
    d = device_normal(shape, 42)
    lam = device_normal(shape, 43)
    # the map is quadratic: J d = (F(x + d) - F(x - d)) / 2 exactly, with a
    # full-scale direction so that only the rounding of the two forwards
    # (relative ~1e-16) separates the two sides
    fp = op.forward(*(a + b for a, b in zip(x, d)))
    fm = op.forward(*(a - b for a, b in zip(x, d)))
    jd = [(a - b) * 0.5 for a, b in zip(fp, fm)]
    del fp, fm
    jt = op.adjoint(*x, *lam)
    lhs = fsum_dot(jd, lam)
    rhs = fsum_dot(d, jt)
    mag = fsum_dot([a.abs() for a in d], [b.abs() for b in jt])
    assert abs(lhs - rhs) <= 1e-12 * mag, (lhs, rhs, mag)
    del jd, d
    rng = np.random.default_rng(44)
    eps = 1e-6
    out_p = op.forward(*x)
    for _ in range(64):
        f = int(rng.integers(3))
        p = tuple(int(rng.integers(n)) for n in shape)
        keep = x[f][p].item()
        x[f][p] = keep + eps
        op.forward(*x, out=out_p)
        # only the 3x3x3 neighbourhood of p changes
        sl = tuple(slice(max(c - 1, 0), c + 2) for c in p)
        plus = [o[sl].clone() for o in out_p]
        x[f][p] = keep - eps
        op.forward(*x, out=out_p)
        minus = [o[sl].clone() for o in out_p]
        x[f][p] = keep
        fd = sum(torch.sum((a - b) * l[sl]).item() for a, b, l in zip(plus, minus, lam)) / (2 * eps)
        # probes away from the periodic seams see their whole neighbourhood
        if all(0 < c < n - 1 for c, n in zip(p[:2], shape[:2])):
            jt_p = jt[f][p].item()
            assert abs(fd - jt_p) <= 1e-7 * (1 + abs(jt_p)), (f, p, fd, jt_p)


def test_adjoint_f32_1024x1024x128_against_oracle_on_blocks():
    """The binary32 adjoint at the differentiation workload's size, in the
    launch configuration the benchmark uses, against the FP64 oracle adjoint
    on the same binary32 inputs, on 34 x 34 x 128 blocks cut (periodically)
    around chosen points -- including the seams of the periodic domain --
    whose interior 32 x 32 columns see their whole neighbourhood."""
    shape = (1024, 1024, 128)
    op, grid = make_op(shape, "f32")
    x = device_winds(shape, 45, torch.float32)
    lam = device_normal(shape, 46, dtype=torch.float32)
    got = op.adjoint(*x, *lam)
    torch.cuda.synchronize()
    c = oracle.coefficients(grid)
    for i0, j0 in ((0, 0), (1023, 511), (500, 1023), (257, 33)):
        ii = torch.arange(i0 - 17, i0 + 17, device="cuda") % shape[0]
        jj = torch.arange(j0 - 17, j0 + 17, device="cuda") % shape[1]
        blk = [t[ii[:, None], jj[None, :]].to(torch.float64).cpu().numpy() for t in (*x, *lam)]
        ref = oracle.adjoint(*blk, c)
        for g, r, name in zip(got, ref, ("du", "dv", "dw")):
            gi = g[ii[1:-1, None], jj[None, 1:-1]].to(torch.float64).cpu().numpy()
            ri = r[1:-1, 1:-1]
            err = float(np.max(np.abs(gi - ri)) / np.max(np.abs(ri)))
            assert err <= 5e-6, f"{name} at ({i0},{j0}): normwise error {err:.3e} ({op.kernel_name(True)})"


def test_ensemble_48_members_as_benchmarked():
    """The 48-member FP32 ensemble of the benchmark (autotuned, one persistent
    launch per direction): every member's forward against the oracle on
    sampled columns, every member's adjoint bitwise against the single-grid
    adjoint, and the three smallest members' adjoints fully against the
    oracle."""
    from gpu_util import ensure_built, lib_coeffs, oracle_adjoint
    from paper_2010_01545_gb300 import torch_api
    ensure_built()
    shapes = workload.ensemble_shapes(48)
    grids = [workload.vertical_grid(s[2]) for s in shapes]
    coeffs = [lib_coeffs(g) for g in grids]
    ens = torch_api.AdvectEnsemble(shapes, coeffs, "f32")
    ens.autotune(True)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(workload.DEFAULT_SEED)
    x = [[torch.rand(s, generator=gen, device="cuda") * 20 - 10 for s in shapes] for _ in range(3)]
    lam = [[torch.randn(s, generator=gen, device="cuda") for s in shapes] for _ in range(3)]
    y = ens.forward(*x)
    g = ens.adjoint(*x, *lam)
    torch.cuda.synchronize()
    for m, s in enumerate(shapes):
        cols = sample_columns(s, 60, 7 + m)
        ref = oracle.forward(*column_blocks([f[m] for f in x], cols), oracle.coefficients(grids[m]))
        for f in range(3):
            got = column_values(y[f][m], cols)
            r = middles(ref[f])
            err = np.max(np.abs(got - r)) / max(np.max(np.abs(r)), 1e-30)
            assert err <= 2e-6, (m, s, f, err)
        op = torch_api.Advect(*s, coeffs[m], "f32")
        single = op.adjoint(*(f[m] for f in x), *(f[m] for f in lam))
        for f in range(3):
            assert torch.equal(g[f][m], single[f]), (m, s, f)
        op.close()
    for m in sorted(range(len(shapes)), key=lambda q: np.prod(shapes[q]))[:3]:
        xm = [f[m].to(torch.float64).cpu().numpy() for f in x]
        lm = [f[m].to(torch.float64).cpu().numpy() for f in lam]
        ref = oracle_adjoint(*xm, *lm, grids[m])
        for f in range(3):
            got = host(g[f][m])
            err = np.max(np.abs(got - ref[f])) / np.max(np.abs(ref[f]))
            assert err <= 5e-6, (m, f, err)
