"""The FP64-accurate double-float mode (ADVECT_F64_FF): binary64 in memory,
pairs of binary32 on the binary32 pipes.  It must meet the FP64 parity bar
against the oracle (normwise 1e-12 per field) for the forward and the
adjoint, on the sweep and the point kernels, and over a wide dynamic range."""
import numpy as np
import pytest

import workload
from gpu_util import dev, host, make_op, normwise, oracle_adjoint, oracle_forward

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 64), (33, 17, 65), (130, 66, 20), (5, 7, 3), (1, 1, 4), (16, 32, 128), (23, 19, 32), (9, 40, 16),
          (7, 33, 8), (6, 10, 256)]


def _grid(shape):
    """The benchmark's vertical grid, gentler stretching for deep columns
    (with 256 levels at the 1.05 ratio the top density underflows)."""
    nz = shape[2]
    return workload.vertical_grid(nz) if nz <= 128 else workload.vertical_grid(nz, ratio=1.01)


@pytest.mark.parametrize("shape", SHAPES)
def test_ff_forward_meets_the_fp64_bar(shape):
    op, grid = make_op(shape, "f64ff", grid=_grid(shape))
    x = workload.winds(*shape, seed=41)
    out = op.forward(*(dev(a) for a in x))
    ref = oracle_forward(*x, grid)
    for g, r, name in zip(out, ref, ("su", "sv", "sw")):
        err = normwise(host(g), r)
        assert err <= 1e-12, f"{name} {err:.2e} ({op.kernel_name()})"


@pytest.mark.parametrize("shape", SHAPES)
def test_ff_adjoint_meets_the_fp64_bar(shape):
    op, grid = make_op(shape, "f64ff", grid=_grid(shape))
    x = workload.winds(*shape, seed=42)
    lam = workload.cotangents(*shape, seed=43)
    g = op.adjoint(*(dev(a) for a in (*x, *lam)))
    ref = oracle_adjoint(*x, *lam, grid)
    for t, r, name in zip(g, ref, ("du", "dv", "dw")):
        err = normwise(host(t), r)
        assert err <= 1e-12, f"{name} {err:.2e} ({op.kernel_name(True)})"


def test_ff_wide_dynamic_range():
    """Fields scaled by factors from 1e-6 to 1e6 across x-planes."""
    shape = (40, 24, 64)
    op, grid = make_op(shape, "f64ff")
    scale = 10.0 ** np.linspace(-6, 6, shape[0])[:, None, None]
    x = [a * scale for a in workload.winds(*shape, seed=44)]
    out = op.forward(*(dev(a) for a in x))
    ref = oracle_forward(*x, grid)
    for g, r in zip(out, ref):
        assert normwise(host(g), r) <= 1e-12
    # plane by plane the relative error stays small where the planes are small
    su = host(out[0])
    for i in (0, 5, 20):
        m = np.max(np.abs(ref[0][i]))
        assert np.max(np.abs(su[i] - ref[0][i])) <= 1e-11 * m


def test_ff_sweep_configs(monkeypatch):
    shape = (37, 45, 64)
    x = workload.winds(*shape, seed=45)
    # the converter-warp sweep at 1, 2 (default, 7 rows), 3 and 4 CTAs per SM
    for cfg in [(4, 64, 7, 3), (2, 5, 4, 1), (4, 300, 6, 1), (4, 64, 5, 4), (7, 9, 4, 2), (3, 64, 8, 2)]:
        monkeypatch.setenv("ADVECT_SWEEP", ",".join(map(str, cfg)))
        op, grid = make_op(shape, "f64ff")
        assert op.kernel_name() == "fwd_sweep"
        assert op.tuned_config() == "ty=%d,lx=%d,nb=%d,occ=%d" % cfg, (cfg, op.tuned_config())
        out = op.forward(*(dev(a) for a in x))
        for g, r in zip(out, oracle_forward(*x, grid)):
            assert normwise(host(g), r) <= 1e-12, cfg


@pytest.mark.parametrize("shape,cfgs", [
    # 128 levels: a row's level pairs span two warps
    ((37, 45, 128), [(6, 64, 4), (2, 5, 4), (3, 300, 5), (1, 7, 4)]),
    # 64 and 16 levels: rows within a warp (one, and four rows per warp)
    ((21, 30, 64), [(12, 64, 5), (1, 3, 4), (5, 8, 6)]),
    ((19, 50, 16), [(48, 64, 4), (4, 2, 4)]),
])
def test_ff_adjoint_sweep_configs(monkeypatch, shape, cfgs):
    """The double-float adjoint's own sweep over tile shapes: ragged rows
    (ny not a multiple of ty), tiles of a few planes, shallow and deep rings."""
    x = workload.winds(*shape, seed=46)
    lam = workload.cotangents(*shape, seed=47)
    for cfg in cfgs:
        monkeypatch.setenv("ADVECT_ADJ_SWEEP", ",".join(map(str, cfg)))
        op, grid = make_op(shape, "f64ff")
        assert op.kernel_name(True) == "adj_sweep"
        assert op.tuned_config(True).startswith("ty=%d,lx=%d,nb=%d," % cfg), (cfg, op.tuned_config(True))
        out = op.adjoint(*(dev(a) for a in x), *(dev(a) for a in lam))
        for g, r in zip(out, oracle_adjoint(*x, *lam, grid)):
            assert normwise(host(g), r) <= 1e-12, cfg
