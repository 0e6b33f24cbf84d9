"""The x-slab decomposition run with the library's kernels: the grid's
sub-domains held on one device (ranks emulated in one process, each slab its
own context and launch; no kernel waits on another), halos filled from the
neighbouring slabs, and the owned planes compared with the full-grid call."""
import pytest
import torch

import workload
from gpu_util import dev, make_op
from paper_2010_01545_gb300 import decomp

pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32, "f64ff": torch.float64}


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64ff"])
@pytest.mark.parametrize("world", [2, 3, 7])
def test_decomposed_forward_is_bitwise_the_full_grid(dtype, world):
    shape = (45, 24, 64)
    op, grid = make_op(shape, dtype)
    fields = [dev(a, TDT[dtype]) for a in workload.winds(*shape, seed=95)]
    full = op.forward(*fields)
    bounds = [decomp.slab_bounds(shape[0], world, r) for r in range(world)]
    slabs = [[decomp.padded_slab(f, i0, i1) for f in fields] for i0, i1 in bounds]
    decomp.fill_x_halos_local(slabs)
    for (i0, i1), sl in zip(bounds, slabs):
        sub, _ = make_op((i1 - i0 + 2,) + shape[1:], dtype, grid=grid)
        out = sub.forward(*sl)
        for o, r in zip(out, full):
            assert torch.equal(o[1:-1], r[i0:i1])
        sub.close()
    op.close()


def test_decomposed_adjoint_is_bitwise_the_full_grid():
    """The adjoint reads the cotangents at +-1 too, so they are exchanged
    like the winds; the owned planes of each slab's gradient are the full
    grid's."""
    shape = (40, 16, 64)
    op, grid = make_op(shape, "f32")
    fields = [dev(a, torch.float32) for a in workload.winds(*shape, seed=96)]
    lam = [dev(a, torch.float32) for a in workload.cotangents(*shape, seed=97)]
    full = op.adjoint(*fields, *lam)
    world = 4
    bounds = [decomp.slab_bounds(shape[0], world, r) for r in range(world)]
    slabs = [[decomp.padded_slab(f, i0, i1) for f in (*fields, *lam)] for i0, i1 in bounds]
    decomp.fill_x_halos_local(slabs)
    for (i0, i1), sl in zip(bounds, slabs):
        sub, _ = make_op((i1 - i0 + 2,) + shape[1:], "f32", grid=grid)
        out = sub.adjoint(*sl)
        for o, r in zip(out, full):
            assert torch.equal(o[1:-1], r[i0:i1])
        sub.close()
    op.close()
