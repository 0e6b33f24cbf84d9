"""The plane-sweep kernel under many tile shapes (ADVECT_SWEEP override):
ragged y blocks, x ranges that do not divide nx, one plane per CTA, the
minimum ring depth, and grids smaller than one tile."""
import numpy as np
import pytest
import torch

import workload
from gpu_util import dev, host, make_op, normwise, oracle_forward

pytestmark = pytest.mark.gpu

CASES = {
    "f64": [(8, 64, 4), (4, 7, 5), (1, 1, 4), (2, 300, 6), (8, 2048, 12)],
    "f32": [(16, 64, 8), (2, 5, 4), (6, 33, 7), (16, 1, 4)],
    "f16s": [(16, 64, 7), (4, 3, 4), (12, 9, 5), (32, 1, 4), (8, 64, 6, 4)],
}
# the last shape's rows straddle warps in every sweep (levels per row not a
# divisor of 32: 48, 24 and 12 threads)
SHAPES = [(37, 45, 64), (3, 2, 64), (64, 64, 64), (5, 130, 64), (11, 21, 96)]
TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("shape", SHAPES)
def test_sweep_configs_match_oracle(monkeypatch, dtype, shape):
    winds = workload.winds(*shape, seed=77)
    for cfg in CASES[dtype]:
        monkeypatch.setenv("ADVECT_SWEEP", ",".join(map(str, cfg)))
        op, grid = make_op(shape, dtype)
        assert op.kernel_name() == "fwd_sweep"
        if dtype == "f16s":
            s_in = [float(2.0 ** np.ceil(np.log2(np.max(np.abs(a))))) for a in winds]
            s_out = op.output_scales(s_in)
            h = [torch.from_numpy(a / s).to(torch.float16) for a, s in zip(winds, s_in)]
            deq = [x.to(torch.float64).numpy() * s for x, s in zip(h, s_in)]
            out = op.forward(*(x.cuda() for x in h), scales=s_in + s_out)
            ref = oracle_forward(*deq, grid)
            for t, r, so in zip(out, ref, s_out):
                err = np.max(np.abs(host(t) * so - r))
                assert err <= 2.0 ** -11 * so + 2e-6 * np.max(np.abs(r)), (cfg, err)
        else:
            tdt = torch.float64 if dtype == "f64" else torch.float32
            inp = winds if dtype == "f64" else [a.astype(np.float32).astype(np.float64) for a in winds]
            out = op.forward(*(dev(a, tdt) for a in inp))
            ref = oracle_forward(*inp, grid)
            for t, r in zip(out, ref):
                assert normwise(host(t), r) <= TOL[dtype], cfg
        op.close()


def test_sweep_is_selected_for_aligned_columns():
    for shape, dtype in [((16, 16, 64), "f64"), ((16, 16, 32), "f32"), ((16, 16, 128), "f16s"),
                         ((16, 16, 20), "f64")]:
        op, _ = make_op(shape, dtype)
        assert op.kernel_name() == "fwd_sweep", (shape, dtype)
    for shape, dtype in [((16, 16, 65), "f64"), ((16, 16, 6), "f32"), ((16, 16, 12), "f16s")]:
        op, _ = make_op(shape, dtype)
        assert op.kernel_name() == "fwd_point", (shape, dtype)


ADJ_CASES = {"f64": [(4, 64, 8), (1, 5, 4), (2, 33, 6), (2, 1, 5, 3)],
             "f32": [(4, 64, 6, 4), (1, 7, 4), (8, 300, 5), (2, 2, 6, 3)]}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(37, 45, 64), (3, 2, 64), (9, 70, 32)])
def test_adjoint_sweep_configs_match_oracle(monkeypatch, dtype, shape):
    from gpu_util import oracle_adjoint
    x = workload.winds(*shape, seed=78)
    lam = workload.cotangents(*shape, seed=79)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        x = [a.astype(np.float32).astype(np.float64) for a in x]
        lam = [a.astype(np.float32).astype(np.float64) for a in lam]
    for cfg in ADJ_CASES[dtype]:
        monkeypatch.setenv("ADVECT_ADJ_SWEEP", ",".join(map(str, cfg)))
        op, grid = make_op(shape, dtype)
        assert op.kernel_name(True) == "adj_sweep", cfg
        got = op.adjoint(*(dev(a, tdt) for a in (*x, *lam)))
        ref = oracle_adjoint(*x, *lam, grid)
        for g, r in zip(got, ref):
            assert normwise(host(g), r) <= (1e-12 if dtype == "f64" else 5e-6), cfg
        op.close()
