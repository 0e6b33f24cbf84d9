"""Autotuning of single grids.  After advect_autotune the next forward and
adjoint calls time the point kernel, the context's current tile and every
candidate tile on the call's own buffers, keep the fastest (cached per shape,
type and SM count) and finish the call with it.  The tuned calls must still
meet the parity bars against the oracle, and a new context for the same shape
must read the cached choices and reproduce the tuned results bit for bit."""
import numpy as np
import pytest
import torch

import workload
from gpu_util import dev, host, make_op, normwise, oracle_adjoint, oracle_forward

pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32, "f64ff": torch.float64}
BAR = {"f64": (1e-12, 1e-12), "f64ff": (1e-12, 1e-12), "f32": (2e-6, 5e-6)}


def _inputs(shape, dtype):
    x = workload.winds(*shape, seed=71)
    lam = workload.cotangents(*shape, seed=72)
    if dtype == "f32":  # the oracle runs on the values the GPU reads
        x = [a.astype(np.float32).astype(np.float64) for a in x]
        lam = [a.astype(np.float32).astype(np.float64) for a in lam]
    return x, lam


# the double-float sweeps (converter-warp forward; the adjoint's own sweep,
# rows of two warps at 128 levels) and the binary32 adjoint's 4-level sweep
@pytest.mark.parametrize("dtype,shape", [("f64ff", (40, 36, 64)), ("f64ff", (24, 20, 128)),
                                         ("f32", (40, 36, 128)), ("f64", (30, 26, 64))])
def test_tuned_calls_meet_the_bar_and_are_cached(tmp_path, monkeypatch, dtype, shape):
    monkeypatch.setenv("ADVECT_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.delenv("ADVECT_SWEEP", raising=False)
    monkeypatch.delenv("ADVECT_ADJ_SWEEP", raising=False)
    tdt = TDT[dtype]
    x, lam = _inputs(shape, dtype)
    xd = [dev(a, tdt) for a in x]
    ld = [dev(a, tdt) for a in lam]
    fwd_bar, adj_bar = BAR[dtype]

    op, grid = make_op(shape, dtype)
    op.autotune(True)
    out = [host(t) for t in op.forward(*xd)]
    grads = [host(t) for t in op.adjoint(*xd, *ld)]
    for g, r in zip(out, oracle_forward(*x, grid)):
        assert normwise(g, r) <= fwd_bar, op.tuned_config()
    for g, r in zip(grads, oracle_adjoint(*x, *lam, grid)):
        assert normwise(g, r) <= adj_bar, op.tuned_config(True)
    cfg_f, cfg_a = op.tuned_config(), op.tuned_config(True)
    assert (tmp_path / "tune.json").exists()
    op.close()

    # a new context reads the cached choices; same kernels and tiles, so the
    # same results bit for bit
    op2, _ = make_op(shape, dtype)
    assert op2.tuned_config() == cfg_f and op2.tuned_config(True) == cfg_a
    out2 = [host(t) for t in op2.forward(*xd)]
    grads2 = [host(t) for t in op2.adjoint(*xd, *ld)]
    for a, b in zip(out, out2):
        assert np.array_equal(a, b)
    for a, b in zip(grads, grads2):
        assert np.array_equal(a, b)
    op2.close()
