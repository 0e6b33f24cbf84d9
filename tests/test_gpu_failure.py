"""Failure detection on the GPU without a GPU fault.

Each wait in the sweep kernels is bounded.  With the test-only injection
(ADVECT_TEST_SKIP_PLANE, read when a context is created) the kernels never
issue the copy of one plane of each tile, so the waits on it run out after a
short budget (ADVECT_TEST_WAIT_CYCLES, ~1 ms here): every CTA then stops,
waits for the copies it did issue and returns, the device flag is raised, and
advect_sync reports ADVECT_ETIMEOUT.  The device must stay usable: a context
created afterwards computes correct results.
"""
import pytest
import torch

import workload
from gpu_util import dev, host, make_op, normwise, oracle_adjoint, oracle_forward
from paper_2010_01545_gb300 import AdvectError

pytestmark = pytest.mark.gpu


# (dtype, shape): binary64, binary32 and the double-float sweeps (forward with
# its converter warp, adjoint with the split spread over all warps; 128 levels
# for the adjoint whose rows span two warps)
CASES = [("f64", (20, 24, 64)), ("f32", (20, 24, 64)), ("f64ff", (20, 24, 64)), ("f64ff", (20, 12, 128))]


@pytest.mark.parametrize("dtype,shape", CASES)
def test_bounded_wait_times_out_and_reports(monkeypatch, dtype, shape):
    tdt = torch.float32 if dtype == "f32" else torch.float64
    monkeypatch.setenv("ADVECT_TEST_SKIP_PLANE", "3")
    monkeypatch.setenv("ADVECT_TEST_WAIT_CYCLES", "2000000")
    bad, grid = make_op(shape, dtype)
    assert bad.kernel_name() == "fwd_sweep" and bad.kernel_name(True) == "adj_sweep"
    x = [dev(a, tdt) for a in workload.winds(*shape, seed=5)]
    lam = [dev(a, tdt) for a in workload.cotangents(*shape, seed=6)]
    bad.forward(*x)
    with pytest.raises(AdvectError) as e:
        bad.sync()
    assert e.value.status == 5 and "bounded wait" in str(e.value)
    bad.sync()                      # the flag was cleared by the report
    bad.adjoint(*x, *lam)
    with pytest.raises(AdvectError) as e:
        bad.sync()
    assert e.value.status == 5
    bad.close()

    monkeypatch.delenv("ADVECT_TEST_SKIP_PLANE")
    monkeypatch.delenv("ADVECT_TEST_WAIT_CYCLES")
    good, grid = make_op(shape, dtype)
    xs = workload.winds(*shape, seed=5)
    if dtype == "f32":
        xs = [a.astype("float32").astype("float64") for a in xs]
    out = good.forward(*(dev(a, tdt) for a in xs))
    good.sync()
    for g, r in zip(out, oracle_forward(*xs, grid)):
        assert normwise(host(g), r) <= (2e-6 if dtype == "f32" else 1e-12)
