"""The allocation-free forward entry point, advect_forward_noalloc.

It serves callers that may not allocate device memory (a framework that owns
all device memory through its own pool, latency-critical loops, programs
with a fixed device footprint): it needs no context and keeps its
coefficient tables and error flag in a fixed array inside the library.  This
test calls it through the C ABI, twice in a row with different shapes and
element types (so the second call must overwrite what the first left in the
shared array), and compares each result with the context entry point
advect_forward on the same inputs, within the tolerances of the parity tests.
The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

import workload
from gpu_util import dev, ensure_built, host, lib_coeffs, make_op, normwise
from paper_2010_01545_gb300 import _abi

pytestmark = pytest.mark.gpu

CALLS = [((48, 40, 64), "f64", 1e-12), ((33, 17, 32), "f32", 2e-6)]
CODES = {"f64": (_abi.ADVECT_F64, torch.float64), "f32": (_abi.ADVECT_F32, torch.float32)}


def test_noalloc_forward_matches_the_context_entry_point_on_two_calls():
    ensure_built()
    stream = torch.cuda.current_stream().cuda_stream
    for n, (shape, dtype, tol) in enumerate(CALLS):
        code, tdt = CODES[dtype]
        grid = workload.vertical_grid(shape[2])
        coeffs = lib_coeffs(grid)
        x = [dev(a, tdt) for a in workload.winds(*shape, seed=900 + n)]
        out = [torch.full(shape, float("nan"), dtype=tdt, device="cuda") for _ in range(3)]
        _abi.advect_forward_noalloc(*shape, coeffs, code, *(t.data_ptr() for t in x),
                                    *(t.data_ptr() for t in out), None, stream)
        op, _ = make_op(shape, dtype, grid=grid)
        ref = op.forward(*x)
        torch.cuda.synchronize()
        for g, r in zip(out, ref):
            g, r = host(g), host(r)
            assert np.all(np.isfinite(g))
            assert normwise(g, r) <= tol
        op.close()


def test_noalloc_rejects_columns_above_its_limit():
    ensure_built()
    nz = _abi.NOALLOC_MAX_NZ + 2
    shape = (2, 2, nz)
    z = 10.0 * np.arange(nz)
    coeffs = lib_coeffs(workload.custom_grid(z, z - 5.0, np.ones(nz), np.ones(nz), 50.0, 50.0))
    t = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(6)]
    with pytest.raises(_abi.AdvectError) as e:
        _abi.advect_forward_noalloc(*shape, coeffs, _abi.ADVECT_F64, *(a.data_ptr() for a in t))
    assert e.value.status == 1 and "no-allocation limit" in str(e.value)
