"""The allocation-free forward entry point, advect_forward_noalloc.

It serves callers that may not allocate device memory (a framework that owns
all device memory through its own pool, latency-critical loops, programs
with a fixed device footprint): it needs no context and keeps its
coefficient tables and error flag in a fixed array inside the library.  This
test calls it through the C ABI several times in a row, with every element
type and different shapes (so each call must overwrite what the previous one
left in the shared array), and checks each result two ways: bit for bit
against the context entry point advect_forward on the same inputs (the same
kernels run), and against the FP64 oracle within the tolerances of the
parity tests.  The file name sorts last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import workload
from gpu_util import ensure_built, host, lib_coeffs, make_op, normwise, oracle_forward
from paper_2010_01545_gb300 import _abi

pytestmark = pytest.mark.gpu

TOL_F32 = 2e-6
CODES = {"f64": (_abi.ADVECT_F64, torch.float64), "f32": (_abi.ADVECT_F32, torch.float32),
         "f16s": (_abi.ADVECT_F16S, torch.float16), "f64ff": (_abi.ADVECT_F64_FF, torch.float64)}
# (shape, type): sweep-sized and ragged shapes, then the first call again
CALLS = [((48, 40, 64), "f64"), ((33, 17, 32), "f32"), ((40, 24, 64), "f16s"), ((70, 42, 64), "f64ff"),
         ((9, 5, 7), "f64ff"), ((48, 40, 64), "f64")]


def _inputs(shape, dtype, seed):
    """Device inputs, the values the oracle sees (rounded or quantised to the
    storage type) and the F16S scales."""
    winds = workload.winds(*shape, seed=seed)
    if dtype == "f16s":
        s_in = [float(2.0 ** np.ceil(np.log2(np.max(np.abs(a))))) for a in winds]
        h = [torch.from_numpy(a / s).to(torch.float16) for a, s in zip(winds, s_in)]
        seen = [t.to(torch.float64).numpy() * s for t, s in zip(h, s_in)]
        return [t.cuda() for t in h], seen, s_in
    tdt = CODES[dtype][1]
    x = [torch.from_numpy(a).to("cuda", tdt) for a in winds]
    return x, [host(t) for t in x], None


def test_noalloc_forward_matches_context_path_and_oracle_on_consecutive_calls():
    ensure_built()
    stream = torch.cuda.current_stream().cuda_stream
    for n, (shape, dtype) in enumerate(CALLS):
        code, tdt = CODES[dtype]
        grid = workload.vertical_grid(shape[2])
        coeffs = lib_coeffs(grid)
        op, _ = make_op(shape, dtype, grid=grid)
        x, seen, s_in = _inputs(shape, dtype, 900 + n)
        scales = s_in + op.output_scales(s_in) if s_in else None
        out = [torch.full(shape, float("nan"), dtype=tdt, device="cuda") for _ in range(3)]
        _abi.advect_forward_noalloc(*shape, coeffs, code, *(t.data_ptr() for t in x),
                                    *(t.data_ptr() for t in out), scales, stream)
        ref = op.forward(*x, scales=scales)
        torch.cuda.synchronize()
        for g, r in zip(out, ref):
            assert torch.equal(g, r), f"call {n} ({dtype} {shape}) differs from advect_forward"
        oref = oracle_forward(*seen, grid)
        for f, (g, r) in enumerate(zip(out, oref)):
            gh = host(g)
            assert np.all(np.isfinite(gh))
            if dtype == "f16s":
                so = scales[3 + f]
                bound = 2.0 ** -11 * so + TOL_F32 * np.max(np.abs(r))
                assert np.max(np.abs(gh * so - r)) <= bound, f"call {n} field {f}"
            else:
                tol = TOL_F32 if dtype == "f32" else 1e-12
                err = normwise(gh, r)
                assert err <= tol, f"call {n} ({dtype}) field {f}: normwise error {err:.3e}"
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
