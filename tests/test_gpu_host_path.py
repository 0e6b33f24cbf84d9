"""The host-buffer call (advect_forward_host): chunks of x-planes copied in,
computed and copied out on three streams.  Each chunk runs the same kernel
as the device call on its plane range, so the results are bitwise the
device path's -- for ragged chunks (nx not a multiple of the chunk count),
one-plane chunks, a single chunk, and shapes that take the point kernel."""
import numpy as np
import pytest
import torch

import workload
from gpu_util import dev, make_op

pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32, "f64ff": torch.float64}


def _pinned(arrays, dtype):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dtype).pin_memory() for a in arrays]


@pytest.mark.parametrize("chunks", [None, "1", "7"])
@pytest.mark.parametrize("shape", [(37, 24, 64), (1, 8, 64), (5, 7, 3), (64, 16, 32)])
@pytest.mark.parametrize("dtype", ["f64", "f32", "f64ff"])
def test_host_path_is_bitwise_the_device_path(dtype, shape, chunks, monkeypatch):
    if chunks is not None:
        monkeypatch.setenv("ADVECT_HOST_CHUNKS", chunks)  # read when the context is created
    op, _ = make_op(shape, dtype)
    winds = workload.winds(*shape, seed=91)
    dref = [t.cpu() for t in op.forward(*(dev(a, TDT[dtype]) for a in winds))]
    hin = _pinned(winds, TDT[dtype])
    hout = [torch.full(shape, float("nan"), dtype=TDT[dtype]).pin_memory() for _ in range(3)]
    op.forward_host(*hin, hout)
    for a, b in zip(hout, dref):
        assert torch.equal(a, b)
    op.close()


def test_host_path_f16s_is_bitwise_the_device_path():
    shape = (45, 16, 64)
    op, _ = make_op(shape, "f16s")
    winds = workload.winds(*shape, seed=92)
    s_in = [float(2.0 ** np.ceil(np.log2(np.max(np.abs(a))))) for a in winds]
    scales = s_in + op.output_scales(s_in)
    h = [torch.from_numpy(a / s).to(torch.float16) for a, s in zip(winds, s_in)]
    dref = [t.cpu() for t in op.forward(*(t.cuda() for t in h), scales=scales)]
    hout = [torch.empty(shape, dtype=torch.float16).pin_memory() for _ in range(3)]
    op.forward_host(*(t.pin_memory() for t in h), hout, scales=scales)
    for a, b in zip(hout, dref):
        assert torch.equal(a, b)
    op.close()


def test_host_path_from_pageable_memory():
    """Pageable (not pinned) host buffers are valid too, only slower."""
    shape = (33, 20, 64)
    op, _ = make_op(shape, "f64")
    winds = workload.winds(*shape, seed=93)
    dref = [t.cpu() for t in op.forward(*(dev(a) for a in winds))]
    hin = [torch.from_numpy(np.ascontiguousarray(a)) for a in winds]
    hout = [torch.empty(shape, dtype=torch.float64) for _ in range(3)]
    op.forward_host(*hin, hout)
    for a, b in zip(hout, dref):
        assert torch.equal(a, b)
    op.close()
