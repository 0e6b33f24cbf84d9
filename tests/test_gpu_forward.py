"""GPU parity of the forward pass against the FP64 oracle (through the C ABI).

F64: every element within 1e-12 of the oracle, normwise per field
(max |gpu - oracle| <= 1e-12 * max |oracle|); levels the method does not
compute must be exactly zero.  F32 and F16S are compared with the oracle run
on the same rounded inputs, so the bounds measure the kernel's arithmetic and
output rounding only.
"""
import numpy as np
import pytest
import torch

import workload
from gpu_util import dev, host, make_op, normwise, oracle_forward

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12
# binary32: ~10 roundings of terms up to a few times max|s| -> a few 1e-7
TOL_F32 = 2e-6

SHAPES = [
    (64, 64, 64),      # the 262k-point FP64 case
    (33, 17, 65),      # several tiles with ragged edges in every direction
    (130, 66, 20),
    (5, 7, 3),         # minimum nz
    (1, 1, 3),         # a single periodic column: i+-1, j+-1 wrap onto itself
    (1, 9, 8),
    (9, 1, 8),
    (2, 2, 5),
    (8, 256, 64),
    (3, 5, 127),       # odd nz (the tiled paths need nz * element size % 16 == 0)
]


def run_f64(shape, seed=1545):
    op, grid = make_op(shape, "f64")
    u, v, w = workload.winds(*shape, seed=seed)
    su, sv, sw = op.forward(dev(u), dev(v), dev(w))
    torch.cuda.synchronize()
    return op, (u, v, w), (host(su), host(sv), host(sw)), oracle_forward(u, v, w, grid)


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_f64_matches_oracle(shape):
    op, _, got, ref = run_f64(shape)
    for g, r, name in zip(got, ref, ("su", "sv", "sw")):
        err = normwise(g, r)
        assert err <= TOL_F64, f"{name} normwise error {err:.3e} ({op.kernel_name()})"
    su, sv, sw = got
    assert not su[..., 0].any() and not sv[..., 0].any()
    assert not sw[..., 0].any() and not sw[..., -1].any()


def test_forward_f64_zero_tendency_and_impulse_on_gpu():
    shape = (6, 5, 7)
    op, grid = make_op(shape, "f64")
    u = np.full(shape, 4.25)
    z = np.zeros(shape)
    out = op.forward(dev(u), dev(z), dev(z))
    for t in out:
        assert not host(t).any()
    u = np.zeros(shape)
    u[2, 3, 4] = 1.0
    su, sv, sw = (host(t) for t in op.forward(dev(u), dev(z), dev(z)))
    tcx = op.coeffs[0]
    exp = np.zeros(shape)
    exp[3, 3, 4], exp[1, 3, 4] = tcx, -tcx
    np.testing.assert_allclose(su, exp, rtol=1e-15, atol=1e-300)
    assert not sv.any() and not sw.any()


def test_forward_is_deterministic():
    shape = (40, 24, 64)
    op, _ = make_op(shape, "f64")
    u, v, w = (dev(a) for a in workload.winds(*shape, seed=3))
    a = [host(t) for t in op.forward(u, v, w)]
    b = [host(t) for t in op.forward(u, v, w)]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("shape", [(64, 64, 64), (33, 17, 65), (1, 1, 3), (130, 66, 20)])
@pytest.mark.parametrize("f64_levels", [0, 2, 64])
def test_forward_f32_matches_oracle_on_rounded_inputs(shape, f64_levels):
    op, grid = make_op(shape, "f32", f64_levels=f64_levels)
    u, v, w = (a.astype(np.float32).astype(np.float64) for a in workload.winds(*shape, seed=5))
    su, sv, sw = op.forward(*(dev(a, torch.float32) for a in (u, v, w)))
    ref = oracle_forward(u, v, w, grid)
    for g, r, name in zip((host(su), host(sv), host(sw)), ref, ("su", "sv", "sw")):
        err = normwise(g, r)
        assert err <= TOL_F32, f"{name} normwise error {err:.3e}"


@pytest.mark.parametrize("shape", [(64, 64, 64), (33, 17, 64), (1, 1, 8), (130, 66, 24)])
def test_forward_f16s_matches_oracle_on_quantised_inputs(shape):
    op, grid = make_op(shape, "f16s")
    winds = workload.winds(*shape, seed=6)
    s_in = [float(2.0 ** np.ceil(np.log2(np.max(np.abs(a))))) for a in winds]
    s_out = op.output_scales(s_in)
    h = [torch.from_numpy(a / s).to(torch.float16) for a, s in zip(winds, s_in)]
    deq = [x.to(torch.float64).numpy() * s for x, s in zip(h, s_in)]
    out = op.forward(*(x.cuda() for x in h), scales=s_in + s_out)
    ref = oracle_forward(*deq, grid)
    for t, r, so, name in zip(out, ref, s_out, ("su", "sv", "sw")):
        g = host(t) * so
        assert np.max(np.abs(r)) <= so, f"{name}: a priori bound violated"
        # half an fp16 ulp of the stored value plus binary32 arithmetic
        bound = 2.0 ** -11 * so + TOL_F32 * np.max(np.abs(r))
        assert np.max(np.abs(g - r)) <= bound, f"{name}: {np.max(np.abs(g - r)):.3e} > {bound:.3e}"


def test_forward_host_path_matches_device_path():
    shape = (96, 40, 64)
    op, grid = make_op(shape, "f64")
    winds = workload.winds(*shape, seed=8)
    dref = [host(t) for t in op.forward(*(dev(a) for a in winds))]
    hin = [torch.from_numpy(a).pin_memory() for a in winds]
    hout = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(3)]
    op.forward_host(*hin, hout)
    for a, b in zip(hout, dref):
        assert np.array_equal(a.numpy(), b)


def test_forward_rejects_aliasing_and_wrong_device_memory():
    from paper_2010_01545_gb300 import AdvectError, _abi
    shape = (8, 8, 8)
    op, _ = make_op(shape, "f64")
    u, v, w = (dev(a) for a in workload.winds(*shape, seed=9))
    with pytest.raises(AdvectError) as e:
        _abi.advect_forward(op.handle, u.data_ptr(), v.data_ptr(), w.data_ptr(), u.data_ptr(),
                            v.data_ptr(), w.data_ptr())
    assert e.value.status == 1 and "overlaps" in str(e.value)
    h = torch.zeros(shape, dtype=torch.float64)
    out = [torch.empty_like(u) for _ in range(3)]
    with pytest.raises(AdvectError) as e:
        _abi.advect_forward(op.handle, h.data_ptr(), v.data_ptr(), w.data_ptr(),
                            *(t.data_ptr() for t in out))
    assert e.value.status == 1
    with pytest.raises(AdvectError) as e:
        _abi.advect_forward(op.handle, u.data_ptr() + 4, v.data_ptr(), w.data_ptr(),
                            *(t.data_ptr() for t in out))
    assert "aligned" in str(e.value)


def test_forward_f16s_rejects_scales_that_are_not_powers_of_two():
    from paper_2010_01545_gb300 import AdvectError
    shape = (8, 8, 8)
    op, _ = make_op(shape, "f16s")
    h = [torch.zeros(shape, dtype=torch.float16, device="cuda") for _ in range(3)]
    good = [16.0, 16.0, 8.0] + op.output_scales([16.0, 16.0, 8.0])
    op.forward(*h, scales=good)
    for q, bad in ((0, 12.0), (2, 0.3), (5, 48.0)):
        s = list(good)
        s[q] = bad
        with pytest.raises(AdvectError) as e:
            op.forward(*h, scales=s)
        assert e.value.status == 1 and "power of two" in str(e.value)
