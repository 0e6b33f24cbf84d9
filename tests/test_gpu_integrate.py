"""GPU parity of the fused integration step (out = base + dt * S(u, v, w))
against ``oracle.integrate``, through the C ABI.

Error budget per field: the source-term error of the type's forward path,
scaled by |dt| (tol_s * |dt| * max|S|), plus the rounding of the final add
(tol_out * max|out|).  Levels where the source term is zero must return the
base bit for bit (to the double-float significand for F64_FF).
"""
import numpy as np
import pytest
import torch

import oracle
import workload
from gpu_util import dev, host, make_op, oracle_forward

pytestmark = pytest.mark.gpu

# (tolerance on the dt * S part, tolerance on the result's rounding)
TOL = {"f64": (1e-12, 2.0 ** -51), "f64ff": (1e-12, 1e-13), "f32": (2e-6, 2.0 ** -22)}
TDT = {"f64": torch.float64, "f64ff": torch.float64, "f32": torch.float32}

SHAPES = [(64, 64, 64), (33, 17, 65), (130, 66, 20), (1, 1, 3), (8, 256, 64), (5, 7, 4)]


def _inputs(shape, dtype, seed):
    x = workload.winds(*shape, seed=seed)
    b = workload.winds(*shape, seed=seed + 1000)
    if dtype == "f32":
        x = tuple(a.astype(np.float32).astype(np.float64) for a in x)
        b = tuple(a.astype(np.float32).astype(np.float64) for a in b)
    return x, b


def _check(got, ref, s_ref, dt, dtype, what):
    tol_s, tol_out = TOL[dtype]
    for g, r, s, name in zip(got, ref, s_ref, ("u", "v", "w")):
        bound = tol_s * abs(dt) * np.max(np.abs(s)) + tol_out * np.max(np.abs(r))
        err = np.max(np.abs(g - r))
        assert err <= bound, f"{what} {name}: {err:.3e} > {bound:.3e}"


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64ff"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", ["winds", "base", "in_place"])
def test_integrate_matches_oracle(dtype, shape, mode):
    op, grid = make_op(shape, dtype)
    x, b = _inputs(shape, dtype, seed=51)
    dt = 0.37
    xd = [dev(a, TDT[dtype]) for a in x]
    if mode == "winds":
        out = op.integrate(*xd, dt)
        ref = oracle.integrate(*x, oracle.coefficients(grid), dt)
        base = x
    else:
        bd = [dev(a, TDT[dtype]) for a in b]
        out = op.integrate(*xd, dt, base=bd, out=bd if mode == "in_place" else None)
        if mode == "in_place":
            assert all(o.data_ptr() == t.data_ptr() for o, t in zip(out, bd))
        ref = oracle.integrate(*x, oracle.coefficients(grid), dt, base=b)
        base = b
    torch.cuda.synchronize()
    got = [host(t) for t in out]
    s_ref = oracle_forward(*x, grid)
    _check(got, ref, s_ref, dt, dtype, f"{mode} ({op.kernel_name()})")
    # where the source term is zero the step returns the base: exactly for
    # binary64 and binary32 arithmetic; to the 47-bit significand of a
    # double-float for F64_FF (the base passes through that type)
    eq = np.array_equal if dtype != "f64ff" else (
        lambda a, b: np.max(np.abs(a - b)) <= 2.0 ** -46 * np.max(np.abs(b)))
    assert eq(got[0][..., 0], base[0][..., 0])
    assert eq(got[1][..., 0], base[1][..., 0])
    assert eq(got[2][..., 0], base[2][..., 0])
    assert eq(got[2][..., -1], base[2][..., -1])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_integrate_zero_step_is_the_base_bitwise(dtype):
    shape = (40, 24, 64)
    op, _ = make_op(shape, dtype)
    x, b = _inputs(shape, dtype, seed=52)
    xd = [dev(a, TDT[dtype]) for a in x]
    bd = [dev(a, TDT[dtype]) for a in b]
    for out, base in ((op.integrate(*xd, 0.0), x), (op.integrate(*xd, 0.0, base=bd), b)):
        for o, r in zip(out, base):
            assert np.array_equal(host(o), r)


def test_integrate_agrees_with_forward_then_step():
    """Fused step minus base equals dt times the library's own source terms."""
    shape = (96, 40, 64)
    op, _ = make_op(shape, "f64")
    x, _ = _inputs(shape, "f64", seed=53)
    xd = [dev(a) for a in x]
    s = [host(t) for t in op.forward(*xd)]
    dt = -2.5
    out = [host(t) for t in op.integrate(*xd, dt)]
    for o, a, si in zip(out, x, s):
        d = (o - a) - dt * si
        assert np.max(np.abs(d)) <= 4 * 2.0 ** -53 * np.max(np.abs(o))


def test_integrate_point_kernel_on_unaligned_base():
    """A base 8 but not 16 bytes aligned sends the call to the point kernel;
    results are the same."""
    shape = (32, 16, 64)
    n = shape[0] * shape[1] * shape[2]
    op, grid = make_op(shape, "f64")
    x, b = _inputs(shape, "f64", seed=54)
    xd = [dev(a) for a in x]
    bufs = [torch.empty(n + 1, dtype=torch.float64, device="cuda") for _ in range(3)]
    bd = []
    for buf, a in zip(bufs, b):
        view = buf[1:].view(shape)
        view.copy_(dev(a))
        bd.append(view)
    assert bd[0].data_ptr() % 16 == 8
    dt = 0.61
    out = op.integrate(*xd, dt, base=bd)
    ref = oracle.integrate(*x, oracle.coefficients(grid), dt, base=b)
    _check([host(t) for t in out], ref, oracle_forward(*x, grid), dt, "f64", "unaligned base")


@pytest.mark.parametrize("with_base", [False, True])
def test_integrate_f16s(with_base):
    shape = (64, 64, 64)
    op, grid = make_op(shape, "f16s")
    winds = workload.winds(*shape, seed=55)
    base = workload.winds(*shape, seed=56)
    dt = 0.25
    s_in = [float(2.0 ** np.ceil(np.log2(np.max(np.abs(a))))) for a in winds]
    s_src = op.output_scales(s_in)
    h = [torch.from_numpy(a / s).to(torch.float16) for a, s in zip(winds, s_in)]
    deq = [t.to(torch.float64).numpy() * s for t, s in zip(h, s_in)]
    scales = list(s_in)
    if with_base:
        s_b = [float(2.0 ** np.ceil(np.log2(np.max(np.abs(a))))) for a in base]
        hb = [torch.from_numpy(a / s).to(torch.float16) for a, s in zip(base, s_b)]
        deq_b = [t.to(torch.float64).numpy() * s for t, s in zip(hb, s_b)]
        s_out = [float(2.0 ** np.ceil(np.log2(sb + dt * ss))) for sb, ss in zip(s_b, s_src)]
        out = op.integrate(*(t.cuda() for t in h), dt, base=[t.cuda() for t in hb],
                           scales=scales + s_out + s_b)
        ref = oracle.integrate(*deq, oracle.coefficients(grid), dt, base=deq_b)
    else:
        s_out = [float(2.0 ** np.ceil(np.log2(si + dt * ss))) for si, ss in zip(s_in, s_src)]
        out = op.integrate(*(t.cuda() for t in h), dt, scales=scales + s_out)
        ref = oracle.integrate(*deq, oracle.coefficients(grid), dt)
    s_ref = oracle_forward(*deq, grid)
    for t, r, s, so in zip(out, ref, s_ref, s_out):
        g = host(t) * so
        assert np.max(np.abs(r)) <= so
        bound = 2.0 ** -11 * so + 2e-6 * dt * np.max(np.abs(s))
        assert np.max(np.abs(g - r)) <= bound


def test_integrate_validation():
    from paper_2010_01545_gb300 import AdvectError, _abi
    shape = (8, 8, 8)
    op, _ = make_op(shape, "f64")
    u, v, w = (dev(a) for a in workload.winds(*shape, seed=57))
    b = [torch.zeros_like(u) for _ in range(3)]
    o = [torch.empty_like(u) for _ in range(3)]
    p = lambda ts: [t.data_ptr() for t in ts]

    def call(bases, outs, dt=0.5, scales=None):
        with pytest.raises(AdvectError) as e:
            _abi.advect_forward_integrate(op.handle, u.data_ptr(), v.data_ptr(), w.data_ptr(), *bases,
                                          dt, *outs, scales)
        return e.value

    assert call([None] * 3, [u.data_ptr()] + p(o[1:])).status == 1           # output is an input
    assert call([b[0].data_ptr(), None, None], p(o)).status == 1              # one base of three
    assert call(p(b), p(o), dt=float("inf")).status == 1                      # dt not finite
    e = call([b[0].data_ptr(), o[0].data_ptr(), b[2].data_ptr()], p(o))       # base is another output
    assert e.status == 1 and "overlaps" in str(e)
    e = call([b[0].data_ptr() + 8, b[1].data_ptr(), b[2].data_ptr()], [b[0].data_ptr()] + p(o[1:]))
    assert e.status == 1 and "overlaps" in str(e)                             # partial overlap
    # base == its own output is accepted (in place)
    _abi.advect_forward_integrate(op.handle, u.data_ptr(), v.data_ptr(), w.data_ptr(), *p(b), 0.5,
                                  *p(b), None)
    torch.cuda.synchronize()
    op16, _ = make_op(shape, "f16s")
    h = [t.to(torch.float16) for t in (u, v, w)]
    with pytest.raises(AdvectError):
        _abi.advect_forward_integrate(op16.handle, *p(h), None, None, None, 0.5,
                                      *p([torch.empty_like(h[0]) for _ in range(3)]), None)


@pytest.mark.parametrize("f64_levels", [2, 64])
def test_integrate_f32_with_binary64_near_surface_levels(f64_levels):
    shape = (40, 24, 64)
    op, grid = make_op(shape, "f32", f64_levels=f64_levels)
    x, b = _inputs(shape, "f32", seed=58)
    dt = 0.37
    bd = [dev(a, torch.float32) for a in b]
    out = op.integrate(*(dev(a, torch.float32) for a in x), dt, base=bd, out=bd)
    ref = oracle.integrate(*x, oracle.coefficients(grid), dt, base=b)
    _check([host(t) for t in out], ref, oracle_forward(*x, grid), dt, "f32", f"f64_levels={f64_levels}")


def test_in_place_step_is_applied_once_with_tuning_armed(tmp_path, monkeypatch):
    """The tuner times candidates by repeating a call; an in-place step must
    never be repeated, so the integration call leaves tuning to the next
    plain forward."""
    monkeypatch.setenv("ADVECT_TUNE_CACHE", str(tmp_path / "tune.json"))
    shape = (64, 48, 64)
    op, grid = make_op(shape, "f32")
    op.autotune(True)
    x, b = _inputs(shape, "f32", seed=59)
    dt = 0.5
    xd = [dev(a, torch.float32) for a in x]
    bd = [dev(a, torch.float32) for a in b]
    op.integrate(*xd, dt, base=bd, out=bd)
    ref = oracle.integrate(*x, oracle.coefficients(grid), dt, base=b)
    s_ref = oracle_forward(*x, grid)
    _check([host(t) for t in bd], ref, s_ref, dt, "f32", "in place with tuning armed")
    # the next forward tunes and is still correct
    su = op.forward(*xd)
    for g, r in zip(su, s_ref):
        assert np.max(np.abs(host(g) - r)) <= 2e-6 * np.max(np.abs(r))
    assert (tmp_path / "tune.json").exists()
