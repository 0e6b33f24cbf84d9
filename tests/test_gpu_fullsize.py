"""Parity at the benchmark's full sizes, in the same launch configuration.

The 2048 x 2048 x 64 forward (268M points) runs through the same context
creation as bench.py; the oracle evaluates a sample of points one by one
(every boundary class plus random interior points).  The 1024 x 1024 x 128
adjoint is checked by properties that hold at any size: the dot-product
identity and central differences at 64 random probes.
"""
import numpy as np
import pytest
import torch

import oracle
import workload
from gpu_util import dev, host, make_op

pytestmark = pytest.mark.gpu


def sample_indices(shape, n_random, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    pts = [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(n_random)]
    for i in (0, 1, nx - 1):
        for j in (0, ny - 1, ny // 2):
            for k in (0, 1, 2, nz - 2, nz - 1):
                pts.append((i, j, k))
    return np.array([(i * ny + j) * nz + k for i, j, k in pts], dtype=np.int64)


@pytest.fixture(scope="module")
def big_winds():
    return workload.winds(2048, 2048, 64, seed=workload.DEFAULT_SEED)


def _check_sample(outs, winds, grid, shape, tol, seed):
    idx = sample_indices(shape, 20000, seed)
    ref = oracle.forward_points(*winds, oracle.coefficients(grid), idx)
    for f in range(3):
        g = outs[f].reshape(-1)[torch.from_numpy(idx).cuda()].to(torch.float64).cpu().numpy()
        r = ref[:, f]
        err = np.max(np.abs(g - r)) / np.max(np.abs(r))
        assert err <= tol, f"field {f}: sampled normwise error {err:.3e}"


def test_forward_f64_2048x2048x64_sampled(big_winds):
    shape = (2048, 2048, 64)
    op, grid = make_op(shape, "f64")
    assert op.kernel_name() == "fwd_sweep"
    outs = op.forward(*(dev(a) for a in big_winds))
    torch.cuda.synchronize()
    _check_sample(outs, big_winds, grid, shape, 1e-12, 1)
    del outs
    torch.cuda.empty_cache()


def test_forward_f32_2048x2048x64_sampled(big_winds):
    shape = (2048, 2048, 64)
    op, grid = make_op(shape, "f32")
    w32 = [a.astype(np.float32) for a in big_winds]
    outs = op.forward(*(torch.from_numpy(a).cuda() for a in w32))
    torch.cuda.synchronize()
    _check_sample(outs, [a.astype(np.float64) for a in w32], grid, shape, 2e-6, 2)
    del outs
    torch.cuda.empty_cache()


def test_forward_f64ff_2048x2048x64_sampled(big_winds):
    shape = (2048, 2048, 64)
    op, grid = make_op(shape, "f64ff")
    outs = op.forward(*(dev(a) for a in big_winds))
    torch.cuda.synchronize()
    _check_sample(outs, big_winds, grid, shape, 1e-12, 4)
    del outs
    torch.cuda.empty_cache()


def test_forward_f16s_2048x2048x64_sampled(big_winds):
    shape = (2048, 2048, 64)
    op, grid = make_op(shape, "f16s")
    s_in = [float(2.0 ** np.ceil(np.log2(np.max(np.abs(a))))) for a in big_winds]
    s_out = op.output_scales(s_in)
    h = [(torch.from_numpy(a).cuda() / s).to(torch.float16) for a, s in zip(big_winds, s_in)]
    deq = [t.to(torch.float64).cpu().numpy() * s for t, s in zip(h, s_in)]
    outs = op.forward(*h, scales=s_in + s_out)
    torch.cuda.synchronize()
    idx = sample_indices(shape, 20000, 5)
    ref = oracle.forward_points(*deq, oracle.coefficients(grid), idx)
    for f in range(3):
        g = outs[f].reshape(-1)[torch.from_numpy(idx).cuda()].to(torch.float64).cpu().numpy() * s_out[f]
        r = ref[:, f]
        bound = 2.0 ** -11 * s_out[f] + 2e-6 * np.max(np.abs(r))
        assert np.max(np.abs(g - r)) <= bound, f"field {f}"
    del outs, h, deq
    torch.cuda.empty_cache()


def test_integrate_f64_2048x2048x64_in_place_sampled(big_winds):
    """The fused step, in place on a separate base, at the benchmark size."""
    shape = (2048, 2048, 64)
    op, grid = make_op(shape, "f64")
    base = workload.winds(*shape, seed=workload.DEFAULT_SEED + 7)
    dt = 0.37
    x = [dev(a) for a in big_winds]
    b = [dev(a) for a in base]
    out = op.integrate(*x, dt, base=b, out=b)
    torch.cuda.synchronize()
    idx = sample_indices(shape, 20000, 3)
    s = oracle.forward_points(*big_winds, oracle.coefficients(grid), idx)
    for f in range(3):
        g = out[f].reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
        r = base[f].reshape(-1)[idx] + dt * s[:, f]
        bound = 1e-12 * dt * np.max(np.abs(s[:, f])) + 2.0 ** -51 * np.max(np.abs(r))
        assert np.max(np.abs(g - r)) <= bound, f"field {f}"
    del x, b, out
    torch.cuda.empty_cache()


def test_adjoint_f64_1024x1024x128_dot_product_and_probes():
    shape = (1024, 1024, 128)
    op, _ = make_op(shape, "f64")
    x = [dev(a) for a in workload.winds(*shape, seed=41)]
    d = [dev(a) for a in workload.cotangents(*shape, seed=42)]
    lam = [dev(a) for a in workload.cotangents(*shape, seed=43)]
    h = 2.0 ** -10
    fp = op.forward(*(a + h * b for a, b in zip(x, d)))
    fm = op.forward(*(a - h * b for a, b in zip(x, d)))
    jd = [(a - b) / (2 * h) for a, b in zip(fp, fm)]
    del fp, fm
    jt = op.adjoint(*x, *lam)
    lhs = sum(torch.sum(a * b).item() for a, b in zip(jd, lam))
    rhs = sum(torch.sum(a * b).item() for a, b in zip(d, jt))
    mag = sum(torch.sum(torch.abs(a * b)).item() for a, b in zip(d, jt))
    assert abs(lhs - rhs) <= 1e-10 * mag
    del jd, d
    jt_h = [host(t) for t in jt]
    rng = np.random.default_rng(44)
    eps = 1e-6
    out_p = op.forward(*x)
    for _ in range(64):
        f = int(rng.integers(3))
        p = tuple(int(rng.integers(n)) for n in shape)
        keep = x[f][p].item()
        x[f][p] = keep + eps
        op.forward(*x, out=out_p)
        # only the 3x3x3 neighbourhood of p changes
        sl = tuple(slice(max(c - 1, 0), c + 2) for c in p)
        plus = [o[sl].clone() for o in out_p]
        x[f][p] = keep - eps
        op.forward(*x, out=out_p)
        minus = [o[sl].clone() for o in out_p]
        x[f][p] = keep
        fd = sum(torch.sum((a - b) * l[sl]).item() for a, b, l in zip(plus, minus, lam)) / (2 * eps)
        # probes away from the periodic seams see their whole neighbourhood
        if all(0 < c < n - 1 for c, n in zip(p[:2], shape[:2])):
            assert abs(fd - jt_h[f][p]) <= 1e-7 * (1 + abs(jt_h[f][p])), (f, p, fd, jt_h[f][p])


def test_adjoint_f32_1024x1024x128_against_oracle_on_blocks():
    """The binary32 adjoint at the differentiation workload's size, in the
    launch configuration the benchmark uses, against the FP64 oracle adjoint
    on the same binary32-rounded inputs.  The oracle runs on 34 x 34 x 128
    blocks cut (periodically) around chosen points -- including the seams of
    the periodic domain -- and its interior 32 x 32 columns, which see their
    whole neighbourhood, are compared (keeps the host memory small)."""
    shape = (1024, 1024, 128)
    op, grid = make_op(shape, "f32")
    x = [a.astype(np.float32) for a in workload.winds(*shape, seed=45)]
    lam = [a.astype(np.float32) for a in workload.cotangents(*shape, seed=46)]
    got = [host(t) for t in op.adjoint(*(torch.from_numpy(a).cuda() for a in (*x, *lam)))]
    c = oracle.coefficients(grid)
    for i0, j0 in ((0, 0), (1023, 511), (500, 1023), (257, 33)):
        ii = np.arange(i0 - 17, i0 + 17) % shape[0]
        jj = np.arange(j0 - 17, j0 + 17) % shape[1]
        blk = [a[np.ix_(ii, jj)].astype(np.float64) for a in (*x, *lam)]
        ref = oracle.adjoint(*blk, c)
        for g, r, name in zip(got, ref, ("du", "dv", "dw")):
            gi = g[np.ix_(ii[1:-1], jj[1:-1])]
            ri = r[1:-1, 1:-1]
            err = float(np.max(np.abs(gi - ri)) / np.max(np.abs(ri)))
            assert err <= 5e-6, f"{name} at ({i0},{j0}): normwise error {err:.3e} ({op.kernel_name(True)})"


def test_ensemble_48_members_as_benchmarked():
    """The 48-member FP32 ensemble of the benchmark (autotuned, one persistent
    launch per direction): every member's forward against the oracle on
    sampled points, every member's adjoint bitwise against the single-grid
    adjoint, and the three smallest members' adjoints fully against the
    oracle."""
    from gpu_util import ensure_built, lib_coeffs, oracle_adjoint
    from paper_2010_01545_gb300 import torch_api
    ensure_built()
    shapes = workload.ensemble_shapes(48)
    grids = [workload.vertical_grid(s[2]) for s in shapes]
    coeffs = [lib_coeffs(g) for g in grids]
    ens = torch_api.AdvectEnsemble(shapes, coeffs, "f32")
    ens.autotune(True)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(workload.DEFAULT_SEED)
    x = [[torch.rand(s, generator=gen, device="cuda") * 20 - 10 for s in shapes] for _ in range(3)]
    lam = [[torch.randn(s, generator=gen, device="cuda") for s in shapes] for _ in range(3)]
    y = ens.forward(*x)
    g = ens.adjoint(*x, *lam)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for m, s in enumerate(shapes):
        xm = [f[m].to(torch.float64).cpu().numpy() for f in x]
        n = s[0] * s[1] * s[2]
        idx = np.unique(np.concatenate([rng.integers(0, n, 1500), np.arange(s[2]), n - 1 - np.arange(s[2])]))
        ref = oracle.forward_points(*xm, oracle.coefficients(grids[m]), idx)
        for f in range(3):
            got = y[f][m].reshape(-1)[torch.from_numpy(idx).cuda()].to(torch.float64).cpu().numpy()
            err = np.max(np.abs(got - ref[:, f])) / max(np.max(np.abs(ref[:, f])), 1e-30)
            assert err <= 2e-6, (m, s, f, err)
        op = torch_api.Advect(*s, coeffs[m], "f32")
        single = op.adjoint(*(f[m] for f in x), *(f[m] for f in lam))
        for f in range(3):
            assert torch.equal(g[f][m], single[f]), (m, s, f)
        op.close()
    for m in sorted(range(len(shapes)), key=lambda q: np.prod(shapes[q]))[:3]:
        xm = [f[m].to(torch.float64).cpu().numpy() for f in x]
        lm = [f[m].to(torch.float64).cpu().numpy() for f in lam]
        ref = oracle_adjoint(*xm, *lm, grids[m])
        for f in range(3):
            got = g[f][m].to(torch.float64).cpu().numpy()
            err = np.max(np.abs(got - ref[f])) / np.max(np.abs(ref[f]))
            assert err <= 5e-6, (m, f, err)
