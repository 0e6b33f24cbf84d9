"""GPU parity of the ensemble (persistent multi-grid launch) and of the
autotuner, against the oracle and the single-grid path."""
import os

import numpy as np
import pytest
import torch

import workload
from gpu_util import dev, ensure_built, host, lib_coeffs, make_op, normwise, oracle_adjoint, oracle_forward
from paper_2010_01545_gb300 import AdvectError, torch_api

pytestmark = pytest.mark.gpu

SHAPES = [(96, 128, 64), (33, 47, 32), (8, 5, 128), (130, 64, 64), (1, 3, 32), (64, 96, 128), (17, 9, 64)]


def build_members(shapes, dtype, seed=100):
    ensure_built()
    grids = [workload.vertical_grid(s[2]) for s in shapes]
    coeffs = [lib_coeffs(g) for g in grids]
    ens = torch_api.AdvectEnsemble(shapes, coeffs, dtype)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    x = [workload.winds(*s, seed=seed + m) for m, s in enumerate(shapes)]
    lam = [workload.cotangents(*s, seed=seed + 50 + m) for m, s in enumerate(shapes)]
    if dtype == "f32":
        x = [[a.astype(np.float32).astype(np.float64) for a in xm] for xm in x]
        lam = [[a.astype(np.float32).astype(np.float64) for a in lm] for lm in lam]
    dx = [[dev(a, tdt) for a in xm] for xm in x]
    dl = [[dev(a, tdt) for a in lm] for lm in lam]
    return ens, grids, x, lam, dx, dl


def fields(per_member, f):
    return [pm[f] for pm in per_member]


@pytest.mark.parametrize("dtype,tol,atol", [("f64", 1e-12, 1e-12), ("f32", 2e-6, 5e-6)])
def test_ensemble_forward_and_adjoint_match_oracle(dtype, tol, atol):
    ens, grids, x, lam, dx, dl = build_members(SHAPES, dtype)
    assert ens.kernel_name() == "ens_fwd"
    out = ens.forward(*(fields(dx, f) for f in range(3)))
    grads = ens.adjoint(*(fields(dx, f) for f in range(3)), *(fields(dl, f) for f in range(3)))
    for m, s in enumerate(SHAPES):
        ref = oracle_forward(*x[m], grids[m])
        for f in range(3):
            assert normwise(host(out[f][m]), ref[f]) <= tol, (m, s, f)
        refg = oracle_adjoint(*x[m], *lam[m], grids[m])
        for f in range(3):
            assert normwise(host(grads[f][m]), refg[f]) <= atol, (m, s, f)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ensemble_equals_single_grid_path_bitwise(dtype):
    ens, grids, x, lam, dx, dl = build_members(SHAPES[:4], dtype, seed=300)
    out = ens.forward(*(fields(dx, f) for f in range(3)))
    for m, s in enumerate(SHAPES[:4]):
        op, _ = make_op(s, dtype, grid=grids[m])
        ref = op.forward(*dx[m])
        for f in range(3):
            assert torch.equal(out[f][m], ref[f]), (m, f)


def test_ensemble_graph_replay_and_new_pointers():
    ens, grids, x, lam, dx, dl = build_members(SHAPES[:5], "f32", seed=400)
    a = [[t.clone() for t in o] for o in ens.forward(*(fields(dx, f) for f in range(3)))]
    outs = [ens.empty() for _ in range(3)]
    for _ in range(3):   # replays of the captured graph with the same pointers
        ens.forward(*(fields(dx, f) for f in range(3)), out=outs)
    for f in range(3):
        for m in range(5):
            assert torch.equal(outs[f][m], a[f][m])
    outs2 = [ens.empty() for _ in range(3)]   # new output pointers: table re-uploaded
    ens.forward(*(fields(dx, f) for f in range(3)), out=outs2)
    for f in range(3):
        for m in range(5):
            assert torch.equal(outs2[f][m], a[f][m])


def test_ensemble_rejects_bad_member_buffers():
    ens, grids, x, lam, dx, dl = build_members(SHAPES[:3], "f32", seed=500)
    u, v, w = (fields(dx, f) for f in range(3))
    out = [ens.empty() for _ in range(3)]
    with pytest.raises(AdvectError) as e:   # an output aliases an input
        ens.forward(u, v, w, out=[[u[0]] + out[0][1:], out[1], out[2]])
    assert e.value.status == 1
    with pytest.raises(ValueError):
        ens.forward(u[:2], v, w)
    ens.forward(u, v, w, out=out)   # a valid call still works afterwards


def test_ensemble_autotune_keeps_results_and_writes_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("ADVECT_TUNE_CACHE", str(tmp_path / "tune.json"))
    ens, grids, x, lam, dx, dl = build_members(SHAPES, "f32", seed=600)
    ens.autotune(True)
    out = ens.forward(*(fields(dx, f) for f in range(3)))
    grads = ens.adjoint(*(fields(dx, f) for f in range(3)), *(fields(dl, f) for f in range(3)))
    for m in range(len(SHAPES)):
        ref = oracle_forward(*x[m], grids[m])
        refg = oracle_adjoint(*x[m], *lam[m], grids[m])
        for f in range(3):
            assert normwise(host(out[f][m]), ref[f]) <= 2e-6
            assert normwise(host(grads[f][m]), refg[f]) <= 5e-6
    text = (tmp_path / "tune.json").read_text()
    assert "ens_fwd|f32" in text and "ens_adj|f32" in text
    assert ens.tuned_config().startswith("lx=")
    # a new context for the same members starts from the cached choice
    ens2 = torch_api.AdvectEnsemble(SHAPES, [lib_coeffs(g) for g in grids], "f32")
    assert ens2.tuned_config() == ens.tuned_config()
    assert ens2.tuned_config(True) == ens.tuned_config(True)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
def test_single_grid_autotune(tmp_path, monkeypatch, dtype):
    monkeypatch.setenv("ADVECT_TUNE_CACHE", str(tmp_path / "tune.json"))
    shape = (48, 40, 64)
    op, grid = make_op(shape, dtype)
    op.autotune(True)
    winds = workload.winds(*shape, seed=7)
    if dtype == "f16s":
        s_in = [16.0, 16.0, 16.0]
        h = [torch.from_numpy(a / 16.0).to(torch.float16) for a in winds]
        deq = [t.to(torch.float64).numpy() * 16.0 for t in h]
        s_out = op.output_scales(s_in)
        out = op.forward(*(t.cuda() for t in h), scales=s_in + s_out)
        ref = oracle_forward(*deq, grid)
        for t, r, so in zip(out, ref, s_out):
            assert np.max(np.abs(host(t) * so - r)) <= 2.0 ** -11 * so + 2e-6 * np.max(np.abs(r))
    else:
        tdt = torch.float64 if dtype == "f64" else torch.float32
        inp = winds if dtype == "f64" else [a.astype(np.float32).astype(np.float64) for a in winds]
        out = op.forward(*(dev(a, tdt) for a in inp))
        ref = oracle_forward(*inp, grid)
        for t, r in zip(out, ref):
            assert normwise(host(t), r) <= (1e-12 if dtype == "f64" else 2e-6)
        lam = workload.cotangents(*shape, seed=8)
        if dtype == "f32":
            lam = [a.astype(np.float32).astype(np.float64) for a in lam]
        g = op.adjoint(*(dev(a, tdt) for a in (*inp, *lam)))
        refg = oracle_adjoint(*inp, *lam, grid)
        for t, r in zip(g, refg):
            assert normwise(host(t), r) <= (1e-12 if dtype == "f64" else 5e-6)
    assert f"fwd|{dtype}|48x40x64" in (tmp_path / "tune.json").read_text()
    op2, _ = make_op(shape, dtype)
    assert op2.tuned_config() == op.tuned_config()
