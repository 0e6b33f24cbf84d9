"""The x-slab decomposition run by two processes with the library's kernels.

Two gloo ranks (world size 2), both on the one GPU this run has: each owns an
x-slab of the grid padded with one halo plane per side, fills its halos from
the neighbour with decomp.exchange_x_halos on host-staged planes (the
periodic halo swap of Sec. 2.1), then runs advect_forward and advect_adjoint
on its padded slab through the C ABI.  The owned planes must match the FP64
oracle on the whole grid within the 1e-12 bar.  The ranks exchange planes
only between launches on the host; no kernel of one rank waits for another.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (70, 42, 64)     # several tiles per slab in x and y, ragged tails


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, dtype, q):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import workload
        from paper_2010_01545_gb300 import decomp, torch_api
        torch.cuda.set_device(0)
        grid = workload.vertical_grid(SHAPE[2])
        c = oracle.coefficients(grid)
        tdt = torch.float64 if dtype == "f64" else torch.float32
        winds = [a.astype(np.float32).astype(np.float64) if dtype == "f32" else a
                 for a in workload.winds(*SHAPE, seed=61)]
        lam = [a.astype(np.float32).astype(np.float64) if dtype == "f32" else a
               for a in workload.cotangents(*SHAPE, seed=62)]
        i0, i1 = decomp.slab_bounds(SHAPE[0], world, rank)
        # each rank holds only its owned planes of the global fields; the
        # halo planes come from the neighbours
        own = [torch.from_numpy(np.ascontiguousarray(a[i0:i1])).to(tdt) for a in (*winds, *lam)]
        slabs = []
        for t in own:
            s = torch.empty((i1 - i0 + 2,) + SHAPE[1:], dtype=tdt)
            s[1:-1] = t
            slabs.append(s)
        decomp.exchange_x_halos(slabs)
        nloc = i1 - i0 + 2
        op = torch_api.Advect(nloc, SHAPE[1], SHAPE[2], torch_api.coefficients_from_grid(grid), dtype)
        d = [s.cuda() for s in slabs]
        fwd = [t[1:-1].double().cpu().numpy() for t in op.forward(*d[:3])]
        adj = [t[1:-1].double().cpu().numpy() for t in op.adjoint(*d)]
        full_f = oracle.forward(*winds, c)
        full_a = oracle.adjoint(*winds, *lam, c)
        errs = []
        for g, r in zip(fwd + adj, list(full_f) + list(full_a)):
            r = r[i0:i1]
            errs.append(float(np.max(np.abs(g - r)) / np.max(np.abs(r))))
        q.put((rank, (i0, i1), errs, op.kernel_name(), op.kernel_name(True)))
        op.close()
    except Exception as e:  # report, then leave the group cleanly
        q.put((rank, None, repr(e), "", ""))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 5e-6)])
def test_two_ranks_forward_and_adjoint_on_halo_exchanged_slabs_match_the_oracle(dtype, tol):
    from gpu_util import ensure_built
    ensure_built()                       # build once, before the ranks start
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, dtype, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [(0, 35), (35, 70)], res
    for rank, _, errs, kf, ka in res:
        assert kf == "fwd_sweep" and ka == "adj_sweep", (kf, ka)
        for name, e in zip(("su", "sv", "sw", "du", "dv", "dw"), errs):
            assert e <= tol, f"rank {rank} {name}: normwise error {e:.3e}"
