"""Multi-rank host logic on CPU with the gloo backend (world size 2).

* bench.py's whole-job rate: units summed over ranks over the slowest rank's
  time, the same value on every rank;
* the x-slab decomposition with a periodic one-plane halo exchange: each
  rank computes its slab (here with the oracle, standing in for the kernel)
  and the owned planes equal the full-grid result bitwise.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _rate_worker(rank, world, port, q):
    _init(rank, world, port)
    import bench
    units = [1000.0, 3000.0][rank]
    secs = [2.0, 5.0][rank]
    q.put((rank, bench.whole_job_rate(units, secs, "cpu")))
    dist.destroy_process_group()


def _decomp_worker(rank, world, port, q):
    _init(rank, world, port)
    import oracle
    import workload
    from paper_2010_01545_gb300 import decomp
    shape = (10, 6, 8)
    grid = workload.vertical_grid(shape[2])
    c = oracle.coefficients(grid)
    fields = [torch.from_numpy(a) for a in workload.winds(*shape, seed=5)]
    i0, i1 = decomp.slab_bounds(shape[0], world, rank)
    slabs = [decomp.padded_slab(f, i0, i1) for f in fields]
    decomp.exchange_x_halos(slabs)
    out = oracle.forward(*(s.numpy() for s in slabs), c, i_range=(1, i1 - i0 + 1))
    full = oracle.forward(*(f.numpy() for f in fields), c)
    ok = all(np.array_equal(o[1:-1], r[i0:i1]) for o, r in zip(out, full))
    q.put((rank, ok, (i0, i1)))
    dist.destroy_process_group()


def _run(worker, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res)


def test_whole_job_rate_two_gloo_ranks():
    res = _run(_rate_worker)
    for _, (value, secs) in res:
        assert secs == 5.0
        assert value == pytest.approx(4000.0 / 5.0)


@pytest.mark.parametrize("world,bounds", [(2, [(0, 5), (5, 10)]), (3, [(0, 3), (3, 6), (6, 10)])])
def test_slab_decomposition_with_halo_exchange_matches_full_grid(world, bounds):
    res = _run(_decomp_worker, world)
    assert [r[2] for r in res] == bounds
    assert all(r[1] for r in res)


def test_slab_bounds():
    from paper_2010_01545_gb300 import decomp
    assert [decomp.slab_bounds(10, 3, r) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    with pytest.raises(ValueError):
        decomp.slab_bounds(2, 3, 0)


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_local_halo_fill_matches_full_grid(world):
    """Sub-domains held by one process: the oracle on each padded slab gives
    the full-grid result on the owned planes, bitwise."""
    import oracle
    import workload
    from paper_2010_01545_gb300 import decomp
    shape = (11, 5, 8)
    c = oracle.coefficients(workload.vertical_grid(shape[2]))
    fields = [torch.from_numpy(a) for a in workload.winds(*shape, seed=6)]
    bounds = [decomp.slab_bounds(shape[0], world, r) for r in range(world)]
    slabs = [[decomp.padded_slab(f, i0, i1) for f in fields] for i0, i1 in bounds]
    decomp.fill_x_halos_local(slabs)
    full = oracle.forward(*(f.numpy() for f in fields), c)
    for (i0, i1), sl in zip(bounds, slabs):
        assert all(torch.equal(s[0], f[(i0 - 1) % shape[0]]) and torch.equal(s[-1], f[i1 % shape[0]])
                   for s, f in zip(sl, fields))
        out = oracle.forward(*(s.numpy() for s in sl), c, i_range=(1, i1 - i0 + 1))
        assert all(np.array_equal(o[1:-1], r[i0:i1]) for o, r in zip(out, full))
