"""x-slab domain decomposition with a periodic one-plane halo exchange.

The stencil reads the +-1 neighbours, so a grid split into x-slabs across
ranks needs, before each call, the last plane of the left neighbour and the
first plane of the right neighbour (periodic in x) -- MONC's halo swap of the
prognostic fields (Sec. 2.1).  In the [nx][ny][nz] layout a plane is one
contiguous block, so a slab padded with one halo plane on each side is
contiguous too, and the single-grid kernel computes the owned planes
1..n_local of the padded slab unchanged (its periodic wrap only touches the
two halo planes, whose outputs are discarded).

Host-side logic over torch.distributed (any backend); the exchange is the
only communication and uses point-to-point send/recv.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def slab_bounds(nx: int, world: int, rank: int):
    """[i0, i1) of the x-planes owned by rank (as even as possible)."""
    if not 0 <= rank < world or nx < world:
        raise ValueError("need 0 <= rank < world <= nx")
    return nx * rank // world, nx * (rank + 1) // world


def padded_slab(field: torch.Tensor, i0: int, i1: int) -> torch.Tensor:
    """Owned planes [i0, i1) of a global field with two empty halo planes."""
    out = torch.empty((i1 - i0 + 2,) + tuple(field.shape[1:]), dtype=field.dtype, device=field.device)
    out[1:-1] = field[i0:i1]
    return out


def exchange_x_halos(slabs, group=None) -> None:
    """Fill halo planes 0 and -1 of each padded slab from the neighbours.

    Every rank sends its first owned plane to the left neighbour and its last
    owned plane to the right neighbour (periodic), and receives the matching
    planes into its halos.  With one rank the slab is its own neighbour."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    left, right = (rank - 1) % world, (rank + 1) % world
    for s in slabs:
        if world == 1:
            s[0] = s[-2]
            s[-1] = s[1]
            continue
        first = s[1].contiguous()
        last = s[-2].contiguous()
        recv_left = torch.empty_like(first)
        recv_right = torch.empty_like(last)
        # tags tell the two planes apart when left and right are the same rank
        to_right_halo, to_left_halo = 1, 2
        ops = [dist.P2POp(dist.isend, first, left, group, to_right_halo),
               dist.P2POp(dist.isend, last, right, group, to_left_halo),
               dist.P2POp(dist.irecv, recv_left, left, group, to_left_halo),
               dist.P2POp(dist.irecv, recv_right, right, group, to_right_halo)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        s[0] = recv_left
        s[-1] = recv_right


def fill_x_halos_local(slabs_by_rank) -> None:
    """The same exchange for sub-domains held by one process (several slabs
    on one device, e.g. to run a decomposed grid on fewer GPUs than ranks):
    slabs_by_rank[r] is rank r's list of padded slabs (one per field); halo
    plane 0 of rank r takes the last owned plane of rank r-1 and halo plane
    -1 the first owned plane of rank r+1 (periodic)."""
    world = len(slabs_by_rank)
    for r in range(world):
        left, right = slabs_by_rank[(r - 1) % world], slabs_by_rank[(r + 1) % world]
        for s, sl, sr in zip(slabs_by_rank[r], left, right):
            s[0] = sl[-2]
            s[-1] = sr[1]
