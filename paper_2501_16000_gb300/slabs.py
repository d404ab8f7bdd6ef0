"""One lattice spread over ranks as y-slabs: the halo exchange of a step.

A time step at a node needs the post-collision populations of its eight
neighbours (the streaming of Eqs. 1/7), so a lattice split into slabs of
rows exchanges, per step, one row each way: after the collision a rank
sends the populations of its top row that move up (c_y = +1: directions 2,
5, 6) to the rank above and those of its bottom row that move down
(c_y = -1: directions 4, 7, 8) to the rank below, 3 x nx values each way,
periodic in y over the ranks.  Streaming then runs on the slab extended by
one ghost row on each side holding the received values; x stays periodic
within the slab.  Nothing else crosses ranks, so the slabs together advance
exactly as the whole lattice does.

This module holds the plan (which rows, which directions, where received
values go) and the exchange over ``torch.distributed`` (point-to-point
send/receive, gloo on CPU ranks).  The collision and the streaming are the
caller's.  States are canonical population arrays [9][rows][nx] in the D2Q9
order (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
"""
from __future__ import annotations

import numpy as np

CX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
CY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
UP = tuple(i for i in range(9) if CY[i] == 1)      # (2, 5, 6)
DOWN = tuple(i for i in range(9) if CY[i] == -1)   # (4, 7, 8)

_TAG_UP, _TAG_DOWN = 11, 12


def slab_rows(ny: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [y0, y1) of rank `rank`: ny split into `world` slabs whose
    heights differ by at most one (the first ny % world are one taller)."""
    if not 1 <= world <= ny:
        raise ValueError(f"{world} ranks cannot each hold a row of {ny}")
    base, extra = divmod(ny, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def pack_halos(post: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(to the rank above, to the rank below): the up-moving populations of
    the slab's top row and the down-moving ones of its bottom row, each
    [3][nx] contiguous."""
    return (np.ascontiguousarray(post[list(UP), -1, :]),
            np.ascontiguousarray(post[list(DOWN), 0, :]))


def extend(post: np.ndarray, from_below: np.ndarray, from_above: np.ndarray) -> np.ndarray:
    """The slab's post-collision state [9][rows][nx] with one ghost row below
    and above, [9][rows + 2][nx]: the ghost rows hold the received moving
    populations (the rest zero, as nothing of them streams into the slab).
    Streaming this array periodically leaves the slab's rows exact; what it
    wraps between the two ghost rows is discarded with them."""
    q, rows, nx = post.shape
    ext = np.zeros((q, rows + 2, nx))
    ext[:, 1:rows + 1, :] = post
    ext[list(UP), 0, :] = from_below
    ext[list(DOWN), rows + 1, :] = from_above
    return ext


def interior(streamed: np.ndarray) -> np.ndarray:
    """The slab's own rows of a streamed extended array."""
    return streamed[:, 1:-1, :]


def exchange(post: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Sends this rank's halos to its neighbours and receives theirs over the
    default process group; returns (from_below, from_above), each [3][nx]."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(), dist.get_rank()
    up, down = pack_halos(post)
    if world == 1:                        # the slab is the whole (periodic) lattice
        return up, down
    above, below = (rank + 1) % world, (rank - 1) % world
    recv_below = torch.empty(up.shape, dtype=torch.float64)
    recv_above = torch.empty(down.shape, dtype=torch.float64)
    reqs = [dist.isend(torch.from_numpy(up), above, tag=_TAG_UP),
            dist.isend(torch.from_numpy(down), below, tag=_TAG_DOWN),
            dist.irecv(recv_below, below, tag=_TAG_UP),
            dist.irecv(recv_above, above, tag=_TAG_DOWN)]
    for r in reqs:
        r.wait()
    return recv_below.numpy(), recv_above.numpy()


def step(f: np.ndarray, collide_slab, stream) -> np.ndarray:
    """One time step of this rank's slab S_t [9][rows][nx] -> S_{t+1}:
    `collide_slab(f)` returns the post-collision slab, `stream(a)` streams a
    [9][r][nx] array periodically (push: a_i(x) lands at x + c_i)."""
    post = collide_slab(f)
    from_below, from_above = exchange(post)
    return interior(stream(extend(post, from_below, from_above)))
