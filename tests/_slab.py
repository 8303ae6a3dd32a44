"""Time-slab split helpers for the tests: cutting a global field into the
slabs of P ranks on extended lattices (own slices 1 .. Lt_loc, halo slices
0 and Lt_loc + 1), the face exchange between ranks, and reassembly.

The exchange sends rank r's face for its previous rank to (r - 1) mod P and
its face for the next rank to (r + 1) mod P, and receives the matching
faces.  It runs over torch.distributed point-to-point calls (any backend)
or, for ranks that live in one process, over an in-process loopback.
"""

import numpy as np


def slab(Lt, world, rank):
    """(t0, Lt_loc) of a rank's slab; Lt_loc must be even."""
    assert Lt % world == 0 and (Lt // world) % 2 == 0
    n = Lt // world
    return rank * n, n


def extend(field, t0, n, fill=None):
    """Own slices t0 .. t0 + n - 1 of a [t, ...] array at 1 .. n of an
    array with two more slices; the halo slices hold `fill` (zeros)."""
    out = np.zeros((n + 2,) + field.shape[1:], dtype=field.dtype)
    if fill is not None:
        out[:] = fill
    out[1:n + 1] = field[t0:t0 + n]
    return out


def extend_gauge(U, t0, n):
    """Extended gauge field: the rank's links on its own slices, identity
    links on the halo slices."""
    return extend(U, t0, n, fill=np.eye(3, dtype=U.dtype))


class Loopback:
    """Face exchange among ranks held by one process."""

    def __init__(self, world):
        self.world = world
        self.box = {}

    def post(self, rank, to_prev, to_next):
        self.box[rank] = (to_prev, to_next)

    def collect(self, rank):
        w = self.world
        return self.box[(rank + 1) % w][0], self.box[(rank - 1) % w][1]


def exchange(rank, world, to_prev, to_next, dist=None, loop=None):
    """Send to_prev to rank - 1 and to_next to rank + 1; return
    (from_next, from_prev): the next rank's face for us and the previous
    rank's.  torch tensors over torch.distributed, or any objects over a
    Loopback (post every rank first, then collect)."""
    if loop is not None:
        return loop.collect(rank)
    import torch
    prev, nxt = (rank - 1) % world, (rank + 1) % world
    from_next, from_prev = torch.empty_like(to_prev), torch.empty_like(to_next)
    reqs = [dist.isend(to_prev.contiguous(), prev), dist.isend(to_next.contiguous(), nxt),
            dist.irecv(from_next, nxt), dist.irecv(from_prev, prev)]
    for r in reqs:
        r.wait()
    return from_next, from_prev
