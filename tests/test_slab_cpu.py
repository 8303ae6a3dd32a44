"""The time-slab split of the hopping term on the CPU: two gloo ranks each
hold half of the time slices, exchange their boundary time slices (with the
global antiperiodic sign applied by the sender whose slice crosses the time
boundary) and the t links of their last slice, and apply the oracle's D_hop
on their extended slab.  The reassembled result equals the unsplit oracle's
bit for bit: every site sees the same numbers in the same order (the paper
splits the lattice in time across devices, Sec. 7)."""

import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DIMS = (4, 4, 2, 8)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def split_dhop(rank, world, U, psi, dagger, dist=None, loop=None, step=None):
    """This rank's slab of D_hop psi through the face exchange."""
    import torch
    from tests import _slab
    import oracle
    Lt = U.shape[0]
    t0, n = _slab.slab(Lt, world, rank)
    Ue, pe = _slab.extend_gauge(U, t0, n), _slab.extend(psi, t0, n)
    tb = -1.0  # antiperiodic in time
    first, last = psi[t0], psi[t0 + n - 1]
    to_prev = first * (tb if rank == 0 else 1.0)
    to_next = last * (tb if rank == world - 1 else 1.0)
    # the backward hop of the next rank's first slice needs our last t links
    links = U[t0 + n - 1, :, :, :, 3]
    pack = lambda a: torch.from_numpy(np.ascontiguousarray(a)).view(torch.float64)  # noqa: E731
    if loop is not None:
        loop.post(rank, (to_prev, None), (to_next, links))
        if step == "post":
            return None
        (fn, _), (fp, fl) = loop.collect(rank)
    else:
        from_next, from_prev = _slab.exchange(rank, world, pack(to_prev), pack(to_next), dist=dist)
        _, from_links = _slab.exchange(rank, world, pack(np.zeros_like(links)), pack(links), dist=dist)
        fn = from_next.view(torch.complex128).numpy().reshape(first.shape)
        fp = from_prev.view(torch.complex128).numpy().reshape(first.shape)
        fl = from_links.view(torch.complex128).numpy().reshape(links.shape)
    pe[n + 1] = fn
    pe[0] = fp
    Ue[0, :, :, :, 3] = fl
    out = oracle.dhop(Ue, pe, t_bc=1.0, dagger=dagger)
    return out[1:n + 1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1411_5219_gb300 import synthetic as syn
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    U = syn.gauge_field(DIMS, 0.3, 31)
    psi = syn.gaussian_spinor(DIMS, 32)
    res = [split_dhop(rank, world, U, psi, dagger, dist=dist) for dagger in (False, True)]
    q.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_slab_split_dhop_bitwise_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1411_5219_gb300 import synthetic as syn
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    U = syn.gauge_field(DIMS, 0.3, 31)
    psi = syn.gaussian_spinor(DIMS, 32)
    for k, dagger in enumerate((False, True)):
        whole = oracle.dhop(U, psi, t_bc=-1.0, dagger=dagger)
        split = np.concatenate([got[0][k], got[1][k]], axis=0)
        assert np.array_equal(split, whole), dagger


def test_slab_split_three_ranks_in_process():
    """The same exchange harness with three ranks in one process."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1411_5219_gb300 import synthetic as syn
    from tests import _slab
    dims = (4, 2, 2, 12)
    U = syn.gauge_field(dims, 0.3, 33)
    psi = syn.gaussian_spinor(dims, 34)
    loop = _slab.Loopback(3)
    for r in range(3):
        split_dhop(r, 3, U, psi, False, loop=loop, step="post")
    parts = [split_dhop(r, 3, U, psi, False, loop=loop) for r in range(3)]
    assert np.array_equal(np.concatenate(parts, axis=0), oracle.dhop(U, psi, t_bc=-1.0))
