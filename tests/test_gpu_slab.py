"""The time-slab split on the GPU: P slabs of one lattice, each on its own
extended lattice (own slices plus two halo slices), exchange projected
half-spinor faces packed by qcd_face_pack, unpack them with
qcd_face_unpack, and apply the unchanged hopping kernel.  The assembled
D_eo matches the unsplit GPU kernel and the oracle.  The ranks live in one
process and exchange through the loopback of the same harness the CPU test
runs over gloo (no kernel waits on another; every exchange is between
launches)."""

import numpy as np
import pytest

import oracle
from paper_1411_5219_gb300 import synthetic as syn
from tests import _fields as F
from tests import _slab

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_1411_5219_gb300 import _build, qcd
    _build.build()
    import torch
    assert torch.cuda.is_available()
    return qcd


def _ext_half(field_ext, dims_ext, parity):
    return syn.to_half(field_ext, parity)


@pytest.mark.parametrize("world,dims", [(2, (6, 4, 4, 8)), (3, (4, 4, 2, 12)), (2, (8, 8, 8, 8))])
@pytest.mark.parametrize("dagger", [False, True])
def test_slab_faces_reproduce_the_unsplit_dslash(q, world, dims, dagger):
    import torch
    U = syn.gauge_field(dims, 0.3, 41)
    psi = syn.gaussian_spinor(dims, 42)
    Lx, Ly, Lz, Lt = dims
    par = syn.parity_of_sites(dims)
    psi_odd = psi * (par == 1)[..., None, None]  # input sites: odd; output: even
    # unsplit reference on the GPU and the oracle
    lat = q.Lattice(dims, -1)
    g = q.Gauge(lat, "f64", 18)
    g.upload(U)
    si, so = q.Spinor(lat, "odd", "f64"), q.Spinor(lat, "even", "f64")
    si.upload(syn.to_half(psi, 1))
    q.apply_dslash(g, so, si, dagger=dagger)
    whole_gpu = so.download()
    whole_oracle = oracle.dhop_eo(U, syn.to_half(psi, 1), 0, dagger=dagger)
    # the slabs: with t0 even, global parity p is local parity 1 - p
    st = Lx * Ly * Lz // 2
    loop = _slab.Loopback(world)
    ranks = []
    for r in range(world):
        t0, n = _slab.slab(Lt, world, r)
        dims_e = (Lx, Ly, Lz, n + 2)
        lat_e = q.Lattice(dims_e, 1)
        g_e = q.Gauge(lat_e, "f64", 18)
        g_e.upload(_slab.extend_gauge(U, t0, n))
        pe = _slab.extend(psi_odd, t0, n)
        ine, oute = q.Spinor(lat_e, "even", "f64"), q.Spinor(lat_e, "odd", "f64")
        ine.upload(syn.to_half(pe, 0))
        to_prev = torch.empty(6 * st * 2, dtype=torch.float64, device="cuda")
        to_next = torch.empty_like(to_prev)
        q.face_pack(g_e, ine, q.FACE_TO_PREV, to_prev.data_ptr(), dagger=dagger, sign=-1.0 if r == 0 else 1.0)
        q.face_pack(g_e, ine, q.FACE_TO_NEXT, to_next.data_ptr(), dagger=dagger,
                    sign=-1.0 if r == world - 1 else 1.0)
        loop.post(r, to_prev, to_next)
        ranks.append((t0, n, dims_e, lat_e, g_e, ine, oute, to_prev, to_next))
    parts = []
    for r, (t0, n, dims_e, lat_e, g_e, ine, oute, to_prev, to_next) in enumerate(ranks):
        from_next, from_prev = _slab.exchange(r, world, to_prev, to_next, loop=loop)
        q.face_unpack(ine, q.FACE_FROM_NEXT, from_next.data_ptr())
        q.face_unpack(ine, q.FACE_FROM_PREV, from_prev.data_ptr())
        q.apply_dslash(g_e, oute, ine, dagger=dagger)
        full_e = syn.from_half(np.zeros_like(oute.download()), oute.download(), dims_e)
        parts.append(full_e[1:n + 1])
    split = np.concatenate(parts, axis=0)
    got = syn.to_half(split, 0)
    assert F.rel_err(got, whole_oracle) <= 1e-13
    assert F.rel_err(got, whole_gpu) <= 1e-14
    # the odd sites of the assembled field stay zero
    assert np.all(syn.to_half(split, 1) == 0)


def test_face_pack_rejects_other_lattices(q):
    import torch
    lat = q.Lattice((4, 4, 4, 4), -1)  # not an extended slab (t_bc = -1)
    g = q.Gauge(lat, "f64", 18)
    g.upload(syn.gauge_field((4, 4, 4, 4), 0.3, 1))
    s = q.Spinor(lat, "even", "f64")
    buf = torch.empty(6 * 32 * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QcdError):
        q.face_pack(g, s, q.FACE_TO_PREV, buf.data_ptr())
