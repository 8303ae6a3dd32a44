"""The FP64 reconstruct-18 hopping kernel with eight threads per output site
(one hop direction each, summed by warp shuffles) against the FP64 oracle,
forced through qcd_set_hop_threads(8): the even-odd and full-lattice Dslash
of both parities with and without dagger, the Schur operator with twisted
mass (the fused epilogues and the fused norm), and FP64 and mixed solves.
The one-thread-per-site kernel, forced with 1, agrees to rounding.
"""

import numpy as np
import pytest

import oracle
from paper_1411_5219_gb300 import synthetic as syn
from tests import _fields as F
from tests._solves import schur_residual_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_1411_5219_gb300 import _build, qcd
    _build.build()
    import torch
    assert torch.cuda.is_available()
    return qcd


@pytest.fixture
def lanes(q):
    """Yields a setter of the threads per site; puts the autotuner back after."""
    yield q.set_hop_threads
    q.set_hop_threads(0)


def _gauge(q, dims, t_bc=-1, eps=0.3, seed=1201):
    lat = q.Lattice(dims, t_bc)
    U = syn.gauge_field(dims, eps, seed)
    g = q.Gauge(lat, "f64", 18)
    g.upload(U)
    return lat, U, g


# ragged extents, a lattice smaller than one block of 128 threads, and one of many blocks
DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 8), (8, 6, 4, 10), (12, 12, 12, 6)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("dagger", [False, True])
def test_lanes8_dslash_eo(q, lanes, dims, dagger):
    lat, U, g = _gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 1202)
    got = {}
    for tps in (8, 1):
        lanes(tps)
        for out_par in (0, 1):
            half_in = syn.to_half(psi, 1 - out_par)
            si = q.Spinor(lat, "odd" if out_par == 0 else "even", "f64")
            so = q.Spinor(lat, "even" if out_par == 0 else "odd", "f64")
            si.upload(half_in)
            q.apply_dslash(g, so, si, dagger=dagger)
            got[(tps, out_par)] = so.download()
            want = oracle.dhop_eo(U, half_in, out_par, dagger=dagger)
            assert F.rel_err(got[(tps, out_par)], want) <= 1e-13, (tps, out_par)
    for out_par in (0, 1):
        assert F.rel_err(got[(8, out_par)], got[(1, out_par)]) <= 1e-15


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_lanes8_dslash_full(q, lanes, dims, t_bc):
    lanes(8)
    lat, U, g = _gauge(q, dims, t_bc=t_bc)
    psi = syn.gaussian_spinor(dims, 1203)
    si, so = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    si.upload(psi)
    for dagger in (False, True):
        q.apply_dslash(g, so, si, dagger=dagger)
        assert F.rel_err(so.download(), oracle.dhop(U, psi, t_bc=t_bc, dagger=dagger)) <= 1e-13


@pytest.mark.parametrize("kappa,mu", [(0.15, 0.0), (0.16, 0.01), (0.13, 0.4)])
@pytest.mark.parametrize("dagger", [False, True])
def test_lanes8_apply_m_full_and_schur(q, lanes, kappa, mu, dagger):
    lanes(8)
    dims = (8, 6, 4, 10)
    lat, U, g = _gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 1204)
    si, so = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    si.upload(psi)
    q.apply_M(g, so, si, kappa, mu, eo=False, dagger=dagger)
    assert F.rel_err(so.download(), oracle.apply_m(U, psi, kappa, mu, dagger=dagger)) <= 1e-13
    xe = syn.to_half(psi, 0)
    ei, eo_ = q.Spinor(lat, "even", "f64"), q.Spinor(lat, "even", "f64")
    ei.upload(xe)
    q.apply_M(g, eo_, ei, kappa, mu, eo=True, dagger=dagger)
    assert F.rel_err(eo_.download(), oracle.apply_mhat(U, xe, kappa, mu, dagger=dagger)) <= 1e-13


@pytest.mark.parametrize("inner", ["f64", "f16"])
@pytest.mark.parametrize("kappa,mu", [(0.155, 0.0), (0.16, 0.01)])
def test_lanes8_solve_matches_oracle(q, lanes, inner, kappa, mu):
    """The CG's fused operator + norm launches and the FP64 defect and
    verification of the mixed solver all take the eight-lane kernel."""
    lanes(8)
    dims = (8, 8, 8, 4)
    lat, U, g = _gauge(q, dims, eps=0.2, seed=1205)
    b = syn.gaussian_spinor(dims, 1206)
    x, bs = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    bs.upload(b)
    status, st = q.solve_cg(g, x, bs, kappa, mu, tol=1e-10, eo=True, inner_prec=inner, inner_recon=12)
    assert status == 0, st
    assert st["true_rel_residual"] <= 1e-10
    xg = x.download()
    assert schur_residual_oracle(U, b, xg, kappa, mu) <= 1.5e-10
    xo, _ = oracle.solve_eo(U, b, kappa, mu, tol=1e-12)
    assert F.rel_err(xg, xo) <= 1e-7
    assert abs(st["full_rel_residual"] - F.rel_err(oracle.apply_m(U, xg, kappa, mu), b)) <= 1e-12


def test_lanes8_graph_and_eager_bitwise(q, lanes):
    """A captured solve replays the eight-lane launches with the same bits."""
    lanes(8)
    dims = (6, 4, 2, 8)
    lat, U, g = _gauge(q, dims, eps=0.2, seed=1207)
    b = syn.gaussian_spinor(dims, 1208)
    bs = q.Spinor(lat, "full", "f64")
    bs.upload(b)
    out = []
    for mode in ("graph", "eager"):
        x = q.Spinor(lat, "full", "f64")
        if mode == "eager":
            q.profile_begin()  # inside a profiling window the solver launches kernel by kernel
        status, _ = q.solve_cg(g, x, bs, 0.15, 0.01, tol=1e-10, eo=True)
        if mode == "eager":
            assert q.profile_end()["f64"]["launches"] > 0
        assert status == 0
        out.append(x.download())
    assert np.array_equal(out[0], out[1])


def test_set_hop_threads_rejects_other_values(q):
    for bad in (2, 4, -1, 16):
        with pytest.raises(q.QcdError) as e:
            q.set_hop_threads(bad)
        assert e.value.status == 1
    q.set_hop_threads(0)
