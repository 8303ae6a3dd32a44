"""Seeded sweep over lattice shapes and batch sizes, against the FP64 oracle.

The launch-shape choices of the hopping kernel depend on the lattice: the
eight-lane FP64 kernel on small lattices, t-major block order for batched
fields whose time slices tile into whole blocks, one- or two-level grid
reductions by block count.  Each case below draws ragged extents (even,
2..12, time up to 16) and a batch size, and checks every right-hand side
of a batched D_eo / D_eo^dagger against the oracle, and a batched solve's
residuals through the oracle.
"""

import numpy as np
import pytest

import oracle
from paper_1411_5219_gb300 import synthetic as syn
from tests import _fields as F
from tests._solves import schur_residual_oracle

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 8 * 2.0 ** -24, "f16": 8 * 2.0 ** -11}


@pytest.fixture(scope="module")
def q():
    from paper_1411_5219_gb300 import _build, qcd
    _build.build()
    import torch
    assert torch.cuda.is_available()
    return qcd


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        dims = tuple(int(2 * rng.integers(1, 7)) for _ in range(3)) + (int(2 * rng.integers(1, 9)),)
        nrhs = int(rng.choice([1, 2, 3, 5, 8, 16]))
        out.append((dims, nrhs))
    return out


@pytest.mark.parametrize("dims,nrhs", _cases(10, 1501))
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 12), ("f16", 12)])
def test_batched_dslash_random_shapes(q, dims, nrhs, prec, recon):
    lat = q.Lattice(dims, -1)
    U = syn.gauge_field(dims, 0.3, 1502)
    g = q.Gauge(lat, "f64", recon)
    g.upload(U)
    srcs = [syn.to_half(syn.gaussian_spinor(dims, 1510 + k), 1) for k in range(nrhs)]
    for dagger in (False, True):
        ins, outs = [], []
        for psi in srcs:
            si = q.Spinor(lat, "odd", prec)
            si.upload(psi)
            ins.append(si)
            outs.append(q.Spinor(lat, "even", prec))
        q.apply_dslash_multi(g, outs, ins, dagger=dagger)
        for k, psi in enumerate(srcs):
            want = oracle.dhop_eo(U, psi, 0, dagger=dagger)
            assert F.rel_err(outs[k].download(), want) <= TOL[prec], (dims, nrhs, k, dagger)


@pytest.mark.parametrize("dims,nrhs", _cases(4, 1601))
def test_batched_solve_random_shapes(q, dims, nrhs):
    """FP16-inner batched solve to 1e-10 on a drawn shape: every system's
    Schur residual recomputed by the oracle."""
    lat = q.Lattice(dims, -1)
    U = syn.gauge_field(dims, 0.2, 1602)
    g = q.Gauge(lat, "f64", 18)
    g.upload(U)
    bs, xs, hs = [], [], []
    for k in range(nrhs):
        b = syn.gaussian_spinor(dims, 1610 + k)
        s = q.Spinor(lat, "full", "f64")
        s.upload(b)
        bs.append(s)
        hs.append(b)
        xs.append(q.Spinor(lat, "full", "f64"))
    status, stats = q.solve_cg_multi(g, xs, bs, 0.14, 0.01, tol=1e-10, inner_prec="f16")
    assert status == 0
    for k in range(nrhs):
        assert stats[k]["true_rel_residual"] <= 1e-10
        assert schur_residual_oracle(U, hs[k], xs[k].download(), 0.14, 0.01) <= 1.5e-10, (dims, nrhs, k)
