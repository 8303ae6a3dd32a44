"""The solver workloads at their own sizes, against the FP64 CPU oracle.

* 32^3 x 8 twisted mass (kappa 0.16, mu 0.01): the FP64 solve and the mixed
  solves with 16-bit inner fields, each compared with the oracle's even-odd
  solve and with the Schur residual the oracle recomputes from the GPU x.
* 32^3 x 8, 12 point sources (one per spin-colour) + 4 Gaussian sources in
  one batched call with FP32 inner iterations and FP64 reliable updates.
* The solve server with 32^3 x 8 and 48^3 x 12 requests beside small ones:
  each result bit for bit the same alone and in the mix, and each meeting
  the target by the oracle's residual.

Tolerances: the GPU's own FP64 true residual <= 1e-10; the oracle's
recomputed residual of the GPU solution <= 1.5e-10 (the same quantity
summed in another order, plus the residual's own rounding); the solution
within 1e-8 of the oracle's solve run to 1e-12 (the condition number of
these systems is below 1e2, so 1e-10 in the residual bounds the error near
1e-8).
"""

import numpy as np
import pytest

import oracle
from paper_1411_5219_gb300 import synthetic as syn
from tests import _fields as F
from tests._solves import schur_residual_oracle, sources_12_point_4_gauss

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def q():
    from paper_1411_5219_gb300 import _build, qcd
    _build.build()
    import torch
    assert torch.cuda.is_available()
    return qcd


@pytest.fixture(scope="module")
def w32(q):
    w = syn.WORKLOADS["32^3x8"]
    dims = w["dims"]
    lat = q.Lattice(dims, -1)
    U = syn.gauge_field(dims, w["eps"], w["seed"])
    g = q.Gauge(lat, "f64", 18)
    g.upload(U)
    return w, lat, U, g


def test_solve_32x8_twisted_full_size(q, w32):
    """32^3 x 8 twisted mass at full size: FP64 and 16-bit mixed solves
    against the oracle's own solve and its recomputed residual."""
    w, lat, U, g = w32
    dims, kappa, mu = w["dims"], w["kappa"], w["mu"]
    b = syn.gaussian_spinor(dims, w["seed"])
    bs = q.Spinor(lat, "full", "f64")
    bs.upload(b)
    xo, sto = oracle.solve_eo(U, b, kappa, mu, tol=1e-12)
    assert sto[1] <= 1e-12
    for inner in ("f64", "f16", "bf16"):
        x = q.Spinor(lat, "full", "f64")
        status, st = q.solve_cg(g, x, bs, kappa, mu, tol=TOL, inner_prec=inner, inner_recon=12)
        assert status == 0 and st["true_rel_residual"] <= TOL, (inner, st)
        xg = x.download()
        assert schur_residual_oracle(U, b, xg, kappa, mu) <= 1.5e-10, inner
        assert F.rel_err(xg, xo) <= 1e-8, inner
        # the full system M x = b: the GPU's own residual agrees with the oracle's
        full = F.rel_err(oracle.apply_m(U, xg, kappa, mu), b)
        assert abs(full - st["full_rel_residual"]) <= 1e-12, inner


def test_solve_multi_12_point_4_gauss_32x8(q, w32):
    """The batched-sources workload at its own size: 32^3 x 8 Wilson,
    kappa 0.16, 12 point + 4 Gaussian sources in one batched CG with FP32
    inner iterations.  Every system's residual is recomputed by the oracle;
    four of them (two point sources, two Gaussian) are also compared with
    the oracle's own solve."""
    w, lat, U, g = w32
    dims, kappa = w["dims"], 0.16
    srcs = sources_12_point_4_gauss(dims, 1005)
    bs, xs = [], []
    for psi in srcs:
        b = q.Spinor(lat, "full", "f64")
        b.upload(psi)
        bs.append(b)
        xs.append(q.Spinor(lat, "full", "f64"))
    status, stats = q.solve_cg_multi(g, xs, bs, kappa, 0.0, tol=TOL, inner_prec="f32", inner_recon=12)
    assert status == 0
    for k, psi in enumerate(srcs):
        assert stats[k]["true_rel_residual"] <= TOL, (k, stats[k])
        xg = xs[k].download()
        assert schur_residual_oracle(U, psi, xg, kappa, 0.0) <= 1.5e-10, k
        if k in (0, 11, 12, 15):
            xo, sto = oracle.solve_eo(U, psi, kappa, 0.0, tol=1e-12)
            assert F.rel_err(xg, xo) <= 1e-8, k


def test_server_mix_with_large_volumes(q):
    """Requests of 8^3x4, 16^3x8, 32^3x8 and 48^3x12 submitted together to
    the solve server: each result equals, bit for bit, the same request run
    alone, and the oracle's residual of each meets the target."""
    vols = [(8, 8, 8, 4), (16, 16, 16, 8), (32, 32, 32, 8), (48, 48, 48, 12)]
    probs = []
    for k, dims in enumerate(vols):
        lat = q.Lattice(dims, -1)
        U = syn.gauge_field(dims, 0.2, 500 + k, device="cuda")
        g = q.Gauge(lat, "f64", 18)
        g.upload(U)
        g.prepare("f16", 12)
        probs.append((lat, U, g))
    sv = q.Server(slots=6, memory_budget=48 << 30)
    gids = [sv.add_gauge(p[2]) for p in probs]
    reqs = []
    for k in range(10):
        pi = [0, 1, 2, 3, 0, 2, 1, 0, 3, 0][k]
        b = syn.gaussian_spinor(vols[pi], 600 + k)
        reqs.append((pi, b, 0.12 + 0.004 * k, 0.01 * (k % 2)))
    alone = []
    for pi, b, kappa, mu in reqs:
        x = np.empty_like(b)
        r = sv.wait(sv.submit(gids[pi], b, x, kappa, mu, inner_prec="f16"))
        assert r["status"] == 0 and r["stats"]["true_rel_residual"] <= TOL, r
        alone.append(x)
    xs = [np.empty_like(b) for _, b, _, _ in reqs]
    ids = [sv.submit(gids[pi], b, xs[k], kappa, mu, inner_prec="f16") for k, (pi, b, kappa, mu) in enumerate(reqs)]
    res = [sv.wait(i) for i in ids]
    sv.close()
    for k, (pi, b, kappa, mu) in enumerate(reqs):
        assert res[k]["status"] == 0, (k, res[k])
        assert np.array_equal(xs[k], alone[k]), k
        assert schur_residual_oracle(probs[pi][1], b, xs[k], kappa, mu) <= 1.5e-10, (k, vols[pi])
