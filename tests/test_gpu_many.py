"""Several even-odd FP64 solves of different lattice volumes in one
persistent launch (qcd_solve_cg_many), against the FP64 CPU oracle.

Each system has its own gauge field, volume, kappa, mu and tolerance.  Every
solution is compared with the oracle's own even-odd solve (run to 1e-12) and
its Schur residual is recomputed by the oracle; the batch result of each
system is bitwise the one it gets alone; a barrier budget that runs out ends
the call with QCD_ERR_TIMEOUT and leaves the context usable.
"""

import numpy as np
import pytest

import oracle
from paper_1411_5219_gb300 import synthetic as syn
from tests import _fields as F
from tests._solves import schur_residual_oracle

pytestmark = pytest.mark.gpu

# (dims, kappa, mu, tol, link seed): uneven volumes, ragged extents, Wilson and twisted mass
SYSTEMS = [((8, 8, 8, 4), 0.13, 0.0, 1e-10, 701),
           ((4, 4, 4, 4), 0.15, 0.01, 1e-10, 702),
           ((6, 4, 2, 8), 0.14, 0.02, 1e-11, 703),
           ((12, 12, 12, 6), 0.155, 0.0, 1e-10, 704),
           ((16, 16, 16, 8), 0.12, 0.01, 1e-10, 705)]


@pytest.fixture(scope="module")
def q():
    from paper_1411_5219_gb300 import _build, qcd
    _build.build()
    import torch
    assert torch.cuda.is_available()
    return qcd


@pytest.fixture(scope="module")
def problems(q):
    out = []
    for k, (dims, kappa, mu, tol, seed) in enumerate(SYSTEMS):
        lat = q.Lattice(dims, -1)
        U = syn.gauge_field(dims, 0.2, seed)
        g = q.Gauge(lat, "f64", 18)
        g.upload(U)
        b = syn.gaussian_spinor(dims, 800 + k)
        bs = q.Spinor(lat, "full", "f64")
        bs.upload(b)
        out.append(dict(dims=dims, kappa=kappa, mu=mu, tol=tol, U=U, g=g, lat=lat, b=b, bs=bs))
    return out


def _solve(q, probs):
    xs = [q.Spinor(p["lat"], "full", "f64") for p in probs]
    status, stats = q.solve_cg_many([p["g"] for p in probs], xs, [p["bs"] for p in probs],
                                    [p["kappa"] for p in probs], [p["mu"] for p in probs],
                                    [p["tol"] for p in probs])
    return status, stats, [x.download() for x in xs]


def test_many_uneven_volumes_match_oracle(q, problems):
    status, stats, xs = _solve(q, problems)
    assert status == 0
    for p, st, x in zip(problems, stats, xs):
        assert st["true_rel_residual"] <= p["tol"], (p["dims"], st)
        assert schur_residual_oracle(p["U"], p["b"], x, p["kappa"], p["mu"]) <= 1.5 * p["tol"], p["dims"]
        xo, sto = oracle.solve_eo(p["U"], p["b"], p["kappa"], p["mu"], tol=1e-12)
        assert F.rel_err(x, xo) <= 1e-8, p["dims"]
        full = F.rel_err(oracle.apply_m(p["U"], x, p["kappa"], p["mu"]), p["b"])
        assert abs(full - st["full_rel_residual"]) <= 1e-12, p["dims"]


def test_many_same_alone_and_in_batch(q, problems):
    """Blocks are shared out per system and every sum has a fixed order: a
    system's solution has the same bits alone and in the batch."""
    _, _, batch = _solve(q, problems)
    for k in (0, 2, 4):
        _, _, alone = _solve(q, [problems[k]])
        assert np.array_equal(alone[0], batch[k]), k


def test_many_systems_sharing_a_gauge_field(q, problems):
    """Several kappa values on one gauge field (one lattice handle): each
    system keeps its own scratch fields."""
    p = problems[0]
    probs = [dict(p, kappa=kap) for kap in (0.12, 0.13, 0.135)]
    status, stats, xs = _solve(q, probs)
    assert status == 0
    for pp, st, x in zip(probs, stats, xs):
        assert st["true_rel_residual"] <= 1e-10
        assert schur_residual_oracle(p["U"], p["b"], x, pp["kappa"], 0.0) <= 1.5e-10


def test_many_barrier_timeout_is_reported(q, problems):
    """A barrier budget of one cycle cannot be met: the call ends with
    QCD_ERR_TIMEOUT, and a normal call afterwards succeeds."""
    xs = [q.Spinor(p["lat"], "full", "f64") for p in problems[:2]]
    status, _ = q.solve_cg_many([p["g"] for p in problems[:2]], xs, [p["bs"] for p in problems[:2]],
                                [0.13, 0.15], wait_cycles=1, raise_on_error=False)
    assert status == 6  # QCD_ERR_TIMEOUT
    status, stats, _ = _solve(q, problems[:2])
    assert status == 0 and all(st["true_rel_residual"] <= 1e-10 for st in stats)


def test_many_rejects_bad_arguments(q, problems):
    p = problems[0]
    x = q.Spinor(p["lat"], "full", "f64")
    with pytest.raises(q.QcdError) as e:
        q.solve_cg_many([], [], [], [])
    assert e.value.status == 1
    # x on another lattice than its gauge field
    x2 = q.Spinor(problems[1]["lat"], "full", "f64")
    with pytest.raises(q.QcdError):
        q.solve_cg_many([p["g"]], [x2], [p["bs"]], [0.13])
    # one x for two systems
    with pytest.raises(q.QcdError):
        q.solve_cg_many([p["g"], p["g"]], [x, x], [p["bs"], p["bs"]], [0.13, 0.12])


def test_server_batches_small_requests(q):
    """Small requests queued together on one slot run as one persistent
    launch: several share start and end times, and each meets its target by
    the oracle's residual."""
    dims = (8, 8, 8, 4)
    lat = q.Lattice(dims, -1)
    U = syn.gauge_field(dims, 0.2, 710)
    g = q.Gauge(lat, "f64", 18)
    g.upload(U)
    sv = q.Server(slots=1, memory_budget=4 << 30, batch_small_sites=8192)
    gid = sv.add_gauge(g)
    reqs = [(syn.gaussian_spinor(dims, 720 + k), 0.12 + 0.003 * k) for k in range(12)]
    xs = [np.empty_like(b) for b, _ in reqs]
    ids = [sv.submit(gid, b, x, kap) for (b, kap), x in zip(reqs, xs)]
    res = [sv.wait(i) for i in ids]
    sv.close()
    assert all(r["status"] == 0 for r in res)
    starts = [r["t_start"] for r in res]
    assert max(starts.count(t) for t in starts) >= 2  # at least one batch of two or more
    for (b, kap), x in zip(reqs, xs):
        assert schur_residual_oracle(U, b, x, kap, 0.0) <= 1.5e-10


def test_many_grid_cap_keeps_the_bits(q, problems):
    """A grid capped at one block per system (max_blocks = n) gives the same
    bits as the full resident grid: reductions are summed per fixed chunk."""
    probs = problems[:3]
    _, _, full = _solve(q, probs)
    xs = [q.Spinor(p["lat"], "full", "f64") for p in probs]
    status, _ = q.solve_cg_many([p["g"] for p in probs], xs, [p["bs"] for p in probs],
                                [p["kappa"] for p in probs], [p["mu"] for p in probs], [p["tol"] for p in probs],
                                max_blocks=len(probs))
    assert status == 0
    for a, x in zip(full, xs):
        assert np.array_equal(a, x.download())
    with pytest.raises(q.QcdError):
        q.solve_cg_many([p["g"] for p in probs], xs, [p["bs"] for p in probs], [0.13] * 3, max_blocks=2)
