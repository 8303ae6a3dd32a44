"""GPU (libqcd, sm_103a) against the FP64 CPU oracle, element by element.

Every call goes through the C ABI (ctypes binding).  Tolerances:
* FP64 operators: norm-wise relative error <= 1e-13 (the Dslash target);
* low-precision storage: norm-wise relative error <= c * u with u the unit
  roundoff of the storage format (FP32 2^-24, FP16 2^-11, BF16 2^-8): each
  input component is rounded once (relative to the site's largest
  component for FP16), the links are rounded once, the result is rounded
  once, and FP32 arithmetic adds ~1e-7; c = 8 covers these three roundings
  with margin (see the test of the bound itself below);
* solves: FP64 true residual <= tol = 1e-10 on the CG system, and the
  solution within cond * tol of the oracle's (run to 1e-12).
"""

import numpy as np
import pytest

import oracle
from paper_1411_5219_gb300 import synthetic as syn
from tests import _fields as F
from tests._solves import schur_residual_oracle, sources_12_point_4_gauss

pytestmark = pytest.mark.gpu

U_ROUND = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}


def tol_of(prec):
    return 1e-13 if prec == "f64" else 8 * U_ROUND[prec]


@pytest.fixture(scope="module")
def q():
    from paper_1411_5219_gb300 import _build, qcd
    _build.build()
    import torch
    assert torch.cuda.is_available()
    return qcd


_CACHE = {}


def field_set(q, dims, eps=0.3, seed=1001, t_bc=-1):
    key = (dims, eps, seed, t_bc)
    if key not in _CACHE:
        lat = q.Lattice(dims, t_bc)
        U = syn.gauge_field(dims, eps, seed)
        _CACHE[key] = (lat, U, {})
    return _CACHE[key]


def gauge(q, dims, prec="f64", recon=18, eps=0.3, seed=1001, t_bc=-1):
    lat, U, gs = field_set(q, dims, eps, seed, t_bc)
    if (prec, recon) not in gs:
        g = q.Gauge(lat, prec, recon)
        g.upload(U)
        gs[(prec, recon)] = g
    return lat, U, gs[(prec, recon)]


DIMS = [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 2, 8), (8, 6, 4, 10), (12, 12, 12, 6)]


# ----------------------------------------------------------- layout round trip

@pytest.mark.parametrize("parity", ["full", "even", "odd"])
def test_upload_download_roundtrip_f64_bitexact(q, parity):
    dims = (6, 4, 2, 8)
    lat, _, _ = gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 5)
    host = psi if parity == "full" else syn.to_half(psi, 0 if parity == "even" else 1)
    s = q.Spinor(lat, parity, "f64")
    s.upload(host)
    assert np.array_equal(s.download(), host)


def test_upload_f32_rounds_to_nearest(q):
    dims = (4, 4, 4, 4)
    lat, _, _ = gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 6)
    s = q.Spinor(lat, "full", "f32")
    s.upload(psi)
    assert np.array_equal(s.download(), psi.astype(np.complex64).astype(np.complex128))


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_upload_16bit_within_rounding(q, prec):
    dims = (4, 4, 4, 4)
    lat, _, _ = gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 7)
    s = q.Spinor(lat, "full", prec)
    s.upload(psi)
    back = s.download()
    if prec == "f16":  # per-site scale: error <= u * (site max) per component
        smax = np.maximum(np.abs(psi.real), np.abs(psi.imag)).max(axis=(4, 5), keepdims=True)
        assert np.all(np.abs((back - psi).real) <= U_ROUND[prec] * smax * 1.0001)
        assert np.all(np.abs((back - psi).imag) <= U_ROUND[prec] * smax * 1.0001)
    else:
        assert np.all(np.abs((back - psi).real) <= U_ROUND[prec] * np.abs(psi.real) * 1.0001 + 1e-30)


def test_norm2_matches_numpy(q):
    dims = (8, 6, 4, 10)
    lat, _, _ = gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 8)
    s = q.Spinor(lat, "full", "f64")
    s.upload(psi)
    assert abs(s.norm2() - np.vdot(psi, psi).real) < 1e-12 * np.vdot(psi, psi).real


@pytest.mark.parametrize("dims", [(6, 4, 2, 8), (24, 24, 24, 24), (48, 48, 48, 12)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_norm2_one_and_two_level_reductions(q, dims, prec):
    """The grid reduction in one level (a few blocks) and in two (2592 and
    10,368 blocks of 128: groups of 2048 blocks, then the group sums), against
    numpy on the stored values."""
    lat = q.Lattice(dims, -1)
    rng = np.random.default_rng(1401)
    psi = (rng.standard_normal(dims[::-1] + (4, 3)) + 1j * rng.standard_normal(dims[::-1] + (4, 3)))
    if prec == "f32":
        psi = psi.astype(np.complex64).astype(np.complex128)
    s = q.Spinor(lat, "full", prec)
    s.upload(psi)
    want = float(np.vdot(psi, psi).real)
    # FP32 fields: each site's 24 squares are summed in float before the FP64 reduction
    assert abs(s.norm2() - want) <= (1e-13 if prec == "f64" else 2e-7) * want


# -------------------------------------------------------------------- Dslash

@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("recon", [18, 12])
def test_dslash_eo_f64(q, dims, dagger, recon):
    lat, U, g = gauge(q, dims, recon=recon)
    psi = syn.gaussian_spinor(dims, 11)
    for out_par in (0, 1):
        half_in = syn.to_half(psi, 1 - out_par)
        want = oracle.dhop_eo(U, half_in, out_par, dagger=dagger)
        si = q.Spinor(lat, "odd" if out_par == 0 else "even", "f64")
        so = q.Spinor(lat, "even" if out_par == 0 else "odd", "f64")
        si.upload(half_in)
        q.apply_dslash(g, so, si, dagger=dagger)
        assert F.rel_err(so.download(), want) <= 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_dslash_full_f64(q, dims, t_bc):
    lat, U, g = gauge(q, dims, t_bc=t_bc)
    psi = syn.gaussian_spinor(dims, 12)
    si, so = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    si.upload(psi)
    for dagger in (False, True):
        q.apply_dslash(g, so, si, dagger=dagger)
        assert F.rel_err(so.download(), oracle.dhop(U, psi, t_bc=t_bc, dagger=dagger)) <= 1e-13


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("dims", [(8, 6, 4, 10), (12, 12, 12, 6)])
def test_dslash_eo_low_precision(q, prec, recon, dims):
    lat, U, g = gauge(q, dims, recon=recon)
    psi = syn.gaussian_spinor(dims, 13)
    for dagger in (False, True):
        half_in = syn.to_half(psi, 1)
        want = oracle.dhop_eo(U, half_in, 0, dagger=dagger)
        si, so = q.Spinor(lat, "odd", prec), q.Spinor(lat, "even", prec)
        si.upload(half_in)
        q.apply_dslash(g, so, si, dagger=dagger)
        err = F.rel_err(so.download(), want)
        assert err <= tol_of(prec), (prec, recon, err)


def _round16(a, prec):
    """float32 array rounded to FP16 or BF16 (round to nearest even), back in float32."""
    a = np.asarray(a, dtype=np.float32)
    if prec == "f16":
        return a.astype(np.float16).astype(np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _stored_spinor(half, prec):
    """The values a 16-bit half field holds: FP32, then FP16 relative to the
    site's largest |real part| (FP16) or BF16 as is."""
    v = np.stack([half.real, half.imag], axis=-1).astype(np.float32)  # [site, 4, 3, 2]
    if prec == "f16":
        m = np.abs(v).reshape(v.shape[0], -1).max(axis=1).astype(np.float32)
        inv = np.where(m > 0, np.float32(1) / np.where(m > 0, m, 1), 0).astype(np.float32)
        q = _round16(v * inv[:, None, None, None], prec) * m[:, None, None, None]
    else:
        q = _round16(v, prec)
    q = q.astype(np.float64)
    return q[..., 0] + 1j * q[..., 1]


def _stored_links_recon12(U, prec):
    """16-bit reconstruct-12 links: rows 0 and 1 rounded, row 2 rebuilt as
    conj(row0 x row1) (in FP64 here; the GPU rebuilds in FP32)."""
    r = np.stack([U.real, U.imag], axis=-1).astype(np.float32)
    r = _round16(r, prec).astype(np.float64)
    V = r[..., 0] + 1j * r[..., 1]
    V[..., 2, :] = np.conj(np.cross(V[..., 0, :], V[..., 1, :]))
    return V


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_low_precision_bound_from_storage_rounding(q, prec):
    """The 8u tolerance of the 16-bit tests, taken apart: a model that rounds
    the inputs as the storage does and then computes exactly is within 2u of
    the GPU result (the output rounding, FP32 arithmetic and, for FP16, the
    FP16 rounding of each projected half spinor), and within 6u of the exact
    result (the input and link roundings)."""
    dims = (8, 6, 4, 10)
    lat, U, g = gauge(q, dims, recon=12)
    half_in = syn.to_half(syn.gaussian_spinor(dims, 13), 1)
    si, so = q.Spinor(lat, "odd", prec), q.Spinor(lat, "even", prec)
    si.upload(half_in)
    q.apply_dslash(g, so, si)
    exact = oracle.dhop_eo(U, half_in, 0)
    model = oracle.dhop_eo(_stored_links_recon12(U, prec), _stored_spinor(half_in, prec), 0)
    u = U_ROUND[prec]
    assert F.rel_err(so.download(), model) <= 2 * u
    assert F.rel_err(model, exact) <= 6 * u
    assert F.rel_err(so.download(), exact) <= tol_of(prec)


def test_dslash_point_source_support(q):
    """A delta source feeds exactly the 8 neighbour sites (bit-exact zeros elsewhere)."""
    dims = (6, 4, 4, 4)
    lat, U, g = gauge(q, dims)
    src = syn.point_source(dims, 1, 2, site=(3, 0, 2, 3))
    si, so = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    si.upload(src)
    q.apply_dslash(g, so, si)
    out = so.download()
    nz = {tuple(v) for v in np.argwhere(np.abs(out).sum(axis=(4, 5)) > 0)}
    want = set()
    for mu in range(4):
        for d in (1, -1):
            c = [3, 0, 2, 3]
            c[mu] = (c[mu] + d) % dims[mu]
            want.add((c[3], c[2], c[1], c[0]))
    assert nz == want
    assert F.rel_err(out, oracle.dhop(U, src)) <= 1e-13


# ------------------------------------------------------------------ operators

@pytest.mark.parametrize("kappa,mu", [(0.15, 0.0), (0.16, 0.01), (0.13, 0.4)])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_m_full_and_schur_f64(q, kappa, mu, dagger):
    dims = (8, 6, 4, 10)
    lat, U, g = gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 14)
    si, so = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    si.upload(psi)
    q.apply_M(g, so, si, kappa, mu, eo=False, dagger=dagger)
    assert F.rel_err(so.download(), oracle.apply_m(U, psi, kappa, mu, dagger=dagger)) <= 1e-13
    xe = syn.to_half(psi, 0)
    ei, eo_ = q.Spinor(lat, "even", "f64"), q.Spinor(lat, "even", "f64")
    ei.upload(xe)
    q.apply_M(g, eo_, ei, kappa, mu, eo=True, dagger=dagger)
    assert F.rel_err(eo_.download(), oracle.apply_mhat(U, xe, kappa, mu, dagger=dagger)) <= 1e-13


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_apply_schur_low_precision(q, prec):
    dims = (8, 6, 4, 10)
    kappa, mu = 0.16, 0.01
    lat, U, g = gauge(q, dims, recon=12)
    xe = syn.to_half(syn.gaussian_spinor(dims, 15), 0)
    ei, eo_ = q.Spinor(lat, "even", prec), q.Spinor(lat, "even", prec)
    ei.upload(xe)
    q.apply_M(g, eo_, ei, kappa, mu, eo=True)
    assert F.rel_err(eo_.download(), oracle.apply_mhat(U, xe, kappa, mu)) <= tol_of(prec)


def test_lattice_destroyed_before_its_fields(q):
    """Fields keep their lattice alive: destroying the lattice first leaves
    its spinors and gauge field usable, and destroying them afterwards (in
    any order, as a cyclic garbage collection may) frees it."""
    dims = (4, 4, 4, 4)
    lat = q.Lattice(dims, -1)
    U = syn.gauge_field(dims, 0.3, 1301)
    g = q.Gauge(lat, "f64", 18)
    g.upload(U)
    psi = syn.gaussian_spinor(dims, 1302)
    si, so = q.Spinor(lat, "odd", "f64"), q.Spinor(lat, "even", "f64")
    si.upload(syn.to_half(psi, 1))
    lat.close()
    q.apply_dslash(g, so, si)
    assert F.rel_err(so.download(), oracle.dhop_eo(U, syn.to_half(psi, 1), 0)) <= 1e-13
    si.close()
    g.close()
    so.close()
    # a spinor outliving its lattice still uploads and downloads
    lat2 = q.Lattice(dims, -1)
    s2 = q.Spinor(lat2, "full", "f64")
    lat2.close()
    s2.upload(psi)
    assert np.array_equal(s2.download(), psi)
    s2.close()


def test_invalid_arguments_rejected(q):
    lat, U, g = gauge(q, (4, 4, 4, 4))
    a, b = q.Spinor(lat, "even", "f64"), q.Spinor(lat, "even", "f64")
    with pytest.raises(q.QcdError) as e:
        q.apply_dslash(g, a, b)  # same parity
    assert e.value.status == 1
    c = q.Spinor(lat, "odd", "f32")
    with pytest.raises(q.QcdError):
        q.apply_dslash(g, a, c)  # precisions differ
    with pytest.raises(q.QcdError):
        q.apply_M(g, a, b, 0.1, eo=False)  # eo=0 needs FULL fields


# --------------------------------------------------------------------- solves

def test_solve_full_normal_4x4_config(q):
    """4^4, kappa = 0.15, antiperiodic t, eps = 0.3: CG on M^dag M x = b."""
    w = syn.WORKLOADS["4^4"]
    dims = w["dims"]
    lat, U, g = gauge(q, dims, eps=w["eps"], seed=w["seed"])
    b = syn.gaussian_spinor(dims, w["seed"])
    x = q.Spinor(lat, "full", "f64")
    bs = q.Spinor(lat, "full", "f64")
    bs.upload(b)
    status, st = q.solve_cg(g, x, bs, w["kappa"], tol=1e-10, eo=False, normal=True)
    assert status == 0 and st["true_rel_residual"] <= 1e-10 and st["full_rel_residual"] <= 1e-10
    xg = x.download()
    xo, so = oracle.solve_mdagm(U, b, w["kappa"], tol=1e-12)
    assert F.rel_err(xg, xo) <= 1e-8
    r = b - oracle.apply_m(U, oracle.apply_m(U, xg, w["kappa"]), w["kappa"], dagger=True)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


@pytest.mark.parametrize("inner", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("kappa,mu", [(0.155, 0.0), (0.16, 0.01)])
def test_solve_eo_matches_oracle(q, inner, kappa, mu):
    dims = (8, 8, 8, 4)
    lat, U, g = gauge(q, dims, eps=0.2, seed=77)
    b = syn.gaussian_spinor(dims, 78)
    x, bs = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    bs.upload(b)
    status, st = q.solve_cg(g, x, bs, kappa, mu, tol=1e-10, eo=True, inner_prec=inner, inner_recon=12)
    assert status == 0, st
    assert st["true_rel_residual"] <= 1e-10
    xg = x.download()
    assert schur_residual_oracle(U, b, xg, kappa, mu) <= 1.5e-10
    xo, so = oracle.solve_eo(U, b, kappa, mu, tol=1e-12)
    assert F.rel_err(xg, xo) <= 1e-7
    assert abs(st["full_rel_residual"] - F.rel_err(oracle.apply_m(U, xg, kappa, mu), b)) <= 1e-12
    if inner != "f64":
        assert st["reliable_updates"] >= 1


@pytest.mark.parametrize("inner", ["f32", "f16", "bf16"])
def test_reliable_delta_default_by_precision(q, inner):
    """reliable_delta = 0 picks the factor from the inner precision (FP32
    1e-3, FP16 1e-2, BF16 0.1): no more FP64 updates than at 0.1, the same
    target met, and the solution the oracle's; values outside [0, 1) fail."""
    dims = (8, 8, 8, 4)
    lat, U, g = gauge(q, dims, eps=0.2, seed=77)
    b = syn.gaussian_spinor(dims, 81)
    bs = q.Spinor(lat, "full", "f64")
    bs.upload(b)
    res = {}
    for delta in (0.0, 0.1):
        x = q.Spinor(lat, "full", "f64")
        status, st = q.solve_cg(g, x, bs, 0.155, 0.01, tol=1e-10, inner_prec=inner, reliable_delta=delta)
        assert status == 0, (delta, st)
        assert schur_residual_oracle(U, b, x.download(), 0.155, 0.01) <= 1.5e-10
        res[delta] = st["reliable_updates"]
    assert res[0.0] <= res[0.1], res
    if inner != "bf16":
        assert res[0.0] < res[0.1], res
    for bad in (1.0, -0.1):
        with pytest.raises(q.QcdError):
            q.solve_cg(g, q.Spinor(lat, "full", "f64"), bs, 0.155, tol=1e-10, inner_prec=inner, reliable_delta=bad)


@pytest.mark.parametrize("inner", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("kappa", [0.12, 0.125, 0.13])
def test_solve_mixed_near_critical_kappa(q, inner, kappa):
    """Near the critical kappa of these near-identity links the Schur operator
    is badly conditioned: the mixed solve, whose reliable updates recompute
    the residual in FP64, must still reach the FP64 target."""
    dims = (8, 8, 8, 4)
    lat, U, g = gauge(q, dims, eps=0.2, seed=1107)
    src = syn.gaussian_spinor(dims, 86)
    b, x = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    b.upload(src)
    status, st = q.solve_cg(g, x, b, kappa, 0.0, tol=1e-10, inner_prec=inner)
    assert status == 0 and st["true_rel_residual"] <= 1e-10, st
    assert schur_residual_oracle(U, src, x.download(), kappa, 0.0) <= 1.5e-10


def test_solve_full_cgnr_matches_eo(q):
    dims = (4, 4, 4, 8)
    lat, U, g = gauge(q, dims, eps=0.2, seed=90)
    b = syn.gaussian_spinor(dims, 91)
    bs = q.Spinor(lat, "full", "f64")
    bs.upload(b)
    xs = []
    for eo in (True, False):
        x = q.Spinor(lat, "full", "f64")
        status, st = q.solve_cg(g, x, bs, 0.15, 0.02, tol=1e-11, eo=eo)
        assert status == 0
        xs.append(x.download())
    assert F.rel_err(xs[0], xs[1]) <= 1e-8


@pytest.mark.parametrize("inner", ["f16", "f32"])
@pytest.mark.parametrize("normal", [False, True])
def test_solve_full_lattice_mixed(q, inner, normal):
    """Mixed-precision CG on the full lattice, CGNR on M and CG on
    M^dag M x = b (each reliable update recomputes the residual in FP64),
    against the oracle's solves."""
    dims = (4, 4, 4, 8)
    kappa, mu = 0.15, 0.02
    lat, U, g = gauge(q, dims, eps=0.2, seed=90)
    b = syn.gaussian_spinor(dims, 92)
    bs, x = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    bs.upload(b)
    status, st = q.solve_cg(g, x, bs, kappa, mu, tol=1e-10, eo=False, normal=normal, inner_prec=inner)
    assert status == 0 and st["true_rel_residual"] <= 1e-10, st
    if normal:
        xo, _ = oracle.solve_mdagm(U, b, kappa, mu, tol=1e-12)
    else:
        xo, _ = oracle.solve_m(U, b, kappa, mu, tol=1e-12)
    assert F.rel_err(x.download(), xo) <= 1e-7


def test_solve_zero_source_and_errors(q):
    dims = (4, 4, 4, 4)
    lat, U, g = gauge(q, dims)
    x, bs = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    bs.upload(np.zeros((4, 4, 4, 4, 4, 3), dtype=complex))
    status, st = q.solve_cg(g, x, bs, 0.15)
    assert status == 0 and st["iterations"] == 0 and np.all(x.download() == 0)
    bs.upload(syn.gaussian_spinor(dims, 3))
    status, st = q.solve_cg(g, x, bs, 0.15, maxiter=3, raise_on_error=False)
    assert status == 4 and st["iterations"] == 3 and st["true_rel_residual"] > 1e-10
    nanb = syn.gaussian_spinor(dims, 3)
    nanb[0, 0, 0, 0, 0, 0] = np.nan
    bs.upload(nanb)
    status, st = q.solve_cg(g, x, bs, 0.15, raise_on_error=False)
    assert status == 5


# ------------------------------------------------ full-size workloads (sampled)

@pytest.mark.parametrize("name", ["24^3x8", "48^3x12"])
def test_dslash_full_size_sampled(q, name):
    """At the benchmark volumes: the FP64 D_eo of the bench launch shape,
    checked at 4096 sampled even sites against the oracle, site by site."""
    w = syn.WORKLOADS[name]
    dims = w["dims"]
    lat, U, g = gauge(q, dims, eps=w["eps"], seed=w["seed"])
    psi = syn.gaussian_spinor(dims, w["seed"])
    half_in = syn.to_half(psi, 1)
    si, so = q.Spinor(lat, "odd", "f64"), q.Spinor(lat, "even", "f64")
    si.upload(half_in)
    q.apply_dslash(g, so, si)
    out = so.download()
    full_in = psi * (syn.parity_of_sites(dims) == 1)[..., None, None]
    even_sites = np.flatnonzero(syn.parity_of_sites(dims).reshape(-1) == 0)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(len(even_sites), 4096, replace=False))
    pick[:2] = [0, len(even_sites) - 1]  # first and last site (boundary wrap)
    want = oracle.dhop_sites(U, full_in, even_sites[pick])
    got = out[pick]
    assert F.rel_err(got, want) <= 1e-13
    # every output finite, and the norm consistent with a random field
    assert np.all(np.isfinite(out))


@pytest.mark.parametrize("name", ["24^3x8", "48^3x12"])
@pytest.mark.parametrize("prec,recon", [("f32", 12), ("f16", 12), ("bf16", 12), ("f16", 8)])
def test_dslash_low_precision_full_size_sampled(q, name, prec, recon):
    """The inner-solver formats at the benchmark volumes, in the bench's launch
    shape: 4096 sampled output sites against the oracle, norm-wise within the
    storage tolerance, and every output finite."""
    w = syn.WORKLOADS[name]
    dims = w["dims"]
    lat, U, g = gauge(q, dims, recon=recon, eps=w["eps"], seed=w["seed"])
    psi = syn.gaussian_spinor(dims, w["seed"] + 7)
    half_in = syn.to_half(psi, 1)
    si, so = q.Spinor(lat, "odd", prec), q.Spinor(lat, "even", prec)
    si.upload(half_in)
    q.apply_dslash(g, so, si)
    out = so.download()
    full_in = psi * (syn.parity_of_sites(dims) == 1)[..., None, None]
    even_sites = np.flatnonzero(syn.parity_of_sites(dims).reshape(-1) == 0)
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(len(even_sites), 4096, replace=False))
    pick[:2] = [0, len(even_sites) - 1]
    want = oracle.dhop_sites(U, full_in, even_sites[pick])
    assert F.rel_err(out[pick], want) <= tol_of(prec), (name, prec, recon)
    assert np.all(np.isfinite(out))


def test_solve_48x12_twisted_full_size(q):
    """The 48^3 x 12 twisted-mass workload (kappa 0.16, mu 0.01) at full size,
    as the bench runs it: the FP16 mixed solve and the FP64 solve both reach
    1e-10, the oracle's recomputed Schur residual of the GPU solution agrees,
    and the two solutions match."""
    w = syn.WORKLOADS["48^3x12"]
    dims, kappa, mu = w["dims"], w["kappa"], w["mu"]
    lat, U, g = gauge(q, dims, eps=w["eps"], seed=w["seed"])
    b = syn.gaussian_spinor(dims, w["seed"] + 1)
    bs = q.Spinor(lat, "full", "f64")
    bs.upload(b)
    xs = {}
    for inner in ("f16", "f64"):
        x = q.Spinor(lat, "full", "f64")
        status, st = q.solve_cg(g, x, bs, kappa, mu, tol=1e-10, inner_prec=inner)
        assert status == 0 and st["true_rel_residual"] <= 1e-10, (inner, st)
        xs[inner] = x.download()
    assert schur_residual_oracle(U, b, xs["f16"], kappa, mu) <= 1.5e-10
    assert F.rel_err(xs["f16"], xs["f64"]) <= 1e-8
    # the oracle's own even-odd CG at this volume, run once to 1e-12
    xo, sto = oracle.solve_eo(U, b, kappa, mu, tol=1e-12)
    assert sto[1] <= 1e-12
    for inner in ("f16", "f64"):
        assert F.rel_err(xs[inner], xo) <= 1e-8, inner


def test_solve_eo_24x8_true_residual(q):
    """The 24^3 x 8 FP64 even-odd solve: its true residual recomputed by the oracle."""
    w = syn.WORKLOADS["24^3x8"]
    dims = w["dims"]
    lat, U, g = gauge(q, dims, eps=w["eps"], seed=w["seed"])
    b = syn.gaussian_spinor(dims, w["seed"])
    x, bs = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    bs.upload(b)
    status, st = q.solve_cg(g, x, bs, w["kappa"], tol=1e-10, eo=True)
    assert status == 0 and st["true_rel_residual"] <= 1e-10
    xg = x.download()
    assert abs(F.rel_err(oracle.apply_m(U, xg, w["kappa"]), b) - st["full_rel_residual"]) <= 1e-12
    assert schur_residual_oracle(U, b, xg, w["kappa"], 0.0) <= 1.5e-10


# ------------------------------------------- graph path, eager path, profiling

@pytest.mark.parametrize("inner", ["f64", "f16"])
def test_graph_and_eager_solves_bitwise_identical(q, inner):
    """The solver replays a captured CUDA graph of the CG loop; inside a
    profiling window it launches kernel by kernel.  Both run the same kernels
    on the same data with fixed-order reductions: identical bits."""
    dims = (8, 8, 8, 4)
    lat, U, g = gauge(q, dims, eps=0.2, seed=77)
    b = syn.gaussian_spinor(dims, 79)
    bs = q.Spinor(lat, "full", "f64")
    bs.upload(b)
    outs = []
    for mode in ("graph", "graph", "eager"):
        x = q.Spinor(lat, "full", "f64")
        if mode == "eager":
            q.profile_begin()
        status, st = q.solve_cg(g, x, bs, 0.16, 0.01, tol=1e-10, inner_prec=inner)
        if mode == "eager":
            prof = q.profile_end()
            assert prof["f64"]["launches"] > 0
        assert status == 0
        outs.append((x.download(), st["iterations"], st["reliable_updates"]))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and o[1:] == outs[0][1:]


def test_profile_accounting(q):
    dims = (8, 6, 4, 10)
    lat, U, g = gauge(q, dims)
    h = syn.volume(dims) // 2
    si, so = q.Spinor(lat, "odd", "f64"), q.Spinor(lat, "even", "f64")
    q.profile_begin()
    q.apply_dslash(g, so, si)
    p = q.profile_end()
    e = p["f64"]
    assert e["launches"] == 1 and e["sites"] == h
    assert e["bytes"] == h * (8 * 144 + 2 * 192) and e["flops"] == h * 1320 and e["ms"] > 0
    n0 = q.kernel_launches()
    q.apply_dslash(g, so, si)
    assert q.kernel_launches() == n0 + 1


# --------------------------------------------------------- double-float (DF64)

def test_df64_roundtrip_48_bits(q):
    dims = (6, 4, 2, 8)
    lat, _, _ = gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 21)
    s = q.Spinor(lat, "full", "df64")
    s.upload(psi)
    back = s.download()
    # hi = RN(d), lo = RN(d - hi): |d - (hi + lo)| <= 2^-48 |d| per real part
    assert np.all(np.abs((back - psi).real) <= 2.0 ** -48 * np.abs(psi.real))
    assert np.all(np.abs((back - psi).imag) <= 2.0 ** -48 * np.abs(psi.imag))


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_eo_df64(q, dims, dagger):
    """Double-float Dslash from FP64 data: within the FP64 target 1e-13."""
    lat, U, g = gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 22)
    for out_par in (0, 1):
        half_in = syn.to_half(psi, 1 - out_par)
        want = oracle.dhop_eo(U, half_in, out_par, dagger=dagger)
        si = q.Spinor(lat, "odd" if out_par == 0 else "even", "df64")
        so = q.Spinor(lat, "even" if out_par == 0 else "odd", "df64")
        si.upload(half_in)
        q.apply_dslash(g, so, si, dagger=dagger)
        err = F.rel_err(so.download(), want)
        assert err <= 1e-13, err


@pytest.mark.parametrize("kappa,mu", [(0.155, 0.0), (0.16, 0.01)])
def test_apply_m_df64(q, kappa, mu):
    dims = (8, 6, 4, 10)
    lat, U, g = gauge(q, dims)
    psi = syn.gaussian_spinor(dims, 23)
    si, so = q.Spinor(lat, "full", "df64"), q.Spinor(lat, "full", "df64")
    si.upload(psi)
    for dagger in (False, True):
        q.apply_M(g, so, si, kappa, mu, eo=False, dagger=dagger)
        assert F.rel_err(so.download(), oracle.apply_m(U, psi, kappa, mu, dagger=dagger)) <= 1e-13
        xe = syn.to_half(psi, 0)
        ei, eo_ = q.Spinor(lat, "even", "df64"), q.Spinor(lat, "even", "df64")
        ei.upload(xe)
        q.apply_M(g, eo_, ei, kappa, mu, eo=True, dagger=dagger)
        assert F.rel_err(eo_.download(), oracle.apply_mhat(U, xe, kappa, mu, dagger=dagger)) <= 1e-13


@pytest.mark.parametrize("kappa,mu", [(0.155, 0.0), (0.16, 0.01)])
def test_solve_df64_inner(q, kappa, mu):
    """CG iterating in double-float, FP64 reliable updates (delta = 1e-5)."""
    dims = (8, 8, 8, 4)
    lat, U, g = gauge(q, dims, eps=0.2, seed=77)
    b = syn.gaussian_spinor(dims, 78)
    x, bs = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    bs.upload(b)
    status, st = q.solve_cg(g, x, bs, kappa, mu, tol=1e-10, eo=True, inner_prec="df64", reliable_delta=1e-5)
    assert status == 0 and st["true_rel_residual"] <= 1e-10
    assert 1 <= st["reliable_updates"] <= 4
    xg = x.download()
    assert schur_residual_oracle(U, b, xg, kappa, mu) <= 1.5e-10
    xo, _ = oracle.solve_eo(U, b, kappa, mu, tol=1e-12)
    assert F.rel_err(xg, xo) <= 1e-7


def test_df64_recon12_rejected(q):
    lat, U, g = gauge(q, (4, 4, 4, 4), recon=12)
    si, so = q.Spinor(lat, "odd", "df64"), q.Spinor(lat, "even", "df64")
    with pytest.raises(q.QcdError):
        q.apply_dslash(g, so, si)


# ------------------------------------------------------ batched multi-RHS

@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 12), ("f16", 12), ("df64", 18)])
@pytest.mark.parametrize("nrhs", [16, 3])
def test_dslash_multi_matches_oracle(q, prec, recon, nrhs):
    dims = (8, 6, 4, 10)
    lat, U, g = gauge(q, dims, recon=recon)
    srcs = sources_12_point_4_gauss(dims, 40)[:nrhs]
    for dagger in (False, True):
        ins, outs = [], []
        for k, psi in enumerate(srcs):
            si = q.Spinor(lat, "odd", prec)
            si.upload(syn.to_half(psi, 1))
            ins.append(si)
            outs.append(q.Spinor(lat, "even", prec))
        q.apply_dslash_multi(g, outs, ins, dagger=dagger)
        for k, psi in enumerate(srcs):
            want = oracle.dhop_eo(U, syn.to_half(psi, 1), 0, dagger=dagger)
            if not np.any(want):
                continue
            assert F.rel_err(outs[k].download(), want) <= tol_of(prec if prec != "df64" else "f64"), (k, prec)


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
def test_solve_multi_12_point_4_gauss(q, inner):
    """16 sources (one point source per spin-colour + 4 Gaussian) in one
    batched CG; each solution matches its single-RHS solve and meets 1e-10."""
    dims = (8, 8, 8, 4)
    kappa, mu = 0.155, 0.0
    lat, U, g = gauge(q, dims, eps=0.2, seed=77)
    srcs = sources_12_point_4_gauss(dims, 50)
    bs, xs = [], []
    for psi in srcs:
        b = q.Spinor(lat, "full", "f64")
        b.upload(psi)
        bs.append(b)
        xs.append(q.Spinor(lat, "full", "f64"))
    status, stats = q.solve_cg_multi(g, xs, bs, kappa, mu, tol=1e-10, inner_prec=inner)
    assert status == 0
    for k, psi in enumerate(srcs):
        assert stats[k]["true_rel_residual"] <= 1e-10, (k, stats[k])
        x1 = q.Spinor(lat, "full", "f64")
        st1, s1 = q.solve_cg(g, x1, bs[k], kappa, mu, tol=1e-10, inner_prec=inner)
        xb = xs[k].download()
        assert F.rel_err(xb, x1.download()) <= 1e-8
        if k in (0, 7, 12, 15):
            assert schur_residual_oracle(U, psi, xb, kappa, mu) <= 1.5e-10


def test_solve_multi_padding_and_zero(q):
    """3 systems (padded to 4) including a zero source: that one is solved at once."""
    dims = (4, 4, 4, 8)
    lat, U, g = gauge(q, dims, eps=0.2, seed=90)
    srcs = [syn.gaussian_spinor(dims, 91), np.zeros((8, 4, 4, 4, 4, 3), dtype=complex), syn.gaussian_spinor(dims, 92)]
    bs, xs = [], []
    for psi in srcs:
        b = q.Spinor(lat, "full", "f64")
        b.upload(psi)
        bs.append(b)
        xs.append(q.Spinor(lat, "full", "f64"))
    status, stats = q.solve_cg_multi(g, xs, bs, 0.15, 0.02, tol=1e-10)
    assert status == 0
    assert np.all(xs[1].download() == 0) and stats[1]["iterations"] == 0
    for k in (0, 2):
        xo, _ = oracle.solve_eo(U, srcs[k], 0.15, 0.02, tol=1e-12)
        assert F.rel_err(xs[k].download(), xo) <= 1e-7


@pytest.mark.parametrize("inner", ["f64", "f16"])
def test_solve_batch_mixed_kappa_mu_tol(q, inner):
    """Four systems with their own kappa, mu and tolerance in one batched CG
    (the operator's coefficients are read per right-hand side): each meets its
    own tolerance, the oracle's recomputed residual agrees, and each matches
    its single-system solve."""
    dims = (8, 8, 8, 4)
    lat, U, g = gauge(q, dims, eps=0.2, seed=77)
    kappas, mus, tols = [0.12, 0.14, 0.155, 0.16], [0.0, 0.05, 0.0, 0.01], [1e-10, 1e-8, 1e-10, 1e-11]
    srcs = [syn.gaussian_spinor(dims, 80 + k) for k in range(4)]
    bs, xs = [], []
    for psi in srcs:
        b = q.Spinor(lat, "full", "f64")
        b.upload(psi)
        bs.append(b)
        xs.append(q.Spinor(lat, "full", "f64"))
    status, stats = q.solve_cg_batch(g, xs, bs, kappas, mus, tols, inner_prec=inner)
    assert status == 0
    for k in range(4):
        assert stats[k]["true_rel_residual"] <= tols[k], (k, stats[k])
        xb = xs[k].download()
        assert schur_residual_oracle(U, srcs[k], xb, kappas[k], mus[k]) <= 1.5 * tols[k], k
        x1 = q.Spinor(lat, "full", "f64")
        q.solve_cg(g, x1, bs[k], kappas[k], mus[k], tol=tols[k], inner_prec=inner)
        assert F.rel_err(xb, x1.download()) <= 1e3 * tols[k], k
    if inner == "f64":
        # systems that meet their tolerance early keep iterating until all have:
        # the FP64 batch pays one true-residual check, not one per system
        assert all(s_["reliable_updates"] == 1 for s_ in stats)


def test_solve_batch_rejects_mixed_settings(q):
    import ctypes
    from paper_1411_5219_gb300.qcd import SolverParams, SolverStats, PREC, lib, _handles
    dims = (4, 4, 4, 4)
    lat, U, g = gauge(q, dims)
    bs = [q.Spinor(lat, "full", "f64") for _ in range(2)]
    xs = [q.Spinor(lat, "full", "f64") for _ in range(2)]
    for b in bs:
        b.upload(syn.gaussian_spinor(dims, 85))
    prm = (SolverParams * 2)(SolverParams(0.15, 0.0, 1e-10, 1000, 1, 0, PREC["f64"], 12, 0.1),
                             SolverParams(0.15, 0.0, 1e-10, 1000, 1, 0, PREC["f16"], 12, 0.1))
    st = (SolverStats * 2)()
    assert lib().qcd_solve_cg_batch(g.handle, _handles(xs), _handles(bs), 2, prm, st, None) == 1
    assert b"kappa, mu and tol only" in lib().qcd_last_error()


def test_autotuner_file_cache(tmp_path):
    """The block-size autotuner writes its choice to QCD_TUNE_CACHE; a second
    process reads it back instead of timing again."""
    import os
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1411_5219_gb300 import qcd, synthetic as syn\n"
        "lat = qcd.Lattice((8, 8, 8, 4), -1); g = qcd.Gauge(lat, 'f64', 12); g.upload(syn.gauge_field((8, 8, 8, 4), 0.2, 1))\n"
        "a, b = qcd.Spinor(lat, 'odd', 'f32'), qcd.Spinor(lat, 'even', 'f32')\n"
        "qcd.apply_dslash(g, b, a); qcd.stream_sync()\n"
    ) % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, QCD_TUNE_CACHE=str(cache))
    subprocess.run([sys.executable, "-c", code], check=True, env=env)
    lines = cache.read_text().split()
    assert len(lines) == 2 and lines[0].startswith("dslash:p1:r12:n0:b0:8x8x8x4") and lines[1] in ("64", "128", "256")
    subprocess.run([sys.executable, "-c", code], check=True, env=env)
    assert cache.read_text().split() == lines


# ----------------------------------------------------------------- server

def _server_problem(q, dims, seed):
    lat = q.Lattice(dims, -1)
    U = syn.gauge_field(dims, 0.2, seed)
    g = q.Gauge(lat, "f64", 18)
    g.upload(U)
    g.prepare("f16", 12)
    return lat, U, g


def test_server_same_alone_and_in_mix(q):
    """Each request's solution is bit for bit the same when it runs alone and
    when it runs concurrently with other requests of other volumes."""
    probs = [_server_problem(q, d, 300 + k) for k, d in enumerate([(8, 8, 8, 4), (12, 12, 12, 4), (16, 16, 16, 8)])]
    sv = q.Server(slots=4, memory_budget=8 << 30)
    gids = [sv.add_gauge(p[2]) for p in probs]
    reqs = []
    for k in range(9):
        pi = k % 3
        dims = probs[pi][0].dims
        b = syn.gaussian_spinor(dims, 400 + k)
        reqs.append((pi, b, 0.12 + 0.005 * k))
    alone = []
    for pi, b, kappa in reqs:
        x = np.empty_like(b)
        r = sv.wait(sv.submit(gids[pi], b, x, kappa, inner_prec="f16"))
        assert r["status"] == 0 and r["stats"]["true_rel_residual"] <= 1e-10
        alone.append(x)
    xs = [np.empty_like(b) for _, b, _ in reqs]
    ids = [sv.submit(gids[pi], b, xs[k], kappa, inner_prec="f16") for k, (pi, b, kappa) in enumerate(reqs)]
    res = [sv.wait(i) for i in ids]
    for k in range(len(reqs)):
        assert res[k]["status"] == 0
        assert np.array_equal(xs[k], alone[k]), k
    pi, b, kappa = reqs[4]
    assert schur_residual_oracle(probs[pi][1], b, xs[4], kappa, 0.0) <= 1.5e-10
    sv.close()


def test_server_recovers_from_a_failed_context_build(q):
    """A solver context whose build fails part-way (its first spinor
    allocation fails, injected on the host) is dropped whole: that request
    ends with QCD_ERR_OOM, and the next request for the same volume on the
    same slot builds the context again and solves."""
    dims = (8, 8, 8, 4)
    lat, U, g = _server_problem(q, dims, 321)
    sv = q.Server(slots=1, memory_budget=4 << 30)
    gid = sv.add_gauge(g)
    b = syn.gaussian_spinor(dims, 5)
    x = np.empty_like(b)
    try:
        for skip_b in (True, False):
            # the lattice is built, then the spinor b (skip_b) or x fails
            q.debug_inject(q.INJECT_SPINOR_CREATE, 1)
            if not skip_b:
                q.debug_inject(q.INJECT_SPINOR_CREATE, 0)
            r = sv.wait(sv.submit(gid, b, x, 0.13, inner_prec="f16"))
            if skip_b:
                assert r["status"] == 2, r
            r = sv.wait(sv.submit(gid, b, x, 0.13, inner_prec="f16"))
            assert r["status"] == 0 and r["stats"]["true_rel_residual"] <= 1e-10, r
        assert schur_residual_oracle(U, b, x, 0.13, 0.0) <= 1.5e-10
    finally:
        q.debug_inject(q.INJECT_SPINOR_CREATE, 0)
        sv.close()


def test_server_destroy_cancels_queued_requests(q):
    """Destroying a server with requests still queued: threads blocked in
    wait() on queued requests return QCD_ERR_CANCELLED, the running request
    finishes, and destroy returns only after the waiters have left."""
    import threading
    import time
    dims = (32, 32, 32, 8)
    lat, U, g = _server_problem(q, dims, 322)
    sv = q.Server(slots=1, memory_budget=16 << 30)
    gid = sv.add_gauge(g)
    bs = [syn.gaussian_spinor(dims, 10 + k) for k in range(6)]
    xs = [np.empty_like(b) for b in bs]
    # FP64 solves of ~30 ms each on one slot: while the first runs, the rest queue
    ids = [sv.submit(gid, b, x, 0.16, tol=1e-12, inner_prec="f64") for b, x in zip(bs, xs)]
    out = {}

    def waiter(k):
        out[k] = sv.wait(ids[k])

    ths = [threading.Thread(target=waiter, args=(k,)) for k in range(len(ids))]
    for t in ths:
        t.start()
    time.sleep(0.01)  # the waiters block inside wait()
    sv.close()
    for t in ths:
        t.join(timeout=60)
        assert not t.is_alive()
    st = [out[k]["status"] for k in range(len(ids))]
    assert st[0] == 0 and all(v in (0, 7) for v in st) and 7 in st, st


def test_server_concurrent_first_use_of_a_precision(q):
    """Requests on a gauge field with no prepared copies, running at the same
    time on several slots: the copies they need (FP16 links, FP32 links for
    the reliable updates) are built by whichever solve comes first, and no
    other slot may read one before its conversion is complete."""
    dims = (16, 16, 16, 8)
    lat = q.Lattice(dims, -1)
    U = syn.gauge_field(dims, 0.2, 312)
    g = q.Gauge(lat, "f64", 18)
    g.upload(U)
    sv = q.Server(slots=4, memory_budget=8 << 30)
    gid = sv.add_gauge(g)
    jobs = []
    for k in range(8):
        b = syn.gaussian_spinor(dims, 600 + k)
        x = np.empty_like(b)
        jobs.append((sv.submit(gid, b, x, 0.13 + 0.004 * k, inner_prec="f16"), b, x, 0.13 + 0.004 * k))
    for rid, b, x, kappa in jobs:
        r = sv.wait(rid)
        assert r["status"] == 0 and r["stats"]["true_rel_residual"] <= 1e-10, r
    for rid, b, x, kappa in jobs[:2]:
        assert schur_residual_oracle(U, b, x, kappa, 0.0) <= 1.5e-10
    sv.close()


def test_created_fields_are_zeroed_before_other_streams_use_them(q):
    """A new lattice (CG state, reduction counter), gauge field and spinor are
    zeroed before their create call returns.  With the legacy default stream
    held busy by a bounded spin kernel, fields created next and filled on a
    non-blocking stream keep what was uploaded, and a solve on that stream
    over a fresh lattice converges."""
    import torch
    dims = (8, 8, 8, 4)
    U = syn.gauge_field(dims, 0.2, 1401)
    src = syn.gaussian_spinor(dims, 1402)
    side = torch.cuda.Stream()  # created non-blocking: no implicit wait on the legacy stream
    torch.cuda.synchronize()
    with torch.cuda.stream(torch.cuda.default_stream()):
        torch.cuda._sleep(200_000_000)  # ~0.1 s on the legacy default stream
    lat = q.Lattice(dims)
    g = q.Gauge(lat)
    g.upload(U, stream=side)
    b, x = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    b.upload(src, stream=side)
    status, st = q.solve_cg(g, x, b, 0.15, 0.0, tol=1e-10, inner_prec="f16", stream=side)
    torch.cuda.synchronize()
    assert status == 0 and st["true_rel_residual"] <= 1e-10, st
    assert np.array_equal(b.download(), src)
    assert schur_residual_oracle(U, src, x.download(), 0.15, 0.0) <= 1.5e-10


def test_server_overlap_and_memory_budget(q):
    lat, U, g = _server_problem(q, (8, 8, 8, 4), 310)
    lat2, U2, g2 = _server_problem(q, (16, 16, 16, 8), 311)
    # a budget that holds one 16^3x8 context at a time: requests still finish
    one_ctx = 24 * 2 * (16 ** 3 * 8 // 2) * 192
    sv = q.Server(slots=4, memory_budget=one_ctx + 24 * 2 * (8 ** 3 * 4 // 2) * 192)
    gid, gid2 = sv.add_gauge(g), sv.add_gauge(g2)
    jobs = []
    for k in range(12):
        gg, d = (gid, (8, 8, 8, 4)) if k % 2 == 0 else (gid2, (16, 16, 16, 8))
        b = syn.gaussian_spinor(d, 500 + k)
        x = np.empty_like(b)
        jobs.append((sv.submit(gg, b, x, 0.13, inner_prec="f16"), x))
    res = [sv.wait(i) for i, _ in jobs]
    assert all(r["status"] == 0 for r in res)
    assert sv.info()["used_bytes"] <= one_ctx + 24 * 2 * (8 ** 3 * 4 // 2) * 192
    # concurrency, with room for every slot's context (under the tight budget
    # above most requests first rebuild an evicted context, so whether two
    # happen to overlap depends on timing): requests run at the same time
    # on different slots
    roomy = q.Server(slots=4, memory_budget=8 << 30)
    rg, rg2 = roomy.add_gauge(g), roomy.add_gauge(g2)
    rjobs = []
    for k in range(16):
        gg, d = (rg, (8, 8, 8, 4)) if k % 2 == 0 else (rg2, (16, 16, 16, 8))
        b = syn.gaussian_spinor(d, 520 + k)
        x = np.empty_like(b)
        rjobs.append(roomy.submit(gg, b, x, 0.13, inner_prec="f16"))
    rres = [roomy.wait(i) for i in rjobs]
    assert all(r["status"] == 0 for r in rres)
    iv = sorted((r["t_start"], r["t_end"], r["slot"]) for r in rres)
    overlaps = sum(1 for a, b_ in zip(iv, iv[1:]) if b_[0] < a[1] and b_[2] != a[2])
    assert overlaps >= 1
    roomy.close()
    big = q.Server(slots=1, memory_budget=1 << 20)
    gbig = big.add_gauge(g2)
    b = syn.gaussian_spinor((16, 16, 16, 8), 1)
    with pytest.raises(q.QcdError) as e:
        big.submit(gbig, b, np.empty_like(b), 0.13)
    assert e.value.status == 2
    sv.close()
    big.close()


# ------------------------------------------------------- staggered D_KS

def ks_half(chi, parity):
    dims = chi.shape[:4][::-1]
    p = syn.parity_of_sites(dims).reshape(-1)
    return np.ascontiguousarray(chi.reshape(-1, 3)[p == parity])


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64", 12), ("f32", 12), ("f16", 12), ("bf16", 12),
                                        ("f64", 8), ("f32", 8), ("f16", 8), ("bf16", 8)])
def test_dslash_ks_matches_oracle(q, dims, prec, recon):
    lat, U, g = gauge(q, dims, recon=recon)
    lx, ly, lz, lt = dims
    chi = syn.gaussian_complex(60, syn.STREAM_AUX, (lt, lz, ly, lx, 3))
    for out_par in (0, 1):
        src = chi * (syn.parity_of_sites(dims) == 1 - out_par)[..., None]
        want = ks_half(oracle.dks(U, src), out_par)
        si = q.Spinor(lat, "odd" if out_par == 0 else "even", prec, ks=True)
        so = q.Spinor(lat, "even" if out_par == 0 else "odd", prec, ks=True)
        si.upload(ks_half(chi, 1 - out_par))
        q.apply_dslash_ks(g, so, si)
        assert F.rel_err(so.download(), want) <= tol_of(prec), (prec, recon)


def test_dslash_ks_full_point_source_and_roundtrip(q):
    dims = (6, 4, 4, 4)
    lat, U, g = gauge(q, dims)
    chi = np.zeros((4, 4, 4, 6, 3), dtype=complex)
    chi[3, 2, 0, 3, 1] = 1.0
    si, so = q.Spinor(lat, "full", "f64", ks=True), q.Spinor(lat, "full", "f64", ks=True)
    si.upload(chi)
    assert np.array_equal(si.download(), chi)
    q.apply_dslash_ks(g, so, si)
    out = so.download()
    assert len(np.argwhere(np.abs(out).sum(axis=4) > 0)) == 8
    assert F.rel_err(out, oracle.dks(U, chi)) <= 1e-13
    with pytest.raises(q.QcdError):
        q.apply_dslash(g, so, si)  # Wilson operator on staggered fields


# ------------------------------------------------------------ reconstruct-8

@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_dslash_recon8_matches_oracle(q, dims, prec):
    """Pivoted 8-real links on near-identity fields: FP64 rebuilds them to
    the 1e-13 Dslash target, the other formats to their storage tolerance."""
    lat, U, g = gauge(q, dims, recon=8)
    psi = syn.gaussian_spinor(dims, 70)
    for out_parity in (0, 1):
        half_in = syn.to_half(psi, 1 - out_parity)
        for dagger in (False, True):
            want = oracle.dhop_eo(U, half_in, out_parity, dagger=dagger)
            si = q.Spinor(lat, "odd" if out_parity == 0 else "even", prec)
            so = q.Spinor(lat, "even" if out_parity == 0 else "odd", prec)
            si.upload(half_in)
            q.apply_dslash(g, so, si, dagger=dagger)
            err = F.rel_err(so.download(), want)
            assert err <= tol_of(prec), (dims, prec, out_parity, dagger, err)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_recon8_full_and_schur_operators(q, prec):
    dims = (8, 6, 4, 10)
    kappa, mu = 0.16, 0.01
    lat, U, g = gauge(q, dims, recon=8)
    psi = syn.gaussian_spinor(dims, 71)
    si, so = q.Spinor(lat, "full", prec), q.Spinor(lat, "full", prec)
    si.upload(psi)
    q.apply_M(g, so, si, kappa, mu, eo=False)
    assert F.rel_err(so.download(), oracle.apply_m(U, psi, kappa, mu)) <= tol_of(prec)
    xe = syn.to_half(psi, 0)
    ei, eo_ = q.Spinor(lat, "even", prec), q.Spinor(lat, "even", prec)
    ei.upload(xe)
    q.apply_M(g, eo_, ei, kappa, mu, eo=True, dagger=True)
    assert F.rel_err(eo_.download(), oracle.apply_mhat(U, xe, kappa, mu, dagger=True)) <= tol_of(prec)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_recon8_dslash_multi(q, prec):
    dims = (6, 4, 2, 8)
    lat, U, g = gauge(q, dims, recon=8)
    srcs = sources_12_point_4_gauss(dims, 72)
    ins, outs = [], []
    for psi in srcs:
        si = q.Spinor(lat, "odd", prec)
        si.upload(syn.to_half(psi, 1))
        ins.append(si)
        outs.append(q.Spinor(lat, "even", prec))
    q.apply_dslash_multi(g, outs, ins, dagger=True)
    for k, psi in enumerate(srcs):
        want = oracle.dhop_eo(U, syn.to_half(psi, 1), 0, dagger=True)
        if np.any(want):
            assert F.rel_err(outs[k].download(), want) <= tol_of(prec), k


@pytest.mark.parametrize("inner", ["f32", "f16", "bf16"])
def test_solve_inner_recon8(q, inner):
    """Mixed-precision CG with the inner operator on reconstruct-8 links
    (from an FP64 reconstruct-18 field) reaches the FP64 target."""
    dims = (8, 8, 8, 4)
    kappa, mu = 0.16, 0.01
    lat, U, g = gauge(q, dims, eps=0.2, seed=77)
    src = syn.gaussian_spinor(dims, 73)
    b, x = q.Spinor(lat, "full", "f64"), q.Spinor(lat, "full", "f64")
    b.upload(src)
    status, st = q.solve_cg(g, x, b, kappa, mu, tol=1e-10, inner_prec=inner, inner_recon=8)
    assert status == 0 and st["true_rel_residual"] <= 1e-10
    xo, _ = oracle.solve_eo(U, src, kappa, mu, tol=1e-12)
    assert F.rel_err(x.download(), xo) <= 1e-7


def test_recon8_refuses_links_far_from_identity(q):
    """Broad link distributions put the pivot out of its range: the library
    refuses the field instead of storing a lossy one."""
    dims = (4, 4, 4, 4)
    lat = q.Lattice(dims, -1)
    U = syn.gauge_field(dims, 1.5, 1104)
    g16 = q.Gauge(lat, "f16", 8)
    with pytest.raises(q.QcdError) as ei:
        g16.upload(U)
    assert ei.value.status == 1 and "reconstruct-8" in str(ei.value)
    g = q.Gauge(lat, "f64", 18)
    g.upload(U)
    for prec in ("f32", "f16", "bf16"):
        with pytest.raises(q.QcdError):
            g.prepare(prec, 8)
    g.prepare("f64", 8)  # FP64 still rebuilds these to ~6e-14, inside its 1e-13 limit
    g.prepare("f16", 12)  # reconstruct-12 is exact for any SU(3) link
    # near-identity links of the same lattice are accepted in every format
    g8 = q.Gauge(lat, "f64", 18)
    g8.upload(syn.gauge_field(dims, 0.3, 1105))
    for prec in ("f64", "f32", "f16", "bf16"):
        g8.prepare(prec, 8)
    with pytest.raises(q.QcdError):
        g8.prepare("df64", 8)


def test_recon8_profile_counts_eight_reals(q):
    """The profiled algorithmic bytes of a reconstruct-8 launch count 8 reals per link."""
    dims = (8, 8, 8, 8)
    lat, U, g = gauge(q, dims, recon=8, eps=0.2, seed=1106)
    si, so = q.Spinor(lat, "odd", "f16"), q.Spinor(lat, "even", "f16")
    si.upload(syn.to_half(syn.gaussian_spinor(dims, 74), 1))
    q.apply_dslash(g, so, si)
    q.stream_sync()
    q.profile_begin()
    q.apply_dslash(g, so, si)
    pr = q.profile_end()["f16"]
    h = lat.volume // 2
    assert pr["launches"] == 1 and pr["bytes"] == h * (8 * 16 + 2 * 52)

