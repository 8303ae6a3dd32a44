"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test states what fixes the expected value: an algebraic identity, a
closed form of the free-field operator, a property of the exact operator
(gamma_5-hermiticity, gauge covariance), a dense linear-algebra routine
from numpy, or an FFT solution.  The paper (CL2QCD, arXiv:1411.5219)
prints no worked example; Sec. 5 asks for tests against analytic results
whose dependence on the lattice size is predictable, over varied lattice
sizes and parameters, and without environment-dependent random numbers.
"""

import itertools

import numpy as np
import pytest

import oracle
from paper_1411_5219_gb300 import synthetic as syn
from tests import _fields as F


# ---------------------------------------------------------------- gamma basis

def test_gamma_basis_matches_textbook_and_clifford():
    g, g5 = F.textbook_gammas()
    for mu in range(4):
        np.testing.assert_allclose(oracle.gamma(mu), g[mu], atol=0)
    np.testing.assert_allclose(oracle.gamma(4), g5, atol=1e-15)
    np.testing.assert_allclose(oracle.gamma(4), np.diag([1, 1, -1, -1]), atol=1e-15)
    for mu, nu in itertools.product(range(4), repeat=2):
        a, b = oracle.gamma(mu), oracle.gamma(nu)
        np.testing.assert_allclose(a @ b + b @ a, 2 * np.eye(4) * (mu == nu), atol=1e-15)
    for mu in range(4):
        a = oracle.gamma(mu)
        np.testing.assert_allclose(a, a.conj().T, atol=0)
        np.testing.assert_allclose(a @ oracle.gamma(4) + oracle.gamma(4) @ a, 0, atol=1e-15)


# ------------------------------------------------------- free-field closed form

def free_field_symbol(p, kappa, mu_tm):
    """M(p) = (1 - 2k sum cos p) + 2ik sum gamma_mu sin p_mu + i a gamma_5."""
    g, g5 = F.textbook_gammas()
    a = 2 * kappa * mu_tm
    m = (1 - 2 * kappa * sum(np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        m = m + 2j * kappa * np.sin(p[mu]) * g[mu]
    return m + 1j * a * g5


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (2, 2, 2, 2)])
@pytest.mark.parametrize("kappa,mu_tm", [(0.15, 0.0), (0.16, 0.01), (0.12, 0.5)])
def test_free_field_plane_wave_eigenrelation(dims, kappa, mu_tm):
    """At U = 1, M exp(ipx) chi = exp(ipx) M(p) chi for lattice momenta.

    Antiperiodic time makes p_t = (2n+1) pi / L_t.  This single identity
    fixes the hop sign, the kappa normalisation, the boundary conditions,
    the gamma basis and the twisted-mass term."""
    lx, ly, lz, lt = dims
    U = syn.unit_gauge_field(dims)
    rng_chi = syn.gaussian_complex(7, syn.STREAM_AUX, (4, 3))
    for n in [(0, 0, 0, 0), (1, 0, 0, 1), (1, 1, 1, 0), (lx - 1, 1, 0, lt - 1)]:
        p = (2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
             (2 * n[3] + 1) * np.pi / lt)
        psi = F.plane_wave(dims, p, rng_chi)
        got = oracle.apply_m(U, psi, kappa, mu_tm, t_bc=-1.0)
        want = F.plane_wave(dims, p, free_field_symbol(p, kappa, mu_tm) @ rng_chi)
        assert F.rel_err(got, want) < 1e-14


def test_free_field_periodic_time_and_hop_term():
    dims = (4, 2, 4, 6)
    U = syn.unit_gauge_field(dims)
    chi = syn.gaussian_complex(8, syn.STREAM_AUX, (4, 3))
    g, _ = F.textbook_gammas()
    p = (np.pi / 2, np.pi, -np.pi / 2, 2 * np.pi / 6)
    psi = F.plane_wave(dims, p, chi)
    got = oracle.dhop(U, psi, t_bc=+1.0)
    sym = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * g[m] for m in range(4))
    assert F.rel_err(got, F.plane_wave(dims, p, sym @ chi)) < 1e-14


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4), (6, 4, 4, 2)])
@pytest.mark.parametrize("kappa,mu_tm", [(0.125, 0.0), (0.16, 0.01)])
def test_constant_field_lattice_size_predictable(dims, kappa, mu_tm):
    """Periodic BCs, U = 1, constant c: M c = (1 - 8 kappa) c + i a gamma_5 c,
    so |M c|^2 = V ((1 - 8 kappa)^2 + a^2) |c|^2 for every volume V."""
    U = syn.unit_gauge_field(dims)
    c = syn.gaussian_complex(9, syn.STREAM_AUX, (4, 3))
    psi = np.broadcast_to(c, (dims[3], dims[2], dims[1], dims[0], 4, 3)).copy()
    got = oracle.apply_m(U, psi, kappa, mu_tm, t_bc=+1.0)
    a = 2 * kappa * mu_tm
    _, g5 = F.textbook_gammas()
    want = (1 - 8 * kappa) * psi + 1j * a * F.apply_spin(g5, psi)
    # kappa = 1/8 is the free critical point: M c = i a gamma_5 c (zero for Wilson)
    assert np.linalg.norm(got - want) < 1e-14 * np.linalg.norm(psi)
    V = syn.volume(dims)
    np.testing.assert_allclose(np.linalg.norm(got) ** 2,
                               V * ((1 - 8 * kappa) ** 2 + a * a) * np.linalg.norm(c) ** 2,
                               rtol=1e-13, atol=1e-26 * V)


def free_field_eigenvalues(dims, kappa, mu_tm):
    """Eigenvalues of M^dag M at U = 1 with antiperiodic t: the scalar
    (1 - 2k sum cos p)^2 + 4k^2 sum sin^2 p + a^2, 12-fold per momentum."""
    lx, ly, lz, lt = dims
    a = 2 * kappa * mu_tm
    vals = []
    for nx, ny, nz, nt in itertools.product(range(lx), range(ly), range(lz), range(lt)):
        p = np.array([2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz, (2 * nt + 1) * np.pi / lt])
        lam = (1 - 2 * kappa * np.cos(p).sum()) ** 2 + 4 * kappa ** 2 * (np.sin(p) ** 2).sum() + a * a
        vals += [lam] * 12
    return np.sort(vals)


@pytest.mark.parametrize("dims,kappa,mu_tm", [((2, 2, 2, 2), 0.15, 0.0), ((4, 2, 2, 4), 0.16, 0.01)])
def test_free_field_spectrum_dense(dims, kappa, mu_tm):
    U = syn.unit_gauge_field(dims)
    shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    M = F.dense_operator(lambda v: oracle.apply_m(U, v, kappa, mu_tm), syn.volume(dims), shape)
    ev = np.sort(np.linalg.eigvalsh(M.conj().T @ M))
    np.testing.assert_allclose(ev, free_field_eigenvalues(dims, kappa, mu_tm), rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------- exact symmetries

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
@pytest.mark.parametrize("mu_tm", [0.0, 0.01])
def test_gamma5_hermiticity_and_adjoint(dims, mu_tm):
    """<x, M(mu) y> = <gamma5 M(-mu) gamma5 x, y> = <M^dag x, y>."""
    kappa = 0.15
    U = syn.gauge_field(dims, 0.3, 1001)
    x = syn.gaussian_spinor(dims, 11)
    y = syn.gaussian_spinor(dims, 12)
    _, g5 = F.textbook_gammas()
    lhs = F.vdot(x, oracle.apply_m(U, y, kappa, mu_tm))
    g5x = F.apply_spin(g5, x)
    rhs = F.vdot(F.apply_spin(g5, oracle.apply_m(U, g5x, kappa, -mu_tm)), y)
    rhs2 = F.vdot(oracle.apply_m(U, x, kappa, mu_tm, dagger=True), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert abs(lhs - rhs2) < 1e-12 * abs(lhs)


def test_eo_blocks_adjoint_relation():
    """<x_e, D_eo y_o> = <gamma5 D_oe gamma5 x_e, y_o> and the dagger flag
    gives the adjoint block."""
    dims = (4, 4, 2, 4)
    U = syn.gauge_field(dims, 0.3, 5)
    xe = syn.to_half(syn.gaussian_spinor(dims, 1), 0)
    yo = syn.to_half(syn.gaussian_spinor(dims, 2), 1)
    _, g5 = F.textbook_gammas()
    lhs = F.vdot(xe, oracle.dhop_eo(U, yo, 0))
    rhs = F.vdot(F.apply_spin(g5, oracle.dhop_eo(U, F.apply_spin(g5, xe), 1)), yo)
    rhs2 = F.vdot(oracle.dhop_eo(U, xe, 1, dagger=True), yo)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert abs(lhs - rhs2) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("t_bc", [-1.0, 1.0])
def test_gauge_covariance(t_bc):
    """U'_mu(x) = W(x) U_mu(x) W(x+mu)^dag, psi' = W psi:
    D[U'] psi' = W D[U] psi for a random SU(3) field W."""
    dims = (4, 6, 2, 4)
    U = syn.gauge_field(dims, 0.3, 21)
    W = syn.gauge_transform(dims, 22)
    Up = np.empty_like(U)
    for mu in range(4):
        Wf = np.roll(W, -1, axis=F.AXIS_OF_MU[mu])
        Up[..., mu, :, :] = W @ U[..., mu, :, :] @ np.conj(np.swapaxes(Wf, -1, -2))
    psi = syn.gaussian_spinor(dims, 23)
    got = oracle.dhop(Up, F.apply_colour_site(W, psi), t_bc=t_bc)
    want = F.apply_colour_site(W, oracle.dhop(U, psi, t_bc=t_bc))
    assert F.rel_err(got, want) < 1e-14


def test_point_source_support_is_eight_neighbours():
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, 0.3, 3)
    src = syn.point_source(dims, 2, 1, site=(1, 2, 3, 0))
    out = oracle.dhop(U, src)
    nz = np.argwhere(np.abs(out).sum(axis=(4, 5)) > 0)
    want = set()
    for mu in range(4):
        for d in (1, -1):
            c = [1, 2, 3, 0]
            c[mu] = (c[mu] + d) % dims[mu]
            want.add((c[3], c[2], c[1], c[0]))
    assert {tuple(v) for v in nz} == want


# ------------------------------------------------------- dense brute force 2^4

@pytest.fixture(scope="module")
def dense_2x4():
    dims = (2, 2, 2, 2)
    kappa, mu_tm = 0.15, 0.02
    U = syn.gauge_field(dims, 0.3, 1001)
    shape = (2, 2, 2, 2, 4, 3)
    V = syn.volume(dims)
    M = F.dense_operator(lambda v: oracle.apply_m(U, v, kappa, mu_tm), V, shape)
    Md = F.dense_operator(lambda v: oracle.apply_m(U, v, kappa, mu_tm, dagger=True), V, shape)
    return dims, kappa, mu_tm, U, M, Md


def test_dense_dagger_is_conjugate_transpose(dense_2x4):
    _, _, _, _, M, Md = dense_2x4
    np.testing.assert_allclose(Md, M.conj().T, atol=1e-15)


def test_dense_solves_match_lu(dense_2x4):
    dims, kappa, mu_tm, U, M, _ = dense_2x4
    b = syn.gaussian_spinor(dims, 31)
    want = np.linalg.solve(M, b.reshape(-1))
    for solver in (oracle.solve_m, oracle.solve_eo):
        x, st = solver(U, b, kappa, mu_tm, tol=1e-13)
        assert st[0] > 0
        assert F.rel_err(x.reshape(-1), want) < 1e-11
    want_n = np.linalg.solve(M.conj().T @ M, b.reshape(-1))
    x, st = oracle.solve_mdagm(U, b, kappa, mu_tm, tol=1e-13)
    assert F.rel_err(x.reshape(-1), want_n) < 1e-11
    assert st[1] < 1e-12


def test_schur_complement_matches_dense_blocks(dense_2x4):
    """Mhat = M_ee - M_eo M_oo^-1 M_oe, the blocks cut from the dense M."""
    dims, kappa, mu_tm, U, M, _ = dense_2x4
    par = np.repeat(F.parity_mask(dims), 12)
    e, o = par == 0, par == 1
    S = M[np.ix_(e, e)] - M[np.ix_(e, o)] @ np.linalg.solve(M[np.ix_(o, o)], M[np.ix_(o, e)])
    xe = syn.to_half(syn.gaussian_spinor(dims, 32), 0)
    got = oracle.apply_mhat(U, xe, kappa, mu_tm)
    assert F.rel_err(got.reshape(-1), S @ xe.reshape(-1)) < 1e-13
    got_d = oracle.apply_mhat(U, xe, kappa, mu_tm, dagger=True)
    assert F.rel_err(got_d.reshape(-1), S.conj().T @ xe.reshape(-1)) < 1e-13
    # the hopping blocks themselves
    Deo = -M[np.ix_(e, o)] / kappa
    yo = syn.to_half(syn.gaussian_spinor(dims, 33), 1)
    assert F.rel_err(oracle.dhop_eo(U, yo, 0).reshape(-1), Deo @ yo.reshape(-1)) < 1e-14


def test_twist_inverse():
    psi = syn.gaussian_spinor((2, 2, 2, 2), 40)
    b = 0.37
    back = oracle.twist(oracle.twist(psi, b), b, inverse=True)
    assert F.rel_err(back, psi) < 1e-15
    _, g5 = F.textbook_gammas()
    assert F.rel_err(oracle.twist(psi, b), psi + 1j * b * F.apply_spin(g5, psi)) < 1e-15


# ------------------------------------------------------------------ solvers

def fft_solve_free_mdagm(b, kappa, mu_tm):
    """Exact x of M^dag M x = b at U = 1, antiperiodic t, by FFT: the
    operator is the scalar lambda(p) in momentum space."""
    lt, lz, ly, lx = b.shape[:4]
    t = np.arange(lt)[:, None, None, None, None, None]
    phase = np.exp(1j * np.pi * t / lt)
    bh = np.fft.fftn(b / phase, axes=(0, 1, 2, 3))
    pt = 2 * np.pi * np.fft.fftfreq(lt) * 1 + np.pi / lt
    pz = 2 * np.pi * np.fft.fftfreq(lz)
    py = 2 * np.pi * np.fft.fftfreq(ly)
    px = 2 * np.pi * np.fft.fftfreq(lx)
    PT, PZ, PY, PX = np.meshgrid(pt, pz, py, px, indexing="ij")
    a = 2 * kappa * mu_tm
    cs = np.cos(PX) + np.cos(PY) + np.cos(PZ) + np.cos(PT)
    s2 = np.sin(PX) ** 2 + np.sin(PY) ** 2 + np.sin(PZ) ** 2 + np.sin(PT) ** 2
    lam = (1 - 2 * kappa * cs) ** 2 + 4 * kappa ** 2 * s2 + a * a
    return phase * np.fft.ifftn(bh / lam[..., None, None], axes=(0, 1, 2, 3))


@pytest.mark.parametrize("mu_tm", [0.0, 0.01])
def test_cg_free_field_matches_fft(mu_tm):
    dims, kappa = (4, 4, 4, 4), 0.15
    U = syn.unit_gauge_field(dims)
    b = syn.gaussian_spinor(dims, 1001)
    x, st = oracle.solve_mdagm(U, b, kappa, mu_tm, tol=1e-12)
    assert st[0] > 0 and st[1] <= 1e-12
    assert F.rel_err(x, fft_solve_free_mdagm(b, kappa, mu_tm)) < 1e-10


def test_eo_solve_equals_full_solve():
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, 0.3, 1001)
    b = syn.gaussian_spinor(dims, 50)
    for kappa, mu_tm in [(0.15, 0.0), (0.16, 0.01)]:
        xf, sf = oracle.solve_m(U, b, kappa, mu_tm, tol=1e-12)
        xe, se = oracle.solve_eo(U, b, kappa, mu_tm, tol=1e-12)
        assert sf[1] < 1e-11 and se[1] <= 1e-12 and se[2] < 1e-11
        assert F.rel_err(xe, xf) < 1e-10
        assert F.rel_err(oracle.apply_m(U, xe, kappa, mu_tm), b) < 1e-11


def test_solver_zero_source_and_maxiter():
    dims = (2, 2, 2, 2)
    U = syn.gauge_field(dims, 0.3, 1)
    b = np.zeros((2, 2, 2, 2, 4, 3), dtype=complex)
    x, st = oracle.solve_eo(U, b, 0.15)
    assert np.all(x == 0)
    b = syn.gaussian_spinor(dims, 2)
    x, st = oracle.solve_mdagm(U, b, 0.15, maxiter=2, tol=1e-14)
    assert st[0] == -1


# ------------------------------------------------------ synthetic input checks

def test_synthetic_links_are_su3_and_deterministic():
    U1 = syn.gauge_field((4, 2, 2, 4), 0.3, 1001)
    U2 = syn.gauge_field((4, 2, 2, 4), 0.3, 1001)
    assert np.array_equal(U1, U2)
    u = U1.reshape(-1, 3, 3)
    assert np.abs(np.conj(np.swapaxes(u, 1, 2)) @ u - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-14
    # near-unit: |U - 1| of order eps
    assert 0.05 < np.abs(u - np.eye(3)).mean() < 0.3


def test_splitmix64_matches_its_published_sequence():
    """The generator behind every synthetic input is SplitMix64 (Steele, Lea
    and Flood, OOPSLA 2014).  Started from state 0, the reference generator
    (state += 0x9E3779B97F4A7C15, then the output mix) yields this sequence."""
    gamma = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        states = np.array([0, gamma, np.uint64(2) * gamma], dtype=np.uint64)
    got = [int(v) for v in syn._splitmix64(states)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_normal_draws():
    """Uniforms lie in the open interval (0, 1); the Box-Muller normals have
    mean 0 and variance 1 within their sampling error, and any slice of the
    sequence is drawn on its own."""
    u = syn.uniform(7, syn.STREAM_AUX, np.arange(1 << 16, dtype=np.uint64))
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    z = syn.normal(7, syn.STREAM_AUX, 0, 1 << 18)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2 / z.size)
    assert abs((z ** 4).mean() - 3.0) < 0.1  # Gaussian fourth moment
    assert np.array_equal(syn.normal(7, syn.STREAM_AUX, 1000, 24), z[1000:1024])
