"""Pins of the oracle's staggered derivative D_KS (the paper's second
operator, Sec. 1 and Sec. 6) against facts that do not come from the oracle:
the free-field square D^2 = -4 sum_mu sin^2 p_mu on plane waves (which holds
only if the staggered phases anticommute like gamma matrices), the dense
free spectrum, anti-hermiticity, gauge covariance, the even-odd block
structure and the support of a point source."""

import itertools

import numpy as np
import pytest

import oracle
from paper_1411_5219_gb300 import synthetic as syn
from tests import _fields as F


def plane_wave_ks(dims, p, chi):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None] * chi[None, None, None, None]


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (2, 2, 2, 2)])
@pytest.mark.parametrize("t_bc", [-1.0, 1.0])
def test_free_field_square(dims, t_bc):
    lx, ly, lz, lt = dims
    U = syn.unit_gauge_field(dims)
    chi = syn.gaussian_complex(3, syn.STREAM_AUX, (3,))
    shift = np.pi / lt if t_bc < 0 else 0.0
    for n in [(0, 0, 0, 0), (1, 0, 1, 1), (lx - 1, 1, 0, lt - 1)]:
        p = (2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz, 2 * np.pi * n[3] / lt + shift)
        psi = plane_wave_ks(dims, p, chi)
        got = oracle.dks(U, oracle.dks(U, psi, t_bc), t_bc)
        want = -4 * sum(np.sin(v) ** 2 for v in p) * psi
        assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(psi)


def test_free_spectrum_dense():
    dims = (4, 2, 2, 4)
    U = syn.unit_gauge_field(dims)
    V = syn.volume(dims)
    shape = (4, 2, 2, 4, 3)
    cols = []
    for j in range(V * 3):
        e = np.zeros(V * 3, dtype=complex)
        e[j] = 1
        cols.append(oracle.dks(U, e.reshape(shape)).reshape(-1))
    D = np.stack(cols, axis=1)
    assert np.abs(D + D.conj().T).max() < 1e-15  # anti-Hermitian
    ev = np.sort(np.linalg.eigvalsh(-(D @ D)).real)
    want = []
    for nx, ny, nz, nt in itertools.product(range(4), range(2), range(2), range(4)):
        p = [2 * np.pi * nx / 4, 2 * np.pi * ny / 2, 2 * np.pi * nz / 2, (2 * nt + 1) * np.pi / 4]
        want += [4 * sum(np.sin(v) ** 2 for v in p)] * 3
    np.testing.assert_allclose(ev, np.sort(want), atol=1e-12)


def test_antihermitian_and_eo_structure():
    dims = (4, 4, 2, 6)
    U = syn.gauge_field(dims, 0.3, 7)
    x = syn.gaussian_complex(1, syn.STREAM_AUX, (6, 2, 4, 4, 3))
    y = syn.gaussian_complex(2, syn.STREAM_AUX, (6, 2, 4, 4, 3))
    lhs = F.vdot(x, oracle.dks(U, y))
    rhs = -F.vdot(oracle.dks(U, x), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    par = syn.parity_of_sites(dims)
    ye = y * (par == 0)[..., None]
    out = oracle.dks(U, ye)
    assert np.all(out[par == 0] == 0)  # an even field only feeds odd sites


def test_gauge_covariance():
    dims = (4, 6, 2, 4)
    U = syn.gauge_field(dims, 0.3, 8)
    W = syn.gauge_transform(dims, 9)
    Up = np.empty_like(U)
    for mu in range(4):
        Wf = np.roll(W, -1, axis=F.AXIS_OF_MU[mu])
        Up[..., mu, :, :] = W @ U[..., mu, :, :] @ np.conj(np.swapaxes(Wf, -1, -2))
    chi = syn.gaussian_complex(3, syn.STREAM_AUX, (4, 2, 6, 4, 3))
    got = oracle.dks(Up, np.einsum("...ab,...b->...a", W, chi))
    want = np.einsum("...ab,...b->...a", W, oracle.dks(U, chi))
    assert F.rel_err(got, want) < 1e-14


def test_point_source_support_and_phases():
    dims = (4, 4, 4, 4)
    U = syn.unit_gauge_field(dims)
    chi = np.zeros((4, 4, 4, 4, 3), dtype=complex)
    chi[0, 0, 0, 1, 2] = 1.0  # site x=1, y=z=t=0, colour 2
    out = oracle.dks(U, chi)
    nz = {tuple(v) for v in np.argwhere(np.abs(out).sum(axis=4) > 0)}
    assert len(nz) == 8
    # hop from the site at x = 0 reaches it forward with eta_x = +1
    assert out[0, 0, 0, 0, 2] == 1.0
    # the site at x = 1, y = 1 reaches it backward in y with eta_y(x=1, y=1) = -1: -(-1) = +1
    assert out[0, 0, 1, 1, 2] == 1.0
    # and at x = 1, y = 3 forward in y (wrap): eta_y = -1
    assert out[0, 0, 3, 1, 2] == -1.0
