"""Test-side helpers: layouts, inner products and an independent gamma basis.

Nothing here computes the Dirac operator; the gamma matrices are typed in
again from their textbook definition (chiral basis) so that the oracle's own
table is checked against them, not against itself.
"""

import numpy as np

from paper_1411_5219_gb300 import synthetic as syn

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=complex),
    np.array([[0, -1j], [1j, 0]], dtype=complex),
    np.array([[1, 0], [0, -1]], dtype=complex),
]


def textbook_gammas():
    """Chiral-basis gamma_1..4 and gamma_5 built from Pauli matrices."""
    z = np.zeros((2, 2), dtype=complex)
    one = np.eye(2, dtype=complex)
    g = [np.block([[z, -1j * s], [1j * s, z]]) for s in SIGMA]
    g.append(np.block([[z, one], [one, z]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


def vdot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def rel_err(a, b):
    return np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1))


def apply_spin(mat, psi):
    """Multiply every site's spinor by a 4x4 spin matrix."""
    return np.einsum("st,...tc->...sc", mat, psi)


def apply_colour_site(omega, psi):
    """psi'(x) = Omega(x) psi(x) for Omega[t,z,y,x,3,3]."""
    return np.einsum("...ab,...sb->...sa", omega, psi)


AXIS_OF_MU = {0: 3, 1: 2, 2: 1, 3: 0}  # array axes are [t, z, y, x]


def plane_wave(dims, p, chi):
    """psi(x) = exp(i p.x) chi with p = (px, py, pz, pt)."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None, None] * chi[None, None, None, None]


def dense_operator(apply, n_sites, shape):
    """Dense matrix of a linear map on fields of `shape` (n_sites*12 columns)."""
    n = n_sites * 12
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1.0
        cols.append(apply(e.reshape(shape)).reshape(-1))
    return np.stack(cols, axis=1)


def parity_mask(dims):
    return syn.parity_of_sites(dims).reshape(-1)
