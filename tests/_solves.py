"""Test-side helpers for solver checks: the even-odd residual recomputed with
the oracle's operators, and the 12 point + 4 Gaussian source set."""

import oracle
from paper_1411_5219_gb300 import synthetic as syn
from tests import _fields as F


def schur_residual_oracle(U, b, x, kappa, mu):
    """|Mhat^dag b' - Mhat^dag Mhat x_e| / |Mhat^dag b'| from oracle operators."""
    be, bo = syn.to_half(b, 0), syn.to_half(b, 1)
    a = 2 * kappa * mu
    bp = be + kappa * oracle.dhop_eo(U, oracle.twist(bo, a, inverse=True), 0)
    rhs = oracle.apply_mhat(U, bp, kappa, mu, dagger=True)
    xe = syn.to_half(x, 0)
    lhs = oracle.apply_mhat(U, oracle.apply_mhat(U, xe, kappa, mu), kappa, mu, dagger=True)
    return F.rel_err(lhs, rhs)


def sources_12_point_4_gauss(dims, seed):
    """One point source at the origin per spin-colour, then four Gaussian ones."""
    srcs = [syn.point_source(dims, s_, c_) for s_ in range(4) for c_ in range(3)]
    srcs += [syn.gaussian_spinor(dims, seed + k) for k in range(4)]
    return srcs
