"""FP64 CPU oracle for the Wilson / twisted-mass Wilson fermion matrix.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code that may import this
package.  It shares no code with the CUDA library.  The arithmetic lives in
``wilson_oracle.c`` (plain C99 complex doubles, one site at a time, OpenMP
over sites, serial reductions); this module builds it with gcc and passes
numpy arrays in the canonical host layouts described in
``paper_1411_5219_gb300.synthetic``.

Paper: CL2QCD, arXiv:1411.5219.  Sec. 1: the fermion matrix is inverted
with CG and its hopping part ("Dslash") dominates; Sec. 3: Wilson and
twisted-mass Wilson fermions; Sec. 4: double precision throughout.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d = ctypes.c_double
        p = ctypes.c_void_p
        i = ctypes.c_int
        lib.oracle_gamma.argtypes = [i, p]
        lib.oracle_dhop.argtypes = [p, d, p, p, p, i]
        lib.oracle_apply_m.argtypes = [p, d, p, d, d, p, p, i]
        lib.oracle_dhop_eo.argtypes = [p, d, p, i, p, p, i]
        lib.oracle_dhop_sites.argtypes = [p, d, p, p, p, ctypes.c_long, p, i]
        lib.oracle_dks.argtypes = [p, d, p, p, p]
        lib.oracle_apply_mhat.argtypes = [p, d, p, d, d, p, p, i]
        lib.oracle_twist.argtypes = [p, p, ctypes.c_long, d, i]
        for f in (lib.oracle_solve_mdagm, lib.oracle_solve_m, lib.oracle_solve_eo):
            f.argtypes = [p, d, p, d, d, p, p, d, i, p]
        lib.oracle_cg_eo_sample.argtypes = [p, d, p, d, d, p, p, i]
        lib.oracle_set_threads.argtypes = [i]
        lib.oracle_get_threads.restype = i
        _lib = lib
    return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dims(U):
    lt, lz, ly, lx = U.shape[:4]
    return (ctypes.c_int * 4)(lx, ly, lz, lt)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def gamma(mu: int) -> np.ndarray:
    """gamma_mu for mu = 0..3 (x, y, z, t) and gamma_5 for mu = 4 (chiral basis)."""
    out = np.zeros((4, 4), dtype=np.complex128)
    _load().oracle_gamma(int(mu), out.ctypes.data_as(ctypes.c_void_p))
    return out


def dhop(U, psi, t_bc=-1.0, dagger=False):
    """D_hop psi (or D_hop^dagger psi) on the full lattice."""
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    _load().oracle_dhop(_dims(U), float(t_bc), pu, pp, out.ctypes.data_as(ctypes.c_void_p), int(dagger))
    return out


def apply_m(U, psi, kappa, mu=0.0, t_bc=-1.0, dagger=False):
    """M psi = (1 + 2 i kappa mu gamma_5) psi - kappa D_hop psi (or M^dagger psi)."""
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    _load().oracle_apply_m(_dims(U), float(t_bc), pu, float(kappa), float(mu), pp,
                           out.ctypes.data_as(ctypes.c_void_p), int(dagger))
    return out


def dks(U, chi, t_bc=-1.0):
    """Staggered derivative D_KS chi on the full lattice; chi[t,z,y,x,3] complex."""
    U, pu = _c(U)
    chi, pc = _c(chi)
    out = np.empty_like(chi)
    _load().oracle_dks(_dims(U), float(t_bc), pu, pc, out.ctypes.data_as(ctypes.c_void_p))
    return out


def dhop_sites(U, psi, sites, t_bc=-1.0, dagger=False):
    """D_hop psi (or D_hop^dagger psi) at the given lexicographic sites only."""
    U, pu = _c(U)
    psi, pp = _c(psi)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    _load().oracle_dhop_sites(_dims(U), float(t_bc), pu, pp, sites.ctypes.data_as(ctypes.c_void_p), len(sites),
                              out.ctypes.data_as(ctypes.c_void_p), int(dagger))
    return out


def dhop_eo(U, half_in, out_parity, t_bc=-1.0, dagger=False):
    """Parity block of D_hop: D_eo (out_parity 0) or D_oe (out_parity 1) on half fields."""
    U, pu = _c(U)
    half_in, ph = _c(half_in)
    out = np.empty_like(half_in)
    _load().oracle_dhop_eo(_dims(U), float(t_bc), pu, int(out_parity), ph,
                           out.ctypes.data_as(ctypes.c_void_p), int(dagger))
    return out


def apply_mhat(U, x_even, kappa, mu=0.0, t_bc=-1.0, dagger=False):
    """Schur complement Mhat = A - kappa^2 D_eo A^-1 D_oe (or Mhat^dagger) on even half fields."""
    U, pu = _c(U)
    x_even, px = _c(x_even)
    out = np.empty_like(x_even)
    _load().oracle_apply_mhat(_dims(U), float(t_bc), pu, float(kappa), float(mu), px,
                              out.ctypes.data_as(ctypes.c_void_p), int(dagger))
    return out


def twist(psi, b, inverse=False):
    """(1 + i b gamma_5) psi, or (1 - i b gamma_5) psi / (1 + b^2) with inverse."""
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    _load().oracle_twist(pp, out.ctypes.data_as(ctypes.c_void_p), psi.size // 12, float(b), int(inverse))
    return out


def _solve(fn, U, b, kappa, mu, t_bc, tol, maxiter, nstats):
    U, pu = _c(U)
    b, pb = _c(b)
    x = np.zeros_like(b)
    st = np.zeros(3)
    fn(_dims(U), float(t_bc), pu, float(kappa), float(mu), pb, x.ctypes.data_as(ctypes.c_void_p),
       float(tol), int(maxiter), st.ctypes.data_as(ctypes.c_void_p))
    return x, st[:nstats]


def solve_mdagm(U, b, kappa, mu=0.0, t_bc=-1.0, tol=1e-12, maxiter=100000):
    """x with M^dagger M x = b (CG); stats = (iterations, |b - M^dag M x|/|b|)."""
    return _solve(_load().oracle_solve_mdagm, U, b, kappa, mu, t_bc, tol, maxiter, 2)


def solve_m(U, b, kappa, mu=0.0, t_bc=-1.0, tol=1e-12, maxiter=100000):
    """x with M x = b by CG on the normal equations; stats = (iterations, |b - M x|/|b|)."""
    return _solve(_load().oracle_solve_m, U, b, kappa, mu, t_bc, tol, maxiter, 2)


def solve_eo(U, b, kappa, mu=0.0, t_bc=-1.0, tol=1e-12, maxiter=100000):
    """x with M x = b through the even-odd Schur complement and CG.

    stats = (iterations, Schur-system relative residual, |b - M x|/|b|).
    """
    return _solve(_load().oracle_solve_eo, U, b, kappa, mu, t_bc, tol, maxiter, 3)


def cg_eo_sample(U, b_even, kappa, mu=0.0, t_bc=-1.0, iters=10):
    """Run a fixed number of even-odd CG iterations (a timing sample)."""
    U, pu = _c(U)
    b_even, pb = _c(b_even)
    x = np.zeros_like(b_even)
    _load().oracle_cg_eo_sample(_dims(U), float(t_bc), pu, float(kappa), float(mu), pb,
                                x.ctypes.data_as(ctypes.c_void_p), int(iters))
    return x
