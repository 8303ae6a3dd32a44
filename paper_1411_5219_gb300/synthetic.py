"""Seeded synthetic inputs: gauge links, sources and gauge transformations.

This module is shared by the CPU oracle side (tests, CPU baseline) and the
GPU side (tests, bench).  It holds none of the Dirac-operator arithmetic:
it only draws random numbers and builds SU(3) matrices and spinor fields in
the canonical host layouts that both sides accept.

Canonical host layouts (complex128, C order):

* gauge field  ``U[t, z, y, x, mu, a, b]`` with ``mu = 0, 1, 2, 3`` for the
  x, y, z, t directions and ``U_mu(x)[a, b]`` the colour matrix of the link
  from site x to site x + mu_hat;
* spinor field ``psi[t, z, y, x, s, c]`` with spin ``s`` (0..3) and colour
  ``c`` (0..2);
* parity-compacted half field ``psi_half[i, s, c]`` holding the sites of one
  parity p = (x + y + z + t) mod 2 in lexicographic order, i = lex // 2 with
  lex = x + Lx*(y + Ly*(z + Lz*t)) (valid because Lx is even).

Random numbers come from a counter-based generator so that every value
depends only on (seed, stream, counter), never on thread count or hardware
(the paper asks for environment-independent tests, Sec. 5).  The generator
is SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to a nested key, followed by Box-Muller.
"""

from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)

# Stream identifiers: one per kind of random field.
STREAM_GAUGE = 1
STREAM_SOURCE = 2
STREAM_GAUGE_TRANSFORM = 3
STREAM_AUX = 4


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 values."""
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def random_u64(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Return one 64-bit random word per counter for (seed, stream)."""
    key = _splitmix64(np.array([seed], dtype=np.uint64))
    key = _splitmix64(key ^ np.uint64(stream))
    return _splitmix64(key ^ np.asarray(counters, dtype=np.uint64))


def uniform(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1), one per counter."""
    bits = random_u64(seed, stream, counters) >> np.uint64(11)
    return (bits.astype(np.float64) + 0.5) * (2.0 ** -53)


def normal(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """n standard normal doubles for counters start .. start+n-1 (Box-Muller).

    Normal k uses the uniforms with counters 2*(start+k) and 2*(start+k)+1,
    so any slice of the sequence can be drawn on its own.
    """
    k = np.arange(start, start + n, dtype=np.uint64)
    u1 = uniform(seed, stream, np.uint64(2) * k)
    u2 = uniform(seed, stream, np.uint64(2) * k + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def check_dims(dims) -> tuple:
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4 or any(d < 2 or d % 2 for d in dims):
        raise ValueError(f"lattice extents must be four even numbers >= 2, got {dims}")
    return dims


def gaussian_complex(seed: int, stream: int, shape, start: int = 0) -> np.ndarray:
    """Complex array with independent N(0,1) real and imaginary parts."""
    n = int(np.prod(shape))
    g = normal(seed, stream, 2 * start, 2 * n)
    return (g[0::2] + 1j * g[1::2]).reshape(shape)


def su3_near_unit(seed: int, stream: int, n: int, eps: float, chunk: int = 1 << 18, device=None) -> np.ndarray:
    """n SU(3) matrices U = exp(i*eps*H), H Hermitian traceless, Gaussian.

    For matrix j, a 3x3 complex Gaussian A (counters 9j .. 9j+8 of the
    complex sequence) gives H = (A + A^dagger)/2 - tr(.)/3.  The exponential
    is taken through the Hermitian eigendecomposition H = V diag(l) V^dagger,
    U = V diag(exp(i eps l)) V^dagger, so U is unitary and det U =
    exp(i eps tr H) = 1.
    """
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        a = gaussian_complex(seed, stream, (m, 3, 3), start=9 * s)
        h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
        tr = np.trace(h, axis1=1, axis2=2).real / 3.0
        h = h - tr[:, None, None] * np.eye(3)
        if device is None:
            lam, v = np.linalg.eigh(h)
            ph = np.exp(1j * eps * lam)
            out[s:s + m] = np.einsum("nab,nb,ncb->nac", v, ph, np.conj(v))
        else:  # the same Gaussian draws, exp(i eps H) by torch's matrix exponential on a device
            import torch
            ht = torch.from_numpy(h).to(device)
            out[s:s + m] = torch.linalg.matrix_exp(1j * eps * ht).cpu().numpy()
    return out


def gauge_field(dims, eps: float, seed: int, device=None) -> np.ndarray:
    """Near-unit random gauge field U[t,z,y,x,mu,3,3], one draw per (site, mu).

    device: None for numpy, or a torch device on which exp(i eps H) of the
    same draws is taken by matrix exponential (faster for large lattices; the
    links agree with the numpy ones to rounding)."""
    lx, ly, lz, lt = check_dims(dims)
    v = volume(dims)
    u = su3_near_unit(seed, STREAM_GAUGE, 4 * v, eps, device=device)
    return u.reshape(lt, lz, ly, lx, 4, 3, 3)


def unit_gauge_field(dims) -> np.ndarray:
    lx, ly, lz, lt = check_dims(dims)
    u = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gauge_transform(dims, seed: int, eps: float = 3.0) -> np.ndarray:
    """Random SU(3) matrix per site, Omega[t,z,y,x,3,3] (far from unit)."""
    lx, ly, lz, lt = check_dims(dims)
    return su3_near_unit(seed, STREAM_GAUGE_TRANSFORM, volume(dims), eps).reshape(lt, lz, ly, lx, 3, 3)


def gaussian_spinor(dims, seed: int, stream: int = STREAM_SOURCE) -> np.ndarray:
    """Gaussian complex source psi[t,z,y,x,4,3]."""
    lx, ly, lz, lt = check_dims(dims)
    return gaussian_complex(seed, stream, (lt, lz, ly, lx, 4, 3))


def point_source(dims, spin: int, colour: int, site=(0, 0, 0, 0)) -> np.ndarray:
    """Unit point source at site (x, y, z, t) in spin-colour component (s, c)."""
    lx, ly, lz, lt = check_dims(dims)
    psi = np.zeros((lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    x, y, z, t = site
    psi[t, z, y, x, spin, colour] = 1.0
    return psi


def parity_of_sites(dims) -> np.ndarray:
    """Array p[t,z,y,x] = (x+y+z+t) mod 2."""
    lx, ly, lz, lt = check_dims(dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return (x + y + z + t) % 2


def to_half(psi: np.ndarray, parity: int) -> np.ndarray:
    """Parity-compacted half field [V/2, 4, 3] from a full field (layout only)."""
    lt, lz, ly, lx = psi.shape[:4]
    p = parity_of_sites((lx, ly, lz, lt)).reshape(-1)
    return np.ascontiguousarray(psi.reshape(-1, 4, 3)[p == parity])


def from_half(half_e: np.ndarray, half_o: np.ndarray, dims) -> np.ndarray:
    """Full field from its two parity-compacted halves (layout only)."""
    lx, ly, lz, lt = check_dims(dims)
    p = parity_of_sites(dims).reshape(-1)
    full = np.empty((volume(dims), 4, 3), dtype=np.complex128)
    full[p == 0] = half_e
    full[p == 1] = half_o
    return full.reshape(lt, lz, ly, lx, 4, 3)


# The workloads: lattice extents (Lx, Ly, Lz, Lt), hopping parameter, twisted
# mass, link spread eps and seed, following the finite-temperature shapes of
# the paper (N_sigma/N_tau ~ 3, Sec. 1) and its 24^3 x 8 setups (Sec. 7).
WORKLOADS = {
    "4^4": dict(dims=(4, 4, 4, 4), kappa=0.15, mu=0.0, eps=0.3, seed=1001),
    "24^3x8": dict(dims=(24, 24, 24, 8), kappa=0.155, mu=0.0, eps=0.2, seed=1002),
    "32^3x8": dict(dims=(32, 32, 32, 8), kappa=0.16, mu=0.01, eps=0.2, seed=1003),
    "48^3x12": dict(dims=(48, 48, 48, 12), kappa=0.16, mu=0.01, eps=0.2, seed=1004),
}

SWEEP_VOLUMES = [(8, 8, 8, 4), (16, 16, 16, 8), (24, 24, 24, 8), (32, 32, 32, 8), (48, 48, 48, 12)]
