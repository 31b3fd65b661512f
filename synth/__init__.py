"""Seeded synthetic inputs for the clover Wilson-Dirac block solvers.

This module is shared by the CPU oracle (``oracle/``) and the CUDA path
(``paper_0903_4936_gb300``).  It holds none of the solver's arithmetic: it
only draws random gauge links and source blocks, so that both sides receive
the very same bytes.

Conventions
-----------
* Lattice ``dims = (Lx, Ly, Lz, Lt)``; periodic in all four directions.
* Site index ``n = x + Lx*(y + Ly*(z + Lz*t))``; numpy arrays put the lattice
  axes in the order ``(t, z, y, x)`` so that a C-order flatten gives ``n``.
* Gauge field: ``U[mu, t, z, y, x, a, b]`` complex128, ``mu = 0..3`` for the
  paper's directions 1..4 (x, y, z, t) (Section 2).
* Source block: ``B[i, t, z, y, x, alpha, a]`` complex128, column ``i`` of the
  N x L right-hand side (N = 12 V); component order spin-major,
  ``3*alpha + a`` (Section 2, point-source definition with 0-based indices).

Random numbers come from numpy's PCG64 (``numpy.random.default_rng``); the
stream is fixed by the seed.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "random_su3_field",
    "unit_gauge_field",
    "point_sources",
    "z2_noise",
    "z4_noise",
    "gaussian_sources",
    "lattice_volume",
]


def lattice_volume(dims) -> int:
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    return Lx * Ly * Lz * Lt


def _lat_shape(dims):
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    return (Lt, Lz, Ly, Lx)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_1..lambda_8 (standard normalisation,
    Tr(lambda_a lambda_b) = 2 delta_ab), shape [8, 3, 3]."""
    g = np.zeros((8, 3, 3), dtype=np.complex128)
    g[0][0, 1] = g[0][1, 0] = 1
    g[1][0, 1] = -1j
    g[1][1, 0] = 1j
    g[2][0, 0] = 1
    g[2][1, 1] = -1
    g[3][0, 2] = g[3][2, 0] = 1
    g[4][0, 2] = -1j
    g[4][2, 0] = 1j
    g[5][1, 2] = g[5][2, 1] = 1
    g[6][1, 2] = -1j
    g[6][2, 1] = 1j
    g[7][0, 0] = g[7][1, 1] = 1 / np.sqrt(3)
    g[7][2, 2] = -2 / np.sqrt(3)
    return g


def _reunitarise(M: np.ndarray) -> np.ndarray:
    """Project rows onto SU(3): Gram-Schmidt of rows 1-2, row 3 = conj(r1 x r2)."""
    r1 = M[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = M[..., 1, :]
    r2 = r2 - np.sum(r1.conj() * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.cross(r1, r2).conj()
    return np.stack([r1, r2, r3], axis=-2)


def random_su3_field(dims, eps: float, seed: int) -> np.ndarray:
    """Links U = exp(i eps H), H = sum_a c_a lambda_a / 2, c_a ~ N(0, 1).

    The exponential uses the eigen-decomposition of the Hermitian 3x3 H;
    the result is re-unitarised to SU(3) to remove rounding.  Returns
    U[mu, t, z, y, x, a, b] complex128.
    """
    rng = np.random.default_rng(seed)
    shape = (4,) + _lat_shape(dims)
    c = rng.standard_normal(shape + (8,))
    H = np.einsum("...k,kab->...ab", c, gell_mann() / 2.0)
    w, Vec = np.linalg.eigh(H)
    U = np.einsum("...ak,...k,...bk->...ab", Vec, np.exp(1j * eps * w), Vec.conj())
    return np.ascontiguousarray(_reunitarise(U))


def unit_gauge_field(dims) -> np.ndarray:
    """Free field: every link is the 3x3 identity."""
    shape = (4,) + _lat_shape(dims) + (3, 3)
    U = np.zeros(shape, dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def point_sources(dims) -> np.ndarray:
    """The twelve point sources at the origin (Section 2): column
    i = 3*alpha + a (0-based) is 1 at site 0, spin alpha, colour a."""
    B = np.zeros((12,) + _lat_shape(dims) + (4, 3), dtype=np.complex128)
    for alpha in range(4):
        for a in range(3):
            B[3 * alpha + a, 0, 0, 0, 0, alpha, a] = 1.0
    return B


def z2_noise(dims, L: int, seed: int) -> np.ndarray:
    """Complex Z2 noise: entries (+-1 +- i)/sqrt(2) with independent signs."""
    rng = np.random.default_rng(seed)
    shape = (L,) + _lat_shape(dims) + (4, 3)
    re = rng.integers(0, 2, size=shape, dtype=np.int8) * 2 - 1
    im = rng.integers(0, 2, size=shape, dtype=np.int8) * 2 - 1
    return (re + 1j * im) / np.sqrt(2.0)


def z4_noise(dims, L: int, seed: int) -> np.ndarray:
    """Z4 noise: entries drawn uniformly from {1, i, -1, -i}."""
    rng = np.random.default_rng(seed)
    shape = (L,) + _lat_shape(dims) + (4, 3)
    k = rng.integers(0, 4, size=shape, dtype=np.int8)
    table = np.array([1.0, 1j, -1.0, -1j], dtype=np.complex128)
    return table[k]


def gaussian_sources(dims, L: int, seed: int) -> np.ndarray:
    """Complex Gaussian entries, re and im ~ N(0, 1/2) (unit mean |z|^2)."""
    rng = np.random.default_rng(seed)
    shape = (L,) + _lat_shape(dims) + (4, 3)
    z = rng.standard_normal(shape + (2,)) * np.sqrt(0.5)
    return z[..., 0] + 1j * z[..., 1]
