"""Even-odd (Schur complement) form of D_W X = B  (TEST INFRASTRUCTURE).

Not part of arXiv:0903.4936: a reordering of the same linear system (Eq.
(linear_mrhs)) by site parity p(n) = (x + y + z + t) mod 2.  Write D_W of Eq.
(wd-op) as D = A - kappa H, with the site-local part
    A(n) = 1 - kappa c_SW sum_{mu,nu} (i/2) sigma_mu_nu F_mu_nu(n)
and the hopping sum H, which only connects sites of opposite parity:

    D = [[A_ee, -kappa H_eo], [-kappa H_oe, A_oo]].

Eliminating the odd sites gives the Schur system on the even sites

    M x_e = b^_e,        M   = 1 - kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe,
                         b^_e = A_ee^-1 (b_e + kappa H_eo A_oo^-1 b_o),
    x_o = A_oo^-1 (b_o + kappa H_oe x_e),

whose solution is the solution of D x = b.  Everything here is computed from
the oracle's own pieces: H from ``dirac.hopping``, the 12 x 12 site blocks of
A by applying A to the 12 unit spinors, their inverses by numpy.  A
half-lattice vector is a full-lattice block that vanishes on the other
parity.  It is test infrastructure only, like the rest of ``oracle``.
"""
from __future__ import annotations

import numpy as np

from .clover import field_strength
from .dirac import clover_term, hopping

__all__ = ["parity_mask", "site_blocks", "apply_site", "schur_apply", "schur_rhs", "reconstruct"]


def parity_mask(dims, parity: int) -> np.ndarray:
    """[t, z, y, x] boolean mask of the sites with (x + y + z + t) mod 2 = parity."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((x + y + z + t) % 2) == parity


def site_blocks(U: np.ndarray, kappa: float, csw: float, F=None) -> np.ndarray:
    """A(n) as [t, z, y, x, 12, 12] matrices (row/column = 3 spin + colour):
    column j is A applied to the unit spinor e_j placed on every site."""
    Lt, Lz, Ly, Lx = U.shape[1:5]
    if F is None and csw != 0.0:
        F = field_strength(U)
    E = np.zeros((12, Lt, Lz, Ly, Lx, 4, 3), dtype=np.complex128)
    for j in range(12):
        E[j, ..., j // 3, j % 3] = 1.0
    AE = E.copy()
    if csw != 0.0:
        AE = AE - kappa * csw * clover_term(F, E)
    # AE[j, site, alpha, a] = (A e_j)(site)[alpha, a] -> A[site, 3 alpha + a, j]
    return np.moveaxis(AE.reshape(12, Lt, Lz, Ly, Lx, 12), 0, -1)


def apply_site(blocks: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y(n) = blocks(n) X(n) for every column of the block X[L, t, z, y, x, 4, 3]."""
    L = X.shape[0]
    Xf = X.reshape(X.shape[:5] + (12,))
    Y = np.einsum("tzyxij,ltzyxj->ltzyxi", blocks, Xf)
    return Y.reshape(X.shape) if L else Y


def _masked(X, mask):
    return X * mask[None, :, :, :, :, None, None]


def schur_apply(U: np.ndarray, Xe: np.ndarray, kappa: float, csw: float) -> np.ndarray:
    """M x_e for a block that vanishes on the odd sites (the result does too)."""
    dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    even, odd = parity_mask(dims, 0), parity_mask(dims, 1)
    Ainv = np.linalg.inv(site_blocks(U, kappa, csw))
    Xe = _masked(np.asarray(Xe, dtype=np.complex128), even)
    T = _masked(apply_site(Ainv, hopping(U, Xe)), odd)          # A_oo^-1 H_oe x_e
    return Xe - kappa ** 2 * _masked(apply_site(Ainv, hopping(U, T)), even)


def schur_rhs(U: np.ndarray, B: np.ndarray, kappa: float, csw: float) -> np.ndarray:
    """b^_e = A_ee^-1 (b_e + kappa H_eo A_oo^-1 b_o), zero on the odd sites."""
    dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    even, odd = parity_mask(dims, 0), parity_mask(dims, 1)
    Ainv = np.linalg.inv(site_blocks(U, kappa, csw))
    B = np.asarray(B, dtype=np.complex128)
    T = _masked(apply_site(Ainv, _masked(B, odd)), odd)
    return _masked(apply_site(Ainv, _masked(B, even) + kappa * _masked(hopping(U, T), even)), even)


def reconstruct(U: np.ndarray, Xe: np.ndarray, B: np.ndarray, kappa: float, csw: float) -> np.ndarray:
    """The full solution: x_e on the even sites, x_o = A_oo^-1 (b_o + kappa H_oe x_e)."""
    dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
    even, odd = parity_mask(dims, 0), parity_mask(dims, 1)
    Ainv = np.linalg.inv(site_blocks(U, kappa, csw))
    Xe = _masked(np.asarray(Xe, dtype=np.complex128), even)
    Xo = _masked(apply_site(Ainv, _masked(np.asarray(B, dtype=np.complex128), odd) + kappa * hopping(U, Xe)), odd)
    return Xe + Xo
