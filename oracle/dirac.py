"""The O(a)-improved Wilson-Dirac operator D_W, Eq. (wd-op) of arXiv:0903.4936.

(D_W q)(n) = q(n)
    - kappa * sum_mu [ (1 - gamma_mu) U_mu(n) q(n+mu)
                       + (1 + gamma_mu) U_mu(n-mu)^dagger q(n-mu) ]
    - kappa * c_SW * sum_{mu,nu} (i/2) sigma_mu_nu F_mu_nu(n) q(n)

The sum over (mu, nu) runs over all 16 ordered pairs, as printed.  The full
4x4 spin matrices are applied (no spin projection), periodic boundaries in
all four directions, including time.

A block X holds L spinor columns: X[i, t, z, y, x, alpha, a].  ``kappa`` may
be a scalar or one value per column.
"""
from __future__ import annotations

import numpy as np

from .clover import field_strength, shift
from .gamma import GAMMA, IDENTITY4, sigma

__all__ = ["apply_dirac", "apply_dirac_at", "apply_gamma5", "hopping", "clover_term"]


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _colour(Ufield, X):
    """(U q)(n)[alpha, a] = sum_b U(n)[a, b] q(n)[alpha, b] for every column."""
    return np.matmul(X, np.swapaxes(Ufield, -1, -2))


def _spin(G, X):
    """(G q)[alpha, a] = sum_beta G[alpha, beta] q[beta, a]."""
    return np.matmul(G, X)


def hopping(U: np.ndarray, X: np.ndarray) -> np.ndarray:
    """sum_mu [(1-gamma_mu) U_mu(n) X(n+mu) + (1+gamma_mu) U_mu(n-mu)^dag X(n-mu)]."""
    H = np.zeros_like(X)
    for mu in range(4):
        fwd = _colour(U[mu], shift(X, mu, +1, lead=1))
        H += _spin(IDENTITY4 - GAMMA[mu], fwd)
        bwd = _colour(_dag(shift(U[mu], mu, -1)), shift(X, mu, -1, lead=1))
        H += _spin(IDENTITY4 + GAMMA[mu], bwd)
    return H


def clover_term(F: np.ndarray, X: np.ndarray) -> np.ndarray:
    """sum over ordered (mu, nu) of (i/2) sigma_mu_nu F_mu_nu(n) X(n)."""
    C = np.zeros_like(X)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            C += _spin(0.5j * sigma(mu, nu), _colour(F[mu, nu], X))
    return C


def _kappa_col(kappa, L):
    k = np.asarray(kappa, dtype=np.float64)
    if k.ndim == 0:
        return k
    assert k.shape == (L,)
    return k.reshape((L,) + (1,) * 6)


def apply_dirac(U, X, kappa, csw, F=None) -> np.ndarray:
    """Y = D_W X, Eq. (wd-op).  ``F`` may be passed to reuse a field strength."""
    X = np.asarray(X, dtype=np.complex128)
    k = _kappa_col(kappa, X.shape[0])
    Y = X - k * hopping(U, X)
    if csw != 0.0:
        if F is None:
            F = field_strength(U)
        Y = Y - k * csw * clover_term(F, X)
    return Y


def apply_gamma5(X: np.ndarray) -> np.ndarray:
    """gamma_5 acting on the spin index of every column."""
    from .gamma import GAMMA5
    return _spin(GAMMA5, X)


# --------------------------------------------------------------------------
# Site-by-site evaluation, for sampling D_W X on lattices too large to apply
# the whole operator in the oracle.  Same formula, written per site.
# --------------------------------------------------------------------------

def _coords(n, dims):
    Lx, Ly, Lz, Lt = dims
    x = n % Lx
    y = (n // Lx) % Ly
    z = (n // (Lx * Ly)) % Lz
    t = n // (Lx * Ly * Lz)
    return [x, y, z, t]


def _step(c, mu, d, dims):
    c = list(c)
    c[mu] = (c[mu] + d) % dims[mu]
    return c


def _at(field, c):
    """field[..., t, z, y, x, ...] at coordinates c = [x, y, z, t]."""
    return field[c[3], c[2], c[1], c[0]]


def _site_field_strength(U, c, dims, mu, nu):
    Um, Un = U[mu], U[nu]
    s = lambda cc, m, d: _step(cc, m, d, dims)  # noqa: E731
    P1 = _at(Um, c) @ _at(Un, s(c, mu, 1)) @ _dag(_at(Um, s(c, nu, 1))) @ _dag(_at(Un, c))
    P2 = (_at(Un, c) @ _dag(_at(Um, s(s(c, mu, -1), nu, 1))) @ _dag(_at(Un, s(c, mu, -1)))
          @ _at(Um, s(c, mu, -1)))
    P3 = (_dag(_at(Um, s(c, mu, -1))) @ _dag(_at(Un, s(s(c, mu, -1), nu, -1)))
          @ _at(Um, s(s(c, mu, -1), nu, -1)) @ _at(Un, s(c, nu, -1)))
    P4 = (_dag(_at(Un, s(c, nu, -1))) @ _at(Um, s(c, nu, -1))
          @ _at(Un, s(s(c, mu, 1), nu, -1)) @ _dag(_at(Um, c)))
    acc = np.zeros((3, 3), dtype=np.complex128)
    for P in (P1, P2, P3, P4):
        acc += (P - _dag(P)) / (2j)
    return acc / 4.0


def apply_dirac_at(U, X, kappa, csw, sites, dims) -> np.ndarray:
    """(D_W X)(n) for the listed flat site indices only; returns [L, len(sites), 4, 3]."""
    X = np.asarray(X)
    L = X.shape[0]
    k = np.asarray(kappa, dtype=np.float64)
    kcol = np.broadcast_to(k, (L,)) if k.ndim == 0 else k
    out = np.zeros((L, len(sites), 4, 3), dtype=np.complex128)
    for j, n in enumerate(sites):
        c = _coords(int(n), dims)
        h = np.zeros((L, 4, 3), dtype=np.complex128)
        for mu in range(4):
            cf = _step(c, mu, 1, dims)
            cb = _step(c, mu, -1, dims)
            qf = X[:, cf[3], cf[2], cf[1], cf[0]]
            qb = X[:, cb[3], cb[2], cb[1], cb[0]]
            h += _spin(IDENTITY4 - GAMMA[mu], _colour(_at(U[mu], c), qf))
            h += _spin(IDENTITY4 + GAMMA[mu], _colour(_dag(_at(U[mu], cb)), qb))
        cl = np.zeros((L, 4, 3), dtype=np.complex128)
        if csw != 0.0:
            for mu in range(4):
                for nu in range(4):
                    if mu != nu:
                        F = _site_field_strength(U, c, dims, mu, nu)
                        cl += _spin(0.5j * sigma(mu, nu), _colour(F, X[:, c[3], c[2], c[1], c[0]]))
        q = X[:, c[3], c[2], c[1], c[0]]
        out[:, j] = q - kcol[:, None, None] * (h + csw * cl)
    return out
