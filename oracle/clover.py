"""Clover-leaf field strength F_mu_nu(n) (Section 2 of arXiv:0903.4936).

F_mu_nu(n) = (1/4) sum_{i=1..4} (1/(2i)) (P_i(n) - P_i(n)^dagger), where the
P_i are the four plaquette leaves in the (mu, nu) plane that start and end
at n.  The trace is NOT subtracted (the paper does not subtract it).

Two factors are misprinted in the paper and are read as follows (a leaf must
be a closed path; the corrected form is gauge covariant, the printed form
is not):

* P_1, third factor: printed U_nu^dagger(n+nu); read U_mu^dagger(n+nu), the
  path n -> n+mu -> n+mu+nu -> n+nu -> n.
* P_4, second factor: printed U_nu(n-nu); read U_mu(n-nu), the path
  n -> n-nu -> n-nu+mu -> n+mu -> n.

P_2 and P_3 are used as printed.
"""
from __future__ import annotations

import numpy as np

__all__ = ["shift", "leaves", "field_strength"]


def shift(f: np.ndarray, mu: int, step: int, lead: int = 0) -> np.ndarray:
    """Return g with g(n) = f(n + step * mu_hat), periodic.

    ``f`` has ``lead`` leading axes, then the lattice axes (t, z, y, x).
    Direction mu = 0..3 is x, y, z, t, i.e. lattice axis ``lead + 3 - mu``.
    """
    return np.roll(f, -step, axis=lead + 3 - mu)


def _dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def leaves(U: np.ndarray, mu: int, nu: int):
    """The four leaves P_1..P_4 of the (mu, nu) plane at every site.

    U[mu, t, z, y, x, a, b]; returns four arrays [t, z, y, x, 3, 3].
    """
    Um, Un = U[mu], U[nu]
    s = shift
    P1 = Um @ s(Un, mu, +1) @ _dag(s(Um, nu, +1)) @ _dag(Un)
    P2 = Un @ _dag(s(s(Um, mu, -1), nu, +1)) @ _dag(s(Un, mu, -1)) @ s(Um, mu, -1)
    P3 = (_dag(s(Um, mu, -1)) @ _dag(s(s(Un, mu, -1), nu, -1))
          @ s(s(Um, mu, -1), nu, -1) @ s(Un, nu, -1))
    P4 = _dag(s(Un, nu, -1)) @ s(Um, nu, -1) @ s(s(Un, mu, +1), nu, -1) @ _dag(Um)
    return P1, P2, P3, P4


def field_strength(U: np.ndarray) -> np.ndarray:
    """F[mu, nu, t, z, y, x, a, b] for all ordered pairs (F[mu, mu] = 0)."""
    lat = U.shape[1:5]
    F = np.zeros((4, 4) + lat + (3, 3), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            acc = np.zeros(lat + (3, 3), dtype=np.complex128)
            for P in leaves(U, mu, nu):
                acc += (P - _dag(P)) / (2j)
            F[mu, nu] = acc / 4.0
    return F
