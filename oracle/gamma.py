"""Euclidean Dirac matrices (Section 2 of arXiv:0903.4936).

gamma_1..gamma_5 are entered exactly as the paper prints them (Dirac /
Bjorken-Drell representation, only the nonzero entries are listed there);
sigma_mu_nu = (1/2)[gamma_mu, gamma_nu].  gamma_5 is taken as printed and is
never derived as a product of the other four (with these matrices the product
gamma_1 gamma_2 gamma_3 gamma_4 equals -gamma_5).

Index convention: ``GAMMA[mu]`` for mu = 0..3 is the paper's gamma_{mu+1}
(directions x, y, z, t); ``GAMMA5`` is gamma_5.  Spin indices 0..3 are the
paper's alpha = 1..4.
"""
from __future__ import annotations

import numpy as np

__all__ = ["GAMMA", "GAMMA5", "IDENTITY4", "sigma"]


def _mat(entries):
    m = np.zeros((4, 4), dtype=np.complex128)
    for (row, col), v in entries.items():
        m[row - 1, col - 1] = v
    return m


# Entries (row, column) -> value, 1-based as printed in Section 2.
_G1 = _mat({(1, 4): -1j, (2, 3): -1j, (3, 2): 1j, (4, 1): 1j})
_G2 = _mat({(1, 4): -1, (2, 3): 1, (3, 2): 1, (4, 1): -1})
_G3 = _mat({(1, 3): -1j, (2, 4): 1j, (3, 1): 1j, (4, 2): -1j})
_G4 = _mat({(1, 1): 1, (2, 2): 1, (3, 3): -1, (4, 4): -1})
_G5 = _mat({(1, 3): 1, (2, 4): 1, (3, 1): 1, (4, 2): 1})

GAMMA = np.stack([_G1, _G2, _G3, _G4])
GAMMA5 = _G5
IDENTITY4 = np.eye(4, dtype=np.complex128)


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_mu_nu = (1/2)[gamma_mu, gamma_nu] (Section 2), 0-based mu, nu."""
    g = GAMMA
    return 0.5 * (g[mu] @ g[nu] - g[nu] @ g[mu])
