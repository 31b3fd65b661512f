"""Dense N x N matrix of D_W on small lattices (N = 12 V).

Row / column index = 12*n + 3*alpha + a (site n, spin alpha, colour a), the
canonical flattening of a spinor.  Column j is D_W applied to the j-th unit
vector, Eq. (wd-op); the operator is assembled in chunks of columns.
"""
from __future__ import annotations

import numpy as np

from .clover import field_strength
from .dirac import apply_dirac

__all__ = ["dense_matrix", "to_columns", "from_columns"]


def to_columns(X: np.ndarray) -> np.ndarray:
    """Block X[L, t, z, y, x, 4, 3] -> the paper's N x L matrix."""
    L = X.shape[0]
    return np.ascontiguousarray(X.reshape(L, -1).T)


def from_columns(M: np.ndarray, dims) -> np.ndarray:
    """N x L matrix -> block [L, t, z, y, x, 4, 3]."""
    Lx, Ly, Lz, Lt = dims
    L = M.shape[1]
    return np.ascontiguousarray(M.T.reshape(L, Lt, Lz, Ly, Lx, 4, 3))


def dense_matrix(U: np.ndarray, kappa: float, csw: float, chunk: int = 384) -> np.ndarray:
    Lt, Lz, Ly, Lx = U.shape[1:5]
    dims = (Lx, Ly, Lz, Lt)
    N = 12 * Lx * Ly * Lz * Lt
    F = field_strength(U) if csw != 0.0 else None
    A = np.zeros((N, N), dtype=np.complex128)
    for j0 in range(0, N, chunk):
        j1 = min(N, j0 + chunk)
        E = np.zeros((N, j1 - j0), dtype=np.complex128)
        E[np.arange(j0, j1), np.arange(j1 - j0)] = 1.0
        A[:, j0:j1] = to_columns(apply_dirac(U, from_columns(E, dims), kappa, csw, F=F))
    return A
