"""Pins of the oracle's even-odd (Schur complement) form of D_W X = B.

The even-odd system is not in the paper; it is a reordering of Eq.
(linear_mrhs), and these tests pin it to the dense matrix of D_W (built from
the oracle's Eq. (wd-op)) and to block elimination, not to itself:
* the hopping term only connects sites of opposite parity, and the site
  blocks A(n) are the diagonal 12 x 12 blocks of the dense D_W;
* M x_e equals (I - D_ee^-1 D_eo D_oo^-1 D_oe) x_e from the dense blocks;
* solving the Schur system and reconstructing the odd sites gives the dense
  LU solution of the full system (a wrong sign of kappa^2, a swapped parity
  or a missing A^-1 fails here)."""
import numpy as np
import pytest

import synth
from oracle import dense, dirac, evenodd

DIMS = (2, 4, 2, 4)
KAPPA, CSW = 0.12, 1.0


@pytest.fixture(scope="module")
def problem():
    U = synth.random_su3_field(DIMS, 0.5, 1101)
    D = dense.dense_matrix(U, KAPPA, CSW)
    # row/column index 12 n + (3 spin + colour); site n in canonical order
    even_site = evenodd.parity_mask(DIMS, 0).reshape(-1)
    idx_e = np.concatenate([np.arange(12 * n, 12 * n + 12) for n in np.nonzero(even_site)[0]])
    idx_o = np.concatenate([np.arange(12 * n, 12 * n + 12) for n in np.nonzero(~even_site)[0]])
    return U, D, idx_e, idx_o


def test_hopping_connects_opposite_parity_only(problem):
    U, D, idx_e, idx_o = problem
    X = synth.gaussian_sources(DIMS, 2, 5)
    Xe = X * evenodd.parity_mask(DIMS, 0)[None, :, :, :, :, None, None]
    H = dirac.hopping(U, Xe)
    assert np.max(np.abs(H * evenodd.parity_mask(DIMS, 0)[None, :, :, :, :, None, None])) == 0.0
    assert np.linalg.norm(H) > 1.0


def test_site_blocks_are_the_diagonal_blocks_of_D(problem):
    U, D, idx_e, idx_o = problem
    A = evenodd.site_blocks(U, KAPPA, CSW).reshape(-1, 12, 12)
    for n in range(A.shape[0]):
        np.testing.assert_allclose(A[n], D[12 * n:12 * n + 12, 12 * n:12 * n + 12], atol=1e-14)
    # and the off-diagonal same-parity blocks of D vanish
    assert np.max(np.abs(D[np.ix_(idx_e, idx_e)] - np.kron(np.eye(len(idx_e) // 12), np.ones((12, 12)))
                         * D[np.ix_(idx_e, idx_e)])) == 0.0


def test_schur_operator_matches_dense_blocks(problem):
    U, D, idx_e, idx_o = problem
    Dee, Deo = D[np.ix_(idx_e, idx_e)], D[np.ix_(idx_e, idx_o)]
    Doe, Doo = D[np.ix_(idx_o, idx_e)], D[np.ix_(idx_o, idx_o)]
    M = np.eye(len(idx_e)) - np.linalg.solve(Dee, Deo @ np.linalg.solve(Doo, Doe))
    X = synth.gaussian_sources(DIMS, 3, 6)
    Y = evenodd.schur_apply(U, X, KAPPA, CSW)
    Yc, Xc = dense.to_columns(Y), dense.to_columns(X)
    np.testing.assert_allclose(Yc[idx_e], M @ Xc[idx_e], atol=1e-12)
    assert np.max(np.abs(Yc[idx_o])) == 0.0


def test_schur_solve_reconstructs_the_full_solution(problem):
    U, D, idx_e, idx_o = problem
    B = synth.z4_noise(DIMS, 2, 7)
    Xd = np.linalg.solve(D, dense.to_columns(B))
    bh = evenodd.schur_rhs(U, B, KAPPA, CSW)
    # dense M from the oracle's own Schur operator applied to the even unit vectors
    ne = len(idx_e)
    E = np.zeros((D.shape[0], ne), dtype=np.complex128)
    E[idx_e, np.arange(ne)] = 1.0
    M = dense.to_columns(evenodd.schur_apply(U, dense.from_columns(E, DIMS), KAPPA, CSW))[idx_e]
    xe = np.linalg.solve(M, dense.to_columns(bh)[idx_e])
    Xe = np.zeros_like(Xd)
    Xe[idx_e] = xe
    X = dense.to_columns(evenodd.reconstruct(U, dense.from_columns(Xe, DIMS), B, KAPPA, CSW))
    np.testing.assert_allclose(X, Xd, rtol=0, atol=1e-11 * np.max(np.abs(Xd)))
