"""Pins of the oracle's D_W (Eq. (wd-op)), gamma matrices and clover field
strength against facts the paper and the mathematics fix (no GPU needed)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import clover, dense, dirac, gamma

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def _facts():
    with open(GOLDEN) as f:
        return json.load(f)


def _parse(v):
    return {"1": 1, "-1": -1, "i": 1j, "-i": -1j}[v]


# ---------------------------------------------------------------- gamma algebra

def test_gamma_matrices_as_printed():
    facts = _facts()["gamma_nonzero_entries"]
    for k, name in enumerate(["gamma1", "gamma2", "gamma3", "gamma4", "gamma5"]):
        m = np.zeros((4, 4), dtype=complex)
        for r, c, v in facts[name]:
            m[r - 1, c - 1] = _parse(v)
        ref = gamma.GAMMA[k] if k < 4 else gamma.GAMMA5
        assert np.array_equal(m, ref), name


def test_clifford_algebra_and_gamma5():
    G, G5, I = gamma.GAMMA, gamma.GAMMA5, np.eye(4)
    for m in range(4):
        assert np.allclose(G[m], G[m].conj().T)            # Hermitian
        for n in range(4):
            assert np.allclose(G[m] @ G[n] + G[n] @ G[m], 2 * (m == n) * I)
        assert np.allclose(G5 @ G[m] + G[m] @ G5, 0)      # anticommutes
    assert np.allclose(G5, G5.conj().T) and np.allclose(G5 @ G5, I)
    # With the printed matrices the product of the four is -gamma_5, which is
    # why the oracle never derives gamma_5 as a product.
    assert np.allclose(G[0] @ G[1] @ G[2] @ G[3], -G5)


def test_sigma_antihermitian_and_antisymmetric():
    for m in range(4):
        for n in range(4):
            s = gamma.sigma(m, n)
            assert np.allclose(s, -s.conj().T)
            assert np.allclose(s, -gamma.sigma(n, m))


# ---------------------------------------------------------------- free field

@pytest.mark.parametrize("kvec", [(1, 0, 2, 1), (0, 3, 1, 5), (2, 2, 2, 3)])
def test_free_field_plane_wave(kvec):
    """U = 1: D_W e^{ip.n} chi = e^{ip.n} D(p) chi, with
    D(p) = (1 - 2 kappa sum cos p_mu) + 2 i kappa sum gamma_mu sin p_mu
    (Fourier transform of Eq. (wd-op), forward hop e^{+ip_mu}), and its
    eigenvalues (1 - 2 kappa sum cos p) +- 2 i kappa sqrt(sum sin^2 p)."""
    dims = (4, 4, 4, 6)
    kappa, csw = 0.11, 1.3
    U = synth.unit_gauge_field(dims)
    p = np.array([2 * np.pi * k / d for k, d in zip(kvec, dims)])
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    X = np.zeros((12,) + phase.shape + (4, 3), dtype=complex)
    for j in range(12):
        X[j, ..., j // 3, j % 3] = phase
    Y = dirac.apply_dirac(U, X, kappa, csw)
    M = np.stack([Y[j, 0, 0, 0, 0].reshape(12) for j in range(12)], axis=1)
    # translation invariance
    for j in range(12):
        assert np.allclose(Y[j], phase[..., None, None] * M[:, j].reshape(4, 3), atol=1e-13)
    Dp = (1 - 2 * kappa * np.sum(np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        Dp = Dp + 2j * kappa * np.sin(p[mu]) * gamma.GAMMA[mu]
    assert np.allclose(M, np.kron(Dp, np.eye(3)), atol=1e-13)
    ev = np.linalg.eigvals(M)
    ev = ev[np.argsort(ev.imag)]
    a = 1 - 2 * kappa * np.sum(np.cos(p))
    b = 2 * kappa * np.sqrt(np.sum(np.sin(p) ** 2))
    ref = np.array([a - 1j * b] * 6 + [a + 1j * b] * 6)
    assert np.allclose(ev, ref, atol=1e-12)


# ---------------------------------------------------------------- symmetries

def _rand_block(dims, L, seed):
    return synth.gaussian_sources(dims, L, seed)


def _inner(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 4, 5, 6), (2, 3, 2, 4)])
def test_gamma5_hermiticity(dims):
    """<x, g5 D g5 y> = <D x, y>: needs sigma anti-Hermitian and the backward
    hop to carry U^dagger(n - mu)."""
    U = synth.random_su3_field(dims, 0.5, 11)
    x, y = _rand_block(dims, 2, 1), _rand_block(dims, 2, 2)
    g5 = dirac.apply_gamma5
    lhs = _inner(x, g5(dirac.apply_dirac(U, g5(y), 0.13, 1.7)))
    rhs = _inner(dirac.apply_dirac(U, x, 0.13, 1.7), y)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def _gauge_transform(U, g):
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = g @ U[mu] @ np.conj(np.swapaxes(clover.shift(g, mu, +1), -1, -2))
    return Ug


@pytest.mark.parametrize("dims", [(3, 3, 3, 3), (4, 3, 4, 5)])
def test_gauge_covariance(dims):
    """D[U^g] (g q) = g (D[U] q) with U^g_mu(n) = g(n) U_mu(n) g(n+mu)^dagger."""
    U = synth.random_su3_field(dims, 0.6, 21)
    g = synth.random_su3_field(dims, 2.0, 22)[0]
    Ug = _gauge_transform(U, g)
    q = _rand_block(dims, 3, 3)
    gq = np.matmul(q, np.swapaxes(g, -1, -2))
    lhs = dirac.apply_dirac(Ug, gq, 0.12, 1.1)
    rhs = np.matmul(dirac.apply_dirac(U, q, 0.12, 1.1), np.swapaxes(g, -1, -2))
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_printed_leaf_breaks_covariance(monkeypatch):
    """The leaf P_1 exactly as printed (third factor U_nu^dagger(n+nu)) is not a
    closed path; the covariance pin detects it.  This justifies reading that
    factor as U_mu^dagger(n+nu)."""
    dims = (3, 3, 3, 3)
    U = synth.random_su3_field(dims, 0.6, 31)
    g = synth.random_su3_field(dims, 2.0, 32)[0]
    orig = clover.leaves

    def printed(U_, mu, nu):
        P1, P2, P3, P4 = orig(U_, mu, nu)
        Um, Un = U_[mu], U_[nu]
        s, dag = clover.shift, lambda m: np.conj(np.swapaxes(m, -1, -2))
        P1 = Um @ s(Un, mu, +1) @ dag(s(Un, nu, +1)) @ dag(Un)
        return P1, P2, P3, P4

    monkeypatch.setattr(clover, "leaves", printed)
    F_bad = clover.field_strength(U)
    F_bad_g = clover.field_strength(_gauge_transform(U, g))
    gF = g @ F_bad[0, 1] @ np.conj(np.swapaxes(g, -1, -2))
    assert np.max(np.abs(F_bad_g[0, 1] - gF)) > 1e-3


def test_field_strength_antisymmetric_hermitian():
    U = synth.random_su3_field((3, 4, 3, 4), 0.5, 41)
    F = clover.field_strength(U)
    for m in range(4):
        assert np.max(np.abs(F[m, m])) == 0
        for n in range(4):
            assert np.allclose(F[m, n], -F[n, m])
            assert np.allclose(F[m, n], np.conj(np.swapaxes(F[m, n], -1, -2)))


# ---------------------------------------------------------------- clover closed forms

def _abelian_field(dims, mu_dir, nu_link, k):
    """U_nu(n) = diag(exp(i theta x_mu Lambda)), Lambda = diag(1,-1,0),
    theta = 2 pi k / L_mu; all other links 1.  Every leaf of the (mu, nu)
    plane is exp(i theta Lambda), so F_mu_nu = diag(sin theta, -sin theta, 0)
    and every other plane has F = 0."""
    U = synth.unit_gauge_field(dims)
    theta = 2 * np.pi * k / dims[mu_dir]
    Lx, Ly, Lz, Lt = dims
    coords = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    xmu = coords[3 - mu_dir]
    lam = np.array([1.0, -1.0, 0.0])
    U[nu_link] = 0
    for c in range(3):
        U[nu_link][..., c, c] = np.exp(1j * theta * xmu * lam[c])
    return U, theta


@pytest.mark.parametrize("plane,spin_mat", [
    # (x, y): -i sigma_12 = diag(1, -1, 1, -1) in the printed representation
    ((0, 1), np.diag([1.0, -1.0, 1.0, -1.0])),
    # (x, t): -i sigma_14 = anti-diagonal ones
    ((0, 3), np.fliplr(np.eye(4))),
])
def test_constant_field_clover_closed_form(plane, spin_mat):
    """For a constant abelian field in one plane the clover part of D_W is
    kappa c_SW (-i sigma_mu_nu) (x) F_mu_nu exactly (sum over both orders)."""
    dims = (4, 4, 4, 4)
    mu, nu = plane
    U, theta = _abelian_field(dims, mu, nu, 1)
    F = clover.field_strength(U)
    Fref = np.diag([np.sin(theta), -np.sin(theta), 0.0])
    assert np.allclose(F[mu, nu], Fref, atol=1e-14)
    for a in range(4):
        for b in range(4):
            if {a, b} != {mu, nu}:
                assert np.max(np.abs(F[a, b])) < 1e-14
    kappa, csw = 0.125, 1.7
    q = _rand_block(dims, 2, 5)
    diff = dirac.apply_dirac(U, q, kappa, csw) - dirac.apply_dirac(U, q, kappa, 0.0)
    ref = kappa * csw * np.einsum("st,ab,l...tb->l...sa", spin_mat, Fref, q)
    assert np.max(np.abs(diff - ref)) < 1e-14


# ---------------------------------------------------------------- sparsity

def test_nonzeros_per_row():
    """51 nonzeros in every row of D_W (Section 2), extents >= 3."""
    expected = _facts()["nonzeros_per_row"]["value"]
    U = synth.random_su3_field((3, 3, 3, 3), 0.4, 51)
    A = dense.dense_matrix(U, 0.12, 1.0)
    counts = np.count_nonzero(np.abs(A) > 0, axis=1)
    assert np.all(counts == expected)


def test_point_sources():
    B = synth.point_sources((4, 4, 4, 4))
    assert B.shape[0] == _facts()["point_source_columns"]["value"]
    M = dense.to_columns(B)
    assert np.array_equal(M[:12, :], np.eye(12))
    assert np.count_nonzero(M) == 12


def test_site_sampled_operator_matches_block_operator():
    dims = (3, 4, 3, 5)
    U = synth.random_su3_field(dims, 0.5, 61)
    X = _rand_block(dims, 3, 62)
    kap = np.array([0.11, 0.12, 0.13])
    Y = dirac.apply_dirac(U, X, kap, 1.2)
    sites = [0, 7, 59, 179]
    Ys = dirac.apply_dirac_at(U, X, kap, 1.2, sites, dims)
    Yf = Y.reshape(3, -1, 4, 3)
    assert np.max(np.abs(Ys - Yf[:, sites])) < 1e-13


def test_synthetic_links_are_su3():
    U = synth.random_su3_field((4, 4, 4, 4), 0.5, 71)
    M = U.reshape(-1, 3, 3)
    assert np.allclose(M @ np.conj(np.swapaxes(M, -1, -2)), np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(M), 1.0, atol=1e-14)


def test_noise_distributions():
    z2 = synth.z2_noise((4, 4, 4, 4), 4, 1)
    assert np.allclose(np.abs(z2), 1.0) and set(np.unique(np.round(z2.real * np.sqrt(2)))) == {-1.0, 1.0}
    z4 = synth.z4_noise((4, 4, 4, 4), 4, 2)
    assert np.allclose(np.abs(z4), 1.0)
    assert abs(np.mean(z4)) < 0.05
    g = synth.gaussian_sources((4, 4, 4, 4), 8, 3)
    assert abs(np.mean(np.abs(g) ** 2) - 1.0) < 0.05
