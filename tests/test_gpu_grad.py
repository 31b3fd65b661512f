"""Gradients of L = Re sum_i <eta_i, D_W^-1 B_i> with respect to B, kappa and
the gauge links, from the adjoint gamma_5 solve and the link-derivative
kernel, against central finite differences: of the oracle's exact loss
(dense LU, 4^4) and of the GPU forward solve (8^4, the differentiation
configuration)."""
import numpy as np
import pytest

import synth
from oracle import dense

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _su3_direction(shape, seed):
    """Random Hermitian traceless Z per link (coefficients of lambda_a / 2)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shape + (8,))
    Z = np.einsum("...k,kab->...ab", z, synth.gell_mann() / 2.0)
    return z, Z


def _expi(Z, t):
    w, V = np.linalg.eigh(Z)
    return np.einsum("...ak,...k,...bk->...ab", V, np.exp(1j * t * w), V.conj())


def _grads(lat, U, B, eta, kappa, csw, tol=1e-13):
    import paper_0903_4936_gb300 as bk
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    Bt = torch.from_numpy(B).cuda().requires_grad_(True)
    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    X = bk.block_solve_autograd(lat, Bt, kt, Ut, csw, prec="fp64", tol=tol)
    loss = (torch.conj(torch.from_numpy(eta).cuda()) * X).sum().real
    loss.backward()
    return Bt.grad.cpu().numpy(), float(kt.grad), Ut.grad.cpu().numpy(), float(loss)


def _dir_deriv_U(gradU, U, Z):
    """d/dt L(exp(i t Z) U) at t = 0 from the complex gradient G:
    dL = Re sum conj(G) dU with dU = i Z U."""
    dU = 1j * Z @ U
    return float(np.real(np.sum(np.conj(gradU) * dU)))


@pytest.fixture(scope="module")
def small():
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.4, 501)
    B = synth.gaussian_sources(dims, 3, 502)
    eta = synth.gaussian_sources(dims, 3, 503)
    return dims, U, B, eta


def _oracle_loss(dims, U, B, eta, kappa, csw):
    D = dense.dense_matrix(U, kappa, csw)
    X = np.linalg.solve(D, dense.to_columns(B))
    return float(np.real(np.vdot(dense.to_columns(eta), X)))


def test_gradients_match_oracle_finite_differences(small):
    import paper_0903_4936_gb300 as bk
    dims, U, B, eta = small
    kappa, csw = 0.12, 1.3
    lat = bk.Lattice(dims)
    gB, gk, gU, loss = _grads(lat, U, B, eta, kappa, csw)
    assert abs(loss - _oracle_loss(dims, U, B, eta, kappa, csw)) < 1e-10 * abs(loss)
    h = 1e-5
    # B
    rng = np.random.default_rng(9)
    dB = rng.standard_normal(B.shape) + 1j * rng.standard_normal(B.shape)
    fd = (_oracle_loss(dims, U, B + h * dB, eta, kappa, csw) - _oracle_loss(dims, U, B - h * dB, eta, kappa, csw)) / (2 * h)
    assert abs(np.real(np.vdot(gB, dB)) - fd) < 1e-6 * abs(fd)
    # kappa
    fd = (_oracle_loss(dims, U, B, eta, kappa + h, csw) - _oracle_loss(dims, U, B, eta, kappa - h, csw)) / (2 * h)
    assert abs(gk - fd) < 1e-6 * abs(fd)
    # links, along a random su(3) direction on every link (hopping + clover force)
    z, Z = _su3_direction(U.shape[:-2], 11)
    fd = (_oracle_loss(dims, _expi(Z, h) @ U, B, eta, kappa, csw)
          - _oracle_loss(dims, _expi(Z, -h) @ U, B, eta, kappa, csw)) / (2 * h)
    an = _dir_deriv_U(gU, U, Z)
    assert abs(an - fd) < 1e-6 * abs(fd)


def test_su3_projection_matches_complex_gradient(small):
    """mode 2 (Re Tr(i T_a U Sigma)) contracted with z_a equals the
    directional derivative built from the complex gradient (mode 1)."""
    import paper_0903_4936_gb300 as bk
    dims, U, B, eta = small
    kappa, csw = 0.12, 1.3
    lat = bk.Lattice(dims)
    lat.upload_gauge(U)
    lat.build_clover(csw)
    X = torch.from_numpy(synth.gaussian_sources(dims, 2, 1)).cuda()
    Lam = torch.from_numpy(synth.gaussian_sources(dims, 2, 2)).cuda()
    G = lat.gauge_force(X, Lam, mode=1, scale=kappa).cpu().numpy().reshape(U.shape)
    g8 = lat.gauge_force(X, Lam, mode=2, scale=kappa).cpu().numpy().reshape(U.shape[:-2] + (8,))
    z, Z = _su3_direction(U.shape[:-2], 12)
    assert abs(np.sum(z * g8) - _dir_deriv_U(G, U, Z)) < 1e-10 * abs(np.sum(z * g8))


def test_clover_force_vanishes_without_clover(small):
    """With c_SW = 0 the link derivative is the hopping part alone: check the
    hopping part in isolation against finite differences of the oracle."""
    import paper_0903_4936_gb300 as bk
    dims, U, B, eta = small
    kappa = 0.12
    lat = bk.Lattice(dims)
    gB, gk, gU, loss = _grads(lat, U, B, eta, kappa, 0.0)
    h = 1e-5
    z, Z = _su3_direction(U.shape[:-2], 13)
    fd = (_oracle_loss(dims, _expi(Z, h) @ U, B, eta, kappa, 0.0)
          - _oracle_loss(dims, _expi(Z, -h) @ U, B, eta, kappa, 0.0)) / (2 * h)
    assert abs(_dir_deriv_U(gU, U, Z) - fd) < 1e-6 * abs(fd)


def test_c5_gradients_match_gpu_finite_differences():
    """8^4, eps = 0.4, kappa = 0.124, c_SW = 1, L = 12 Gaussian sources, seeded
    probe block eta; central differences with step 1e-6 of FP64 GPU solves."""
    import paper_0903_4936_gb300 as bk
    dims = (8, 8, 8, 8)
    kappa, csw = 0.124, 1.0
    U = synth.random_su3_field(dims, 0.4, 1005)
    B = synth.gaussian_sources(dims, 12, 2005)
    eta = synth.gaussian_sources(dims, 12, 3005)
    lat = bk.Lattice(dims)
    gB, gk, gU, loss = _grads(lat, U, B, eta, kappa, csw, tol=1e-13)

    def L_of(Uv, Bv, kv):
        lat.upload_gauge(Uv)
        lat.build_clover(csw)
        X, _ = lat.block_solve(torch.from_numpy(Bv).cuda(), kv, prec="fp64", tol=1e-13, maxiter=5000)
        return float(np.real(np.vdot(eta.reshape(-1), X.cpu().numpy().reshape(-1))))

    h = 1e-6
    rng = np.random.default_rng(21)
    dB = rng.standard_normal(B.shape) + 1j * rng.standard_normal(B.shape)
    fd = (L_of(U, B + h * dB, kappa) - L_of(U, B - h * dB, kappa)) / (2 * h)
    assert abs(np.real(np.vdot(gB, dB)) - fd) < 1e-6 * abs(fd)
    fd = (L_of(U, B, kappa + h) - L_of(U, B, kappa - h)) / (2 * h)
    assert abs(gk - fd) < 1e-6 * abs(fd)
    z, Z = _su3_direction(U.shape[:-2], 22)
    fd = (L_of(_expi(Z, h) @ U, B, kappa) - L_of(_expi(Z, -h) @ U, B, kappa)) / (2 * h)
    assert abs(_dir_deriv_U(gU, U, Z) - fd) < 1e-6 * abs(fd)
