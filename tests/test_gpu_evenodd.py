"""GPU even-odd (Schur complement) form against the FP64 oracle: the Schur
operator per precision against oracle.evenodd, and solves through the Schur
system (bk_solve_params.eo) against dense LU of the full system and the
oracle's block BiCGGR solution.  The even-odd form is not in the paper; it
reorders the same system, so its solutions are the paper's."""
import numpy as np
import pytest

import synth
from oracle import dense, dirac, evenodd, solvers

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# M x = x - kappa^2 A^-1 H A^-1 H x: two hopping sums and two site inverses.
# FP32: unit roundoff times ~100 terms; FP16: the input and the odd-site
# temporary each stored with 11 mantissa bits (2.4e-4 of the site's largest
# component); FP64 / double-float: rounding of the Gauss-Jordan inverse and
# the sums.
TOL = {"fp64": 1e-13, "df64": 1e-12, "fp32": 5e-6, "fp16": 5e-3}


def _lat(dims, eps, seed, csw=1.0):
    import paper_0903_4936_gb300 as bk
    U = synth.random_su3_field(dims, eps, seed)
    lat = bk.Lattice(dims)
    lat.upload_gauge(U)
    lat.build_clover(csw)
    return lat, U


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _dev(X, Xref):
    a = X.reshape(X.shape[0], -1)
    b = Xref.reshape(Xref.shape[0], -1)
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32", "fp16"])
@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 12), ((2, 4, 2, 6), 5), ((6, 4, 4, 8), 13),
                                    ((8, 8, 8, 16), 6)])
def test_schur_operator_matches_oracle(prec, dims, L):
    """Y_e = M X_e for several kappas at once (one per column pair, ragged odd
    L), zero on the odd sites, whatever X holds there."""
    lat, U = _lat(dims, 0.5, 400 + L)
    X = synth.gaussian_sources(dims, L, 11)
    kappa = [0.110 + 0.002 * ((j // 2) % 5) for j in range(L)]
    Y = lat.schur_dslash(torch.from_numpy(X).cuda(), kappa, prec).cpu().numpy()
    odd = evenodd.parity_mask(dims, 1)
    assert np.max(np.abs(Y[:, odd])) == 0.0
    for j in range(L):
        ref = evenodd.schur_apply(U, X[j:j + 1], kappa[j], 1.0)
        assert _rel(Y[j:j + 1], ref) < TOL[prec], (j, _rel(Y[j:j + 1], ref))


@pytest.mark.parametrize("variant", ["1", "2", "4", "5"])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_schur_operator_every_launch_variant(monkeypatch, variant, prec):
    """Each launch form of the packed-pair Schur operator the tuner may pick
    (forced with BK_DSLASH_VARIANT, pair groups of 8; L = 21: a full group and
    a short one, and a padding column); FP16 runs the 128-thread form for the
    FP32-only staged variants 4 and 5."""
    monkeypatch.setenv("BK_DSLASH_VARIANT", variant)
    dims, L = (4, 4, 4, 8), 21
    lat, U = _lat(dims, 0.5, 77)
    X = synth.gaussian_sources(dims, L, 12)
    kappa = [0.112 + 0.003 * ((j // 2) % 3) for j in range(L)]
    Y = lat.schur_dslash(torch.from_numpy(X).cuda(), kappa, prec).cpu().numpy()
    for j in range(L):
        ref = evenodd.schur_apply(U, X[j:j + 1], kappa[j], 1.0)
        assert _rel(Y[j:j + 1], ref) < TOL[prec], (j, _rel(Y[j:j + 1], ref))
    if prec == "fp32":
        B = torch.from_numpy(synth.z4_noise(dims, 6, 9)).cuda()
        X6, info = lat.block_solve(B, 0.12, method="bicgstab", prec="fp32", tol=1e-10, maxiter=1000, eo=True)
        assert info["converged"] == 1 and info["true_res_max"] <= 1e-10


def test_schur_operator_rejects_odd_x_extent_and_split_pairs():
    import paper_0903_4936_gb300 as bk
    lat, U = _lat((3, 4, 4, 4), 0.5, 5)
    X = torch.from_numpy(synth.gaussian_sources((3, 4, 4, 4), 2, 1)).cuda()
    with pytest.raises(bk.BKError):
        lat.schur_dslash(X, [0.12, 0.12], "fp64")
    with pytest.raises(bk.BKError):
        lat.block_solve(X, 0.12, method="bicgstab", prec="fp64", eo=True)
    lat, U = _lat((4, 4, 4, 4), 0.5, 5)
    X = torch.from_numpy(synth.gaussian_sources((4, 4, 4, 4), 2, 1)).cuda()
    with pytest.raises(bk.BKError):
        lat.schur_dslash(X, [0.12, 0.121], "fp32")


@pytest.fixture(scope="module")
def c1():
    """4^4, eps = 0.3, kappa = 0.12, c_SW = 1, 12 point sources; dense LU."""
    dims = (4, 4, 4, 4)
    lat, U = _lat(dims, 0.3, 1001)
    B = synth.point_sources(dims)
    D = dense.dense_matrix(U, 0.12, 1.0)
    Xd = dense.from_columns(np.linalg.solve(D, dense.to_columns(B)), dims)
    return dims, lat, U, B, Xd


@pytest.mark.parametrize("method", ["bicgstab", "bicggr"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eo_solve_matches_dense_lu(c1, method, prec):
    """The Schur solve reconstructs the full solution: FP64 true residual of
    the full system <= tol and the dense LU solution to 1e-8; the library's
    reported true residual is re-checked with the oracle."""
    dims, lat, U, B, Xd = c1
    X, info = lat.block_solve(torch.from_numpy(B).cuda(), 0.12, method=method, prec=prec, tol=1e-10,
                              maxiter=1000, eo=True)
    X = X.cpu().numpy()
    assert info["converged"] == 1 and info["true_res_max"] <= 1e-10
    assert _dev(X, Xd) <= 1e-8
    A = lambda M: dense.to_columns(dirac.apply_dirac(U, dense.from_columns(M, dims), 0.12, 1.0))  # noqa: E731
    tr, _ = solvers.true_residual(A, dense.to_columns(B), dense.to_columns(X))
    assert abs(tr - info["true_res_max"]) <= 1e-6 * max(tr, 1e-12)


def test_eo_needs_fewer_iterations(c1):
    """The Schur system is better conditioned: FP64 block BiCGSTAB on it needs
    fewer iterations than on the full system (same right-hand sides)."""
    dims, lat, U, B, Xd = c1
    Bt = torch.from_numpy(B).cuda()
    _, full = lat.block_solve(Bt, 0.12, method="bicgstab", prec="fp64", tol=1e-10, maxiter=1000)
    _, half = lat.block_solve(Bt, 0.12, method="bicgstab", prec="fp64", tol=1e-10, maxiter=1000, eo=True)
    assert half["iterations"] < full["iterations"], (half["iterations"], full["iterations"])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eo_batched_kappas_match_dense(c1, prec):
    """Batched systems with their own kappa and odd widths (padding columns),
    each against dense LU of its full system."""
    dims, lat, U, B, Xd = c1
    kappas, Ls = [0.11, 0.12, 0.125], [2, 4, 3]
    G = synth.z4_noise(dims, sum(Ls), 21)
    X, infos = lat.block_solve_batched(torch.from_numpy(G).cuda(), kappas, Ls, method="bicgstab", prec=prec,
                                       tol=1e-10, maxiter=1000, eo=True)
    X = X.cpu().numpy()
    c0 = 0
    for k, L, info in zip(kappas, Ls, infos):
        assert info["converged"] == 1 and info["true_res_max"] <= 1e-10
        D = dense.dense_matrix(U, k, 1.0)
        ref = dense.from_columns(np.linalg.solve(D, dense.to_columns(G[c0:c0 + L])), dims)
        assert _dev(X[c0:c0 + L], ref) <= 1e-8
        c0 += L


def test_eo_c2_mixed_matches_oracle():
    """8^3 x 16, eps = 0.5, kappa = 0.125, the 12 point sources as two 6-column
    systems: FP32 inner iterations on the Schur system against the oracle's
    FP64 block BiCGGR solution of the full system."""
    dims = (8, 8, 8, 16)
    lat, U = _lat(dims, 0.5, 1002)
    B = synth.point_sources(dims)
    A = lambda M: dense.to_columns(dirac.apply_dirac(U, dense.from_columns(M, dims), 0.125, 1.0))  # noqa: E731
    Xo, info_o = solvers.block_bicggr(A, dense.to_columns(B), 1e-12, 1000)
    assert info_o["converged"]
    Xo = dense.from_columns(Xo, dims)
    X, infos = lat.block_solve_batched(torch.from_numpy(B).cuda(), [0.125, 0.125], [6, 6], method="bicgstab",
                                       prec="fp32", tol=1e-10, maxiter=1000, eo=True)
    for info in infos:
        assert info["converged"] == 1 and info["true_res_max"] <= 1e-10
    assert _dev(X.cpu().numpy(), Xo) <= 1e-8


def test_eo_initial_guess_and_host_buffers(c1):
    """An initial guess (its even sites) is used, and host buffers go through
    the same staging as the full system."""
    dims, lat, U, B, Xd = c1
    Bh = torch.from_numpy(B).pin_memory()
    X, info = lat.block_solve(Bh, 0.12, method="bicgstab", prec="fp64", tol=1e-10, maxiter=1000, eo=True)
    assert info["converged"] == 1 and _dev(X.numpy(), Xd) <= 1e-8
    X0 = torch.from_numpy(Xd + 1e-6 * synth.gaussian_sources(dims, 12, 3)).cuda()
    X1, info1 = lat.block_solve(torch.from_numpy(B).cuda(), 0.12, method="bicgstab", prec="fp64", tol=1e-10,
                                maxiter=1000, X0=X0, eo=True)
    assert info1["converged"] == 1 and _dev(X1.cpu().numpy(), Xd) <= 1e-8
    assert info1["iterations"] < info["iterations"]


def test_eo_fp16_storage_matches_dense_lu(c1):
    """FP16-stored inner iterations on the Schur system (FP64 replacements and
    true residual): the full solution to dense LU accuracy."""
    dims, lat, U, B, Xd = c1
    X, infos = lat.block_solve_batched(torch.from_numpy(B).cuda(), [0.12, 0.12], [6, 6], method="bicgstab",
                                       prec="fp16", tol=1e-10, maxiter=2000, eo=True)
    for info in infos:
        assert info["converged"] == 1 and info["true_res_max"] <= 1e-10, info
    assert _dev(X.cpu().numpy(), Xd) <= 1e-8


def test_eo_rejects_deflate_and_caller_rtilde(c1):
    import paper_0903_4936_gb300 as bk
    dims, lat, U, B, Xd = c1
    Bt = torch.from_numpy(B).cuda()
    with pytest.raises(bk.BKError):
        lat.block_solve(Bt, 0.12, method="bicgstab", prec="fp64", eo=True, deflate=True)
    with pytest.raises(bk.BKError):
        lat.block_solve(Bt, 0.12, method="bicgstab", prec="fp64", eo=True, rtilde=Bt.clone())
