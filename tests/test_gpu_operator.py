"""GPU parity of the multi-RHS operator and the block linear algebra (C ABI)
against the FP64 oracle and numpy."""
import numpy as np
import pytest

import synth
from oracle import dirac

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# Relative (max-norm) tolerances of D_W X against the FP64 oracle.  FP64: the
# paper's operator to rounding.  FP32: unit roundoff 6e-8 times ~50 terms
# summed per output.  FP16 storage: inputs rounded to 11 mantissa bits
# relative to each site's largest component (2.4e-4), plus the output store.
# Double-float (df64): two floats per real, about 2^-46 per operation
# (sloppy addition), ~50 terms per output.
TOL = {"fp64": 1e-13, "df64": 1e-12, "fp32": 2e-6, "fp16": 2e-3}


def _lat(dims, eps, seed, csw=1.0):
    import paper_0903_4936_gb300 as bk
    U = synth.random_su3_field(dims, eps, seed)
    lat = bk.Lattice(dims)
    lat.upload_gauge(U)
    lat.build_clover(csw)
    return lat, U


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32", "fp16"])
@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 12), ((2, 4, 2, 6), 5), ((3, 5, 4, 6), 1),
                                    ((8, 8, 8, 16), 12), ((6, 4, 4, 4), 17), ((4, 4, 8, 8), 48)])
def test_dslash_matches_oracle(prec, dims, L):
    lat, U = _lat(dims, 0.5, 100 + L)
    X = synth.gaussian_sources(dims, L, 7)
    kappa = [0.11 + 0.002 * j for j in range(L)]
    Y = lat.dslash(torch.from_numpy(X).cuda(), kappa, prec).cpu().numpy()
    Yref = dirac.apply_dirac(U, X, np.array(kappa), 1.0)
    assert _rel(Y, Yref) < TOL[prec]


@pytest.mark.parametrize("csw", [0.0, 1.9])
def test_dslash_csw_values(csw):
    dims = (4, 4, 4, 6)
    lat, U = _lat(dims, 0.6, 5, csw)
    X = synth.z4_noise(dims, 3, 9)
    Y = lat.dslash(torch.from_numpy(X).cuda(), 0.13, "fp64").cpu().numpy()
    assert _rel(Y, dirac.apply_dirac(U, X, 0.13, csw)) < 1e-13


def test_dslash_point_sources_and_free_field():
    import paper_0903_4936_gb300 as bk
    dims = (4, 4, 4, 4)
    lat = bk.Lattice(dims)
    U = synth.unit_gauge_field(dims)
    lat.upload_gauge(U)
    lat.build_clover(1.0)
    B = synth.point_sources(dims)
    Y = lat.dslash(torch.from_numpy(B).cuda(), 0.125, "fp64").cpu().numpy()
    assert _rel(Y, dirac.apply_dirac(U, B, 0.125, 1.0)) < 1e-15


def test_gamma5_and_pack_roundtrip():
    dims = (4, 4, 4, 4)
    lat, U = _lat(dims, 0.3, 3)
    X = synth.gaussian_sources(dims, 4, 1)
    Xt = torch.from_numpy(X).cuda()
    assert np.array_equal(lat.gamma5(Xt).cpu().numpy(), dirac.apply_gamma5(X))
    for prec, tol in [("fp64", 0.0), ("fp32", 1e-7), ("fp16", 1e-3)]:
        back = lat.unpack(lat.pack(Xt, prec), 4, prec).cpu().numpy()
        assert _rel(back, X) <= tol


def test_dslash_dev_layout_single_launch():
    dims = (8, 8, 8, 8)
    lat, U = _lat(dims, 0.4, 11)
    X = synth.gaussian_sources(dims, 12, 2)
    F = lat.pack(torch.from_numpy(X).cuda(), "fp32")
    G = lat.dslash_dev(F, 12, 0.124, "fp32")
    Y = lat.unpack(G, 12, "fp32").cpu().numpy()
    assert _rel(Y, dirac.apply_dirac(U, X, 0.124, 1.0)) < TOL["fp32"]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-5), ("fp16", 2e-3)])
@pytest.mark.parametrize("L", [1, 3, 6, 8, 12, 13, 48, 50])
def test_gram_matches_numpy(prec, tol, L):
    dims = (4, 4, 4, 8)
    lat, _ = _lat(dims, 0.3, 1)
    A = synth.gaussian_sources(dims, L, 21)
    B = synth.z2_noise(dims, L, 22)
    Fa = lat.pack(torch.from_numpy(A).cuda(), prec)
    Fb = lat.pack(torch.from_numpy(B).cuda(), prec)
    G = lat.gram(Fa, Fb, L, prec).cpu().numpy()
    Am, Bm = A.reshape(L, -1).T, B.reshape(L, -1).T
    Gref = Am.conj().T @ Bm
    assert _rel(G, Gref) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32", 1e-6), ("fp16", 2e-3)])
def test_xmy_matches_numpy(prec, tol):
    dims = (4, 4, 4, 4)
    lat, _ = _lat(dims, 0.3, 1)
    L = 7
    X = synth.gaussian_sources(dims, L, 31)
    Z = synth.gaussian_sources(dims, L, 32)
    rng = np.random.default_rng(3)
    M = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    c = 0.3 - 0.7j
    Fx = lat.pack(torch.from_numpy(X).cuda(), prec)
    Fz = lat.pack(torch.from_numpy(Z).cuda(), prec)
    Fy = lat.xmy(Fx, torch.from_numpy(M).cuda(), L, c, Fz, prec)
    Y = lat.unpack(Fy, L, prec).cpu().numpy()
    ref = Z + c * np.einsum("i...,ij->j...", X, M)
    assert _rel(Y, ref) < tol


@pytest.mark.parametrize("L", [1, 3, 12, 48, 60, 96, 100, 128])
def test_small_solve_matches_numpy(L):
    import paper_0903_4936_gb300 as bk
    rng = np.random.default_rng(L)
    G = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    H = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    s = 0.5 + 2.0j
    X, info = bk.small_solve(torch.from_numpy(G).cuda(), torch.from_numpy(H).cuda(), s)
    assert info == 0
    ref = np.linalg.solve(G, s * H)
    assert _rel(X.cpu().numpy(), ref) < 1e-10


def test_small_solve_detects_singular():
    import paper_0903_4936_gb300 as bk
    rng = np.random.default_rng(0)
    G = rng.standard_normal((5, 5)) + 0j
    G[3] = G[1]
    X, info = bk.small_solve(torch.from_numpy(G).cuda(), torch.from_numpy(np.eye(5) + 0j).cuda())
    assert info > 0


def test_dslash_full_size_sampled_sites_fp16():
    """16^3 x 32, L = 12 point sources, FP16 storage: the launch shape the
    benchmark times; compared on sampled sites with the site-wise oracle."""
    dims = (16, 16, 16, 32)
    lat, U = _lat(dims, 0.5, 2003)
    X = synth.z2_noise(dims, 12, 5)
    Y = lat.dslash(torch.from_numpy(X).cuda(), 0.125, "fp16").cpu().numpy()
    V = 16 * 16 * 16 * 32
    sites = [0, 1, 15, 16, 255, 4095, 4096, V // 2 + 17, V - 4096, V - 1]
    ref = dirac.apply_dirac_at(U, X, 0.125, 1.0, sites, dims)
    got = Y.reshape(12, V, 4, 3)[:, sites]
    assert _rel(got, ref) < TOL["fp16"]


def test_df64_operator_tracks_fp64_where_fp32_cannot():
    """Double-float arithmetic on FP64-layout blocks: the residual B - A X of a
    nearly converged X (|B - A X| ~ 1e-9 |B|) agrees with the FP64 result to
    well below the residual itself, which FP32 arithmetic cannot resolve."""
    dims = (8, 8, 8, 8)
    lat, U = _lat(dims, 0.5, 77)
    B = synth.z2_noise(dims, 4, 3)
    Bt = torch.from_numpy(B).cuda()
    X, info = lat.block_solve(Bt, 0.124, prec="fp64", tol=1e-9, maxiter=2000)
    AX64 = lat.dslash(X, 0.124, "fp64").cpu().numpy()
    AXdd = lat.dslash(X, 0.124, "df64").cpu().numpy()
    AX32 = lat.dslash(X, 0.124, "fp32").cpu().numpy()
    r64, rdd, r32 = B - AX64, B - AXdd, B - AX32
    nb = np.linalg.norm(B)
    assert np.linalg.norm(r64) < 2e-9 * nb
    assert np.linalg.norm(rdd - r64) < 1e-3 * np.linalg.norm(r64)
    assert np.linalg.norm(r32 - r64) > 10 * np.linalg.norm(r64)


@pytest.mark.parametrize("variant", ["1", "2", "3", "1:1", "2:2", "2:3", "3:3", "4", "5"])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 12), ((2, 4, 2, 6), 5), ((3, 5, 4, 6), 1), ((8, 8, 8, 16), 13),
                                    ((4, 4, 4, 8), 21)])
def test_dslash_every_launch_variant(monkeypatch, variant, prec, dims, L):
    """Each register-cap variant of the packed-pair operator the autotuner may
    pick, with and without the L2 / L1 prefetch of its rows, in its looped
    form and in the FP32 staged form (variants 4, 5; FP16 runs variant 2's
    kernel for them) (forced with
    BK_DSLASH_VARIANT / BK_DSLASH_PREFETCH, pair groups of 8: L = 21 runs a full
    group of 8 pairs and a short one of 3) against the oracle; odd L leaves a
    padding column in the last pair.  On 4^4 the variant is also the inner operator of
    a mixed-precision solve."""
    import paper_0903_4936_gb300 as bk
    v, _, pf = variant.partition(":")
    monkeypatch.setenv("BK_DSLASH_VARIANT", v)
    monkeypatch.setenv("BK_DSLASH_PREFETCH", pf or "0")
    lat, U = _lat(dims, 0.5, 300 + L)
    X = synth.gaussian_sources(dims, L, 8)
    kappa = [0.115 + 0.001 * j for j in range(L)]
    Y = lat.dslash(torch.from_numpy(X).cuda(), kappa, prec).cpu().numpy()
    assert _rel(Y, dirac.apply_dirac(U, X, np.array(kappa), 1.0)) < TOL[prec]
    if dims == (4, 4, 4, 4) and prec == "fp32":
        B = torch.from_numpy(synth.z4_noise(dims, L, 9)).cuda()
        Xs, info = lat.block_solve(B, 0.12, method="bicgstab", prec="fp32", tol=1e-10, maxiter=1000)
        assert info["converged"] == 1 and info["true_res_max"] <= 1e-10
        R = B.cpu().numpy() - dirac.apply_dirac(U, Xs.cpu().numpy(), 0.12, 1.0)
        assert np.linalg.norm(R) <= 1e-10 * np.linalg.norm(B.cpu().numpy()) * np.sqrt(L)


def test_dslash_multi_and_set_clover():
    """bk_set_clover builds the clover term (FP64 operator against the oracle)
    and bk_dslash_multi (one kappa for all columns) gives bit for bit what
    bk_dslash and bk_dslash_dev give with kappa repeated, in both layouts."""
    import paper_0903_4936_gb300 as bk
    dims = (4, 4, 4, 6)
    U = synth.random_su3_field(dims, 0.5, 61)
    lat = bk.Lattice(dims)
    lat.upload_gauge(U)
    lat.set_clover(1.0)
    X = synth.gaussian_sources(dims, 5, 62)
    Xt = torch.from_numpy(X).cuda()
    Y1 = lat.dslash_multi(Xt, 0.121, prec="fp64").cpu().numpy()
    assert _rel(Y1, dirac.apply_dirac(U, X, 0.121, 1.0)) < TOL["fp64"]
    np.testing.assert_array_equal(Y1, lat.dslash(Xt, 0.121, "fp64").cpu().numpy())
    F = lat.pack(Xt, "fp32")
    G1 = lat.unpack(lat.dslash_multi(F, 0.121, L=5, prec="fp32", layout="device"), 5, "fp32").cpu().numpy()
    G2 = lat.unpack(lat.dslash_dev(F, 5, 0.121, "fp32"), 5, "fp32").cpu().numpy()
    np.testing.assert_array_equal(G1, G2)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("dims,L,kappas", [
    ((16, 16, 16, 32), 180, (0.120, 0.125, 0.130)),
    ((24, 24, 24, 48), 196, (0.120, 0.122, 0.124, 0.126, 0.128, 0.130)),
])
def test_dslash_benchmark_sizes_sampled_sites(prec, dims, L, kappas):
    """The benchmark's lattices and column counts (16^3 x 32 with 180 columns,
    24^3 x 48 with 196 columns), one launch over all columns at the launch
    shape the autotuner picks for that count, per-column kappa as in the
    batched solves.  Column j is c_j Z_(j mod 4): four Z4 noise fields times
    a distinct complex scale per column (D_W is linear), so every column
    differs and a column mix-up changes the result.  Compared on sampled sites
    (including lattice corners and the last site) with the oracle's site-wise
    operator."""
    lat, U = _lat(dims, 0.5, 1003 if dims[0] == 16 else 1004)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    Z = synth.z4_noise(dims, 4, 2048)
    j = np.arange(L)
    cj = (1.0 + j / L) * np.exp(2j * np.pi * j / L)
    kap = np.array([kappas[(jj * len(kappas)) // L] for jj in j])
    Zt = torch.from_numpy(Z).cuda()
    Xt = Zt[torch.from_numpy(j % 4).cuda()] * torch.from_numpy(cj).cuda().reshape((L,) + (1,) * 6)
    del Zt
    Y = lat.dslash(Xt.contiguous(), list(kap), prec)
    del Xt
    sites = [0, 1, dims[0] - 1, dims[0], V // 3 + 5, V // 2 + 17, V - dims[0] * dims[1] * dims[2], V - 1]
    got = Y.reshape(L, V, 4, 3)[:, sites].cpu().numpy()
    del Y
    err = 0.0
    for p in range(4):
        cols = j[j % 4 == p]
        Xp = np.broadcast_to(Z[p:p + 1], (len(cols),) + Z.shape[1:])
        ref = dirac.apply_dirac_at(U, Xp, kap[cols], 1.0, sites, dims) * cj[cols][:, None, None, None]
        err = max(err, _rel(got[cols], ref))
    assert err < TOL[prec], err
