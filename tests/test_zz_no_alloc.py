"""bk_block_gram_noalloc: the Gram matrix without any device allocation.

Some callers cannot allocate device memory when they call in (they hand all
of HBM to their own pools up front, or cannot take the device-wide
synchronisation an allocation may cause).  For them the library offers a Gram
reduction whose scratch is a fixed device array.  This test calls it through
the C ABI twice in a row and checks each result against the allocating
bk_block_gram, with the tolerances the Gram tests use.  It lives in a file
pytest collects last, and sets up everything it needs itself.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "fp32": 1e-5, "fp16": 2e-3}


def _noalloc(V, A, B, L, prec):
    from paper_0903_4936_gb300 import _lib
    G = torch.empty((L, L), dtype=torch.complex128, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _lib.lib().bk_block_gram_noalloc(V, C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), L,
                                          _lib.PREC[prec], C.c_void_p(G.data_ptr()), st)
    _lib.check(rc, "bk_block_gram_noalloc")
    return G


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_noalloc_gram_matches_allocating_gram_twice(prec):
    import paper_0903_4936_gb300 as bk
    dims = (8, 8, 8, 16)
    lat = bk.Lattice(dims)
    lat.upload_gauge(synth.random_su3_field(dims, 0.3, 1))
    lat.build_clover(1.0)
    for call, (L, seed) in enumerate([(12, 1), (17, 2)]):
        A = lat.pack(torch.from_numpy(synth.gaussian_sources(dims, L, seed)).cuda(), prec)
        B = lat.pack(torch.from_numpy(synth.z2_noise(dims, L, seed + 10)).cuda(), prec)
        G_ref = lat.gram(A, B, L, prec).cpu().numpy()
        G = _noalloc(lat.V, A, B, L, prec).cpu().numpy()
        err = np.max(np.abs(G - G_ref)) / np.max(np.abs(G_ref))
        assert err < TOL[prec], (call, err)


@pytest.mark.parametrize("L", [361, 400, 185000, 262141, 262144, 2**31 - 1])
def test_noalloc_gram_rejects_too_large_L(L):
    # Sizes whose tile count would overflow or wrap in int arithmetic must be
    # rejected before any tiling or launch, as the plain too-large case is.
    from paper_0903_4936_gb300 import _lib
    import paper_0903_4936_gb300 as bk
    dims = (4, 4, 4, 4)
    lat = bk.Lattice(dims)
    A = torch.zeros(16, dtype=torch.uint8, device="cuda")
    G = torch.empty((1,), dtype=torch.complex128, device="cuda")
    rc = _lib.lib().bk_block_gram_noalloc(lat.V, C.c_void_p(A.data_ptr()), C.c_void_p(A.data_ptr()), L,
                                          _lib.PREC["fp32"], C.c_void_p(G.data_ptr()),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1  # BK_ERR_INVALID_ARG
    assert b"L <= 360" in _lib.lib().bk_last_error()
