"""GB300 block Krylov solvers for the O(a)-improved Wilson-Dirac equation.

Thin Python binding over the C ABI of ``libbkrylov.so`` (``include/bkrylov.h``):
argument marshalling only, every step runs in the library's CUDA kernels.
PyTorch provides device memory and the current CUDA stream.

Method: Sakurai, Tadano, Kuramashi, arXiv:0903.4936 -- the clover Wilson-Dirac
operator D_W (Eq. (wd-op)), block BiCGSTAB and block BiCGGR (Section 3).

Layouts (canonical, what the user passes):
  * gauge  U: complex128 tensor [4, Lt, Lz, Ly, Lx, 3, 3]  (mu = x, y, z, t)
  * blocks X: complex128 tensor [L, Lt, Lz, Ly, Lx, 4, 3]  (column, site, spin, colour)
"""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import torch

from . import _lib
from ._lib import BKError, PREC, METHOD, SolveInfo, SolveParams, check, lib

__all__ = ["Lattice", "BKError", "PREC", "METHOD", "load", "block_solve_autograd", "small_solve", "probe_peak"]


def load():
    """Load libbkrylov.so (raises ImportError if it has not been built)."""
    return lib()


def _stream_ptr(device) -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


class Lattice:
    """A lattice with its gauge field and clover term on one GPU.

    ``dims = (Lx, Ly, Lz, Lt)``; periodic boundaries in every direction.
    """

    def __init__(self, dims: Sequence[int], device: int | torch.device = 0):
        self.dims = tuple(int(d) for d in dims)
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.V = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        L = lib()
        arr = (C.c_int * 4)(*self.dims)
        h = C.c_void_p()
        check(L.bk_create(arr, self.device.index or 0, C.byref(h)), "bk_create")
        self._h = h
        self.csw = None

    def close(self):
        if getattr(self, "_h", None):
            lib().bk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ shapes
    @property
    def lat_shape(self):
        Lx, Ly, Lz, Lt = self.dims
        return (Lt, Lz, Ly, Lx)

    def block_shape(self, L: int):
        return (L,) + self.lat_shape + (4, 3)

    def _check_block(self, X: torch.Tensor, name: str):
        if X.dtype != torch.complex128 or not X.is_contiguous() or X.shape[1:] != self.block_shape(1)[1:]:
            raise ValueError(f"{name} must be a contiguous complex128 tensor of shape {self.block_shape(-1)}")

    # ------------------------------------------------------------ set-up
    def upload_gauge(self, U):
        """U: complex128 [4, Lt, Lz, Ly, Lx, 3, 3] (numpy array or torch tensor)."""
        if not isinstance(U, torch.Tensor):
            U = torch.from_numpy(U)
        U = U.to(torch.complex128).contiguous()
        if tuple(U.shape) != (4,) + self.lat_shape + (3, 3):
            raise ValueError("gauge field shape must be [4, Lt, Lz, Ly, Lx, 3, 3]")
        on_dev = U.is_cuda
        check(lib().bk_upload_gauge(self._h, _ptr(U), int(on_dev), _stream_ptr(self.device)), "bk_upload_gauge")
        if on_dev:
            torch.cuda.current_stream(self.device).synchronize()

    def build_clover(self, csw: float):
        check(lib().bk_build_clover(self._h, float(csw), _stream_ptr(self.device)), "bk_build_clover")
        self.csw = float(csw)

    def set_clover(self, csw: float):
        """build_clover on the default stream, synchronously (bk_set_clover)."""
        check(lib().bk_set_clover(self._h, float(csw)), "bk_set_clover")
        self.csw = float(csw)

    # ------------------------------------------------------------ operator
    def _kappas(self, kappa, L):
        if isinstance(kappa, (int, float)):
            ks = [float(kappa)] * L
        else:
            ks = [float(k) for k in kappa]
            if len(ks) != L:
                raise ValueError("one kappa per column expected")
        return (C.c_double * L)(*ks)

    def dslash(self, X: torch.Tensor, kappa, prec="fp64", out: torch.Tensor | None = None) -> torch.Tensor:
        """Y = D_W X (Eq. (wd-op)) for every column, computed in `prec`."""
        self._check_block(X, "X")
        L = X.shape[0]
        Y = torch.empty_like(X) if out is None else out
        check(lib().bk_dslash(self._h, self._kappas(kappa, L), _ptr(X), _ptr(Y), L, _prec(prec),
                              _stream_ptr(self.device)), "bk_dslash")
        return Y

    def schur_dslash(self, X: torch.Tensor, kappa, prec="fp64", out: torch.Tensor | None = None) -> torch.Tensor:
        """Y_e = M X_e, the even-odd Schur operator (bk_schur_dslash): Y is zero
        on the odd sites and the odd sites of X are ignored."""
        self._check_block(X, "X")
        L = X.shape[0]
        Y = torch.empty_like(X) if out is None else out
        check(lib().bk_schur_dslash(self._h, self._kappas(kappa, L), _ptr(X), _ptr(Y), L, _prec(prec),
                                    _stream_ptr(self.device)), "bk_schur_dslash")
        return Y

    def dslash_multi(self, X: torch.Tensor, kappa: float, L: int | None = None, prec="fp64", layout="canonical",
                     out: torch.Tensor | None = None) -> torch.Tensor:
        """Y = D_W X with one kappa for every column (bk_dslash_multi).  layout
        "canonical": X a canonical block (L from its shape); "device": X a
        device-layout block of L columns in prec."""
        if layout == "canonical":
            self._check_block(X, "X")
            L = X.shape[0]
            Y = torch.empty_like(X) if out is None else out
        elif layout == "device":
            if L is None:
                raise ValueError("device layout needs L")
            Y = self.empty_field(L, "fp64" if prec == "df64" else prec) if out is None else out
        else:
            raise ValueError("layout must be 'canonical' or 'device'")
        check(lib().bk_dslash_multi(self._h, float(kappa), _ptr(X), _ptr(Y), int(L), _prec(prec),
                                    _lib.LAYOUT[layout], _stream_ptr(self.device)), "bk_dslash_multi")
        return Y

    def gamma5(self, X: torch.Tensor) -> torch.Tensor:
        self._check_block(X, "X")
        Y = torch.empty_like(X)
        check(lib().bk_gamma5(self._h, _ptr(X), _ptr(Y), X.shape[0], _stream_ptr(self.device)), "bk_gamma5")
        return Y

    # ------------------------------------------------------------ device-layout blocks
    def field_bytes(self, L: int, prec="fp64") -> int:
        return int(lib().bk_field_bytes(self._h, L, _prec(prec)))

    def empty_field(self, L: int, prec="fp64") -> torch.Tensor:
        return torch.empty(self.field_bytes(L, prec), dtype=torch.uint8, device=self.device)

    def pack(self, X: torch.Tensor, prec="fp64") -> torch.Tensor:
        self._check_block(X, "X")
        F = self.empty_field(X.shape[0], prec)
        check(lib().bk_pack(self._h, _ptr(X), _ptr(F), X.shape[0], _prec(prec), _stream_ptr(self.device)), "bk_pack")
        return F

    def unpack(self, F: torch.Tensor, L: int, prec="fp64") -> torch.Tensor:
        X = torch.empty(self.block_shape(L), dtype=torch.complex128, device=self.device)
        check(lib().bk_unpack(self._h, _ptr(F), _ptr(X), L, _prec(prec), _stream_ptr(self.device)), "bk_unpack")
        return X

    def dslash_dev(self, F: torch.Tensor, L: int, kappa, prec="fp64", out: torch.Tensor | None = None):
        """Operator on device-layout blocks (one kernel launch)."""
        Y = self.empty_field(L, prec) if out is None else out
        check(lib().bk_dslash_dev(self._h, self._kappas(kappa, L), _ptr(F), _ptr(Y), L, _prec(prec),
                                  _stream_ptr(self.device)), "bk_dslash_dev")
        return Y

    def gram(self, A: torch.Tensor, B: torch.Tensor, L: int, prec="fp64") -> torch.Tensor:
        """G = A^H B (L x L complex128) of two device-layout blocks."""
        G = torch.empty((L, L), dtype=torch.complex128, device=self.device)
        check(lib().bk_block_gram(self._h, _ptr(A), _ptr(B), L, _prec(prec), _ptr(G), _stream_ptr(self.device)),
              "bk_block_gram")
        return G

    def xmy(self, X: torch.Tensor, M: torch.Tensor, L: int, c=1.0, Z: torch.Tensor | None = None, prec="fp64"):
        """Y = Z + c (X M) on device-layout blocks; M is L x L complex128 (cuda)."""
        M = M.to(torch.complex128).contiguous()
        Y = self.empty_field(L, prec)
        cc = (C.c_double * 2)(complex(c).real, complex(c).imag)
        check(lib().bk_block_xmy(self._h, _ptr(X), _ptr(M), cc, _ptr(Z) if Z is not None else None, _ptr(Y), L,
                                 _prec(prec), _stream_ptr(self.device)), "bk_block_xmy")
        return Y

    def dot(self, A: torch.Tensor, B: torch.Tensor) -> complex:
        """sum conj(A) B over two canonical blocks (FP64 device reduction)."""
        self._check_block(A, "A")
        self._check_block(B, "B")
        r = (C.c_double * 2)()
        check(lib().bk_dot(self._h, _ptr(A), _ptr(B), A.shape[0], r, _stream_ptr(self.device)), "bk_dot")
        return complex(r[0], r[1])

    def kappa_grad(self, Lam: torch.Tensor, X: torch.Tensor, B: torch.Tensor, kappa: float) -> float:
        """Re sum conj(Lam) (X - B) / kappa (bk_kappa_grad): dLoss/dkappa for
        X = D_W^-1 B and Lam the adjoint solution."""
        for t, n in ((Lam, "Lam"), (X, "X"), (B, "B")):
            self._check_block(t, n)
        r = C.c_double()
        check(lib().bk_kappa_grad(self._h, float(kappa), _ptr(Lam), _ptr(X), _ptr(B), X.shape[0], C.byref(r),
                                  _stream_ptr(self.device)), "bk_kappa_grad")
        return r.value

    def gauge_force(self, X: torch.Tensor, Lam: torch.Tensor, mode=0, scale=1.0) -> torch.Tensor:
        """Link derivative of Re sum <Lam, (H + C) X> (see bk_gauge_force).
        mode 0/1: complex128 [4, V, 3, 3] (Sigma / Sigma^+); mode 2: float64 [4, V, 8]."""
        self._check_block(X, "X")
        self._check_block(Lam, "Lam")
        if mode == 2:
            out = torch.empty((4, self.V, 8), dtype=torch.float64, device=self.device)
        else:
            out = torch.empty((4, self.V, 3, 3), dtype=torch.complex128, device=self.device)
        check(lib().bk_gauge_force(self._h, _ptr(X), _ptr(Lam), X.shape[0], int(mode), float(scale), _ptr(out),
                                   _stream_ptr(self.device)), "bk_gauge_force")
        return out

    # ------------------------------------------------------------ solves
    def _params(self, method, prec, tol, maxiter, delta, x0_given, on_host, rtilde, seed, history, timing,
                restart=False, orth=None, update="fp64", deflate=False, eo=False, anchor=0.0):
        """rtilde: None -> seeded Gaussian R~_0 (library default), "r0" -> R~_0 = R_0,
        tensor -> the caller's block (canonical layout, where B lives).  update:
        arithmetic of the mixed-precision residual replacements, "df64" or "fp64".
        eo: iterate on the even-odd Schur system (bk_solve_params.eo).  anchor:
        bk_solve_params.fp64_anchor (replacements between FP64 ones in FP32)."""
        if update not in ("df64", "fp64"):
            raise ValueError("update must be 'df64' or 'fp64'")
        mode, ptr = 0, None
        if isinstance(rtilde, str):
            if rtilde != "r0":
                raise ValueError("rtilde must be None, 'r0' or a block")
            mode = 1
        elif rtilde is not None:
            mode, ptr = 2, C.c_void_p(rtilde.data_ptr())
        return SolveParams(METHOD[method] if isinstance(method, str) else int(method), _prec(prec), float(tol),
                           int(maxiter), float(delta), int(x0_given), int(on_host), mode, int(seed), ptr,
                           int(bool(restart)), 0 if orth is None else (1 if orth else 2), int(history),
                           int(timing), 1 if update == "df64" else 0, int(bool(deflate)), int(bool(eo)),
                           float(anchor))

    @staticmethod
    def _info_dict(info: SolveInfo, hist_buf, res_buf):
        d = {f: getattr(info, f) for f, _ in SolveInfo._fields_ if f not in ("true_res", "history")}
        d["true_res"] = list(res_buf) if res_buf is not None else None
        d["history"] = list(hist_buf[: info.history_len]) if hist_buf is not None else None
        return d

    def block_solve(self, B: torch.Tensor, kappa: float, method="bicggr", prec="fp64", tol=1e-10, maxiter=2000,
                    X0: torch.Tensor | None = None, delta=0.0, rtilde=None, seed=0, history=False,
                    timing=False, out: torch.Tensor | None = None, raise_on_fail=True, restart=False,
                    orth=None, update="fp64", deflate=False, eo=False, anchor=0.0):
        """Solve D_W X = B (Eq. (linear_mrhs)).  B on the GPU, or on the host
        (then pinned memory is best): X is returned where B lives."""
        self._check_block(B, "B")
        L = B.shape[0]
        on_host = not B.is_cuda
        X = (torch.empty_like(B, pin_memory=on_host) if on_host else torch.empty_like(B)) if out is None else out
        if X0 is not None:
            X.copy_(X0)
        if rtilde is not None and not isinstance(rtilde, str):
            self._check_block(rtilde, "rtilde")
            if rtilde.shape != B.shape or rtilde.is_cuda != B.is_cuda:
                raise ValueError("rtilde must have B's shape and location")
        prm = self._params(method, prec, tol, maxiter, delta, X0 is not None, on_host, rtilde, seed, history,
                           timing, restart, orth, update, deflate, eo, anchor)
        info = SolveInfo()
        res_buf = (C.c_double * L)()
        info.true_res = C.cast(res_buf, C.POINTER(C.c_double))
        hist_buf = (C.c_double * (maxiter + 1))() if history else None
        if hist_buf is not None:
            info.history = C.cast(hist_buf, C.POINTER(C.c_double))
        st = lib().bk_block_solve(self._h, C.byref(prm), float(kappa), _ptr(B), _ptr(X), L, C.byref(info),
                                  _stream_ptr(self.device))
        d = self._info_dict(info, hist_buf, res_buf)
        d["status"] = _lib.STATUS_NAMES.get(st, st)
        if raise_on_fail:
            check(st, "bk_block_solve")
        return X, d

    def block_solve_batched(self, B: torch.Tensor, kappas: Sequence[float], Ls: Sequence[int], method="bicggr",
                            prec="fp64", tol=1e-10, maxiter=2000, delta=0.0, rtilde=None, seed=0, history=False,
                            timing=False, raise_on_fail=True, restart=False, orth=None, update="fp64",
                            out: torch.Tensor | None = None, deflate=False, eo=False, anchor=0.0):
        """Several systems (kappa_s, L_s columns each, concatenated in B).  X is
        returned where B lives, in `out` if given (same shape and location as
        B; pinned host memory for host blocks)."""
        self._check_block(B, "B")
        nsys = len(Ls)
        if sum(Ls) != B.shape[0] or len(kappas) != nsys:
            raise ValueError("B must hold sum(Ls) columns and one kappa per system")
        on_host = not B.is_cuda
        if out is not None:
            self._check_block(out, "out")
            if out.shape != B.shape or out.is_cuda != B.is_cuda:
                raise ValueError("out must have B's shape and location")
            X = out
        else:
            X = torch.empty_like(B, pin_memory=on_host) if on_host else torch.empty_like(B)
        prm = self._params(method, prec, tol, maxiter, delta, False, on_host, rtilde, seed, history, timing,
                           restart, orth, update, deflate, eo, anchor)
        infos = (SolveInfo * nsys)()
        res_bufs, hist_bufs = [], []
        for s in range(nsys):
            rb = (C.c_double * Ls[s])()
            res_bufs.append(rb)
            infos[s].true_res = C.cast(rb, C.POINTER(C.c_double))
            if history:
                hb = (C.c_double * (maxiter + 1))()
                hist_bufs.append(hb)
                infos[s].history = C.cast(hb, C.POINTER(C.c_double))
            else:
                hist_bufs.append(None)
        ks = (C.c_double * nsys)(*[float(k) for k in kappas])
        ls = (C.c_int * nsys)(*[int(x) for x in Ls])
        st = lib().bk_block_solve_batched(self._h, C.byref(prm), nsys, ks, ls, _ptr(B), _ptr(X), infos,
                                          _stream_ptr(self.device))
        out = [self._info_dict(infos[s], hist_bufs[s], res_bufs[s]) for s in range(nsys)]
        for d in out:
            d["status"] = _lib.STATUS_NAMES.get(st, st)
        if raise_on_fail:
            check(st, "bk_block_solve_batched")
        return X, out


class _BlockSolve(torch.autograd.Function):
    """X = D_W(U, kappa)^-1 B with the adjoint of Section 3's solve.

    backward: lam = D^-H g = gamma_5 D^-1 gamma_5 g (gamma_5-hermiticity of
    D_W), grad_B = lam, grad_kappa from bk_kappa_grad (Re <lam, X - B> / kappa,
    since D = 1 - kappa M), grad_U = kappa Sigma^+ from bk_gauge_force.  The
    adjoint solve recomputes, it stores no Krylov history."""

    @staticmethod
    def forward(ctx, B, kappa, U, lat, csw, method, prec, tol, maxiter):
        lat.upload_gauge(U.detach())
        lat.build_clover(csw)
        k = float(kappa)
        X, info = lat.block_solve(B.detach().contiguous(), k, method=method, prec=prec, tol=tol, maxiter=maxiter)
        ctx.save_for_backward(B.detach(), X, U.detach())
        ctx.lat, ctx.csw, ctx.k = lat, csw, k
        ctx.opts = dict(method=method, prec=prec, tol=tol, maxiter=maxiter)
        return X

    @staticmethod
    def backward(ctx, gX):
        B, X, U = ctx.saved_tensors
        lat, k = ctx.lat, ctx.k
        lat.upload_gauge(U)
        lat.build_clover(ctx.csw)
        Z, _ = lat.block_solve(lat.gamma5(gX.contiguous()), k, **ctx.opts)
        lam = lat.gamma5(Z)
        gB = lam if ctx.needs_input_grad[0] else None
        gk = None
        if ctx.needs_input_grad[1]:
            gk = torch.tensor(lat.kappa_grad(lam, X, B, k), dtype=torch.float64, device=X.device)
        gU = None
        if ctx.needs_input_grad[2]:
            gU = lat.gauge_force(X, lam, mode=1, scale=k).reshape(U.shape)
        return gB, gk, gU, None, None, None, None, None, None


def block_solve_autograd(lat: "Lattice", B: torch.Tensor, kappa: torch.Tensor, U: torch.Tensor, csw: float,
                         method="bicggr", prec="fp64", tol=1e-12, maxiter=5000) -> torch.Tensor:
    """Differentiable X = D_W^-1 B with respect to B, kappa (0-d float64 tensor)
    and the gauge field U (complex128 [4, Lt, Lz, Ly, Lx, 3, 3])."""
    return _BlockSolve.apply(B, kappa, U, lat, csw, method, prec, tol, maxiter)


def small_solve(G: torch.Tensor, H: torch.Tensor, scale=1.0):
    """Solve G X = scale * H for L x L complex128 CUDA matrices (FP64 LU)."""
    L = G.shape[0]
    G = G.to(torch.complex128).contiguous()
    H = H.to(torch.complex128).contiguous()
    Xs = torch.empty_like(G)
    info = torch.zeros(1, dtype=torch.int32, device=G.device)
    cc = (C.c_double * 2)(complex(scale).real, complex(scale).imag)
    check(lib().bk_small_solve(L, _ptr(G), _ptr(H), cc, _ptr(Xs), _ptr(info), _stream_ptr(G.device)),
          "bk_small_solve")
    return Xs, int(info.item())


def probe_peak(kind: str = "fp32", device: int = 0) -> float:
    """Measured arithmetic peak of the GPU in TFLOP/s (bk_probe_peak):
    kind "fp32" (FMA), "fp32x2" (packed FMA) or "fp64" (FMA)."""
    k = {"fp32": 0, "fp32x2": 1, "fp64": 2}[kind]
    r = C.c_double()
    check(lib().bk_probe_peak(k, int(device), C.byref(r)), "bk_probe_peak")
    return r.value
