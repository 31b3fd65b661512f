"""Scalar BiCGSTAB, block BiCGSTAB and block BiCGGR (Section 3 of arXiv:0903.4936).

Each solver follows the steps of the paper's algorithm in the paper's order
and notation.  Blocks are N x L complex matrices (columns = right-hand
sides); ``A`` is any callable mapping an N x L matrix to A times it.

Readings of points the paper leaves open:

* inner product (x, y) = x^H y; Tr(Z^H T) = sum_i z_i^H t_i; zeta is complex;
* X_0 = 0 unless given; R~_0 = R_0 unless given;
* the stopping test max_i ||r_k^(i)|| / ||b^(i)|| <= eps is evaluated on the
  recursively updated residual before every iteration, including k = 0;
  ``iterations`` counts completed loop bodies;
* L x L systems are solved with LU and partial pivoting (numpy.linalg.solve);
* BiCGGR's gamma_k system has matrix R~_0^H R_k (the residual before the
  update) and right-hand side R~_0^H R_{k+1} divided by the scalar zeta_k.

Matvec counts: 2 per iteration, +1 for R_0 when X_0 is given, +1 for
V_0 = W_0 = A R_0 in BiCGGR.
"""
from __future__ import annotations

import numpy as np

__all__ = ["bicgstab", "block_bicgstab", "block_bicggr", "true_residual"]


def _hdot(x, y):
    return np.vdot(x, y)


def _colnorms(M):
    return np.linalg.norm(M, axis=0)


def true_residual(A, B, X):
    """max_i ||A x_i - b_i|| / ||b_i|| and the per-column values (Section 4.3)."""
    r = _colnorms(A(X) - B) / _colnorms(B)
    return float(np.max(r)), r


def bicgstab(A, b, tol, maxiter, x0=None, rt=None):
    """Single right-hand side BiCGSTAB; b and x are N-vectors (N x 1 for A)."""
    Av = lambda v: A(v.reshape(-1, 1)).reshape(-1)  # noqa: E731
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    matvecs = 0
    if x0 is None:
        r = b.copy()
    else:
        r = b - Av(x)
        matvecs += 1
    p = r.copy()
    rt = r.copy() if rt is None else np.asarray(rt, dtype=np.complex128).reshape(-1)
    bnorm = np.linalg.norm(b)
    hist = []
    k = 0
    converged = False
    while True:
        res = np.linalg.norm(r) / bnorm
        hist.append(res)
        if res <= tol:
            converged = True
            break
        if k >= maxiter:
            break
        Ap = Av(p)
        alpha = _hdot(rt, r) / _hdot(rt, Ap)
        t = r - alpha * Ap
        At = Av(t)
        zeta = _hdot(At, t) / _hdot(At, At)
        x = x + alpha * p + zeta * t
        r_new = t - zeta * At
        beta = (alpha / zeta) * _hdot(rt, r_new) / _hdot(rt, r)
        p = r_new + beta * (p - zeta * Ap)
        r = r_new
        matvecs += 2
        k += 1
    return x, dict(iterations=k, matvecs=matvecs, converged=converged,
                   history=np.array(hist), rec_res=np.array([hist[-1]]))


def _start(A, B, X0, Rt):
    B = np.asarray(B, dtype=np.complex128)
    matvecs = 0
    if X0 is None:
        X = np.zeros_like(B)
        R = B.copy()
    else:
        X = np.array(X0, dtype=np.complex128)
        R = B - A(X)
        matvecs += 1
    Rt = R.copy() if Rt is None else np.asarray(Rt, dtype=np.complex128)
    return B, X, R, Rt, matvecs


def block_bicgstab(A, B, tol, maxiter, X0=None, Rt=None):
    """Block BiCGSTAB, Section 3.  Returns (X, info)."""
    B, X, R, Rt, matvecs = _start(A, B, X0, Rt)
    bnorm = _colnorms(B)
    P = R.copy()
    RtH = Rt.conj().T
    hist, k, converged, breakdown = [], 0, False, False
    while True:
        rel = _colnorms(R) / bnorm
        hist.append(float(np.max(rel)))
        if hist[-1] <= tol:
            converged = True
            break
        if k >= maxiter:
            break
        V = A(P)
        G = RtH @ V
        alpha = np.linalg.solve(G, RtH @ R)
        T = R - V @ alpha
        Z = A(T)
        zeta = np.trace(Z.conj().T @ T) / np.trace(Z.conj().T @ Z)
        X = X + P @ alpha + zeta * T
        R = T - zeta * Z
        beta = np.linalg.solve(G, -(RtH @ Z))
        P = R + (P - zeta * V) @ beta
        matvecs += 2
        k += 1
        if not (np.all(np.isfinite(alpha)) and np.all(np.isfinite(beta)) and np.isfinite(zeta)):
            breakdown = True
            break
    return X, dict(iterations=k, matvecs=matvecs, converged=converged, breakdown=breakdown,
                   history=np.array(hist), rec_res=_colnorms(R) / bnorm)


def block_bicggr(A, B, tol, maxiter, X0=None, Rt=None):
    """Block BiCGGR (the method of Ref. alg_tadano as given in Section 3)."""
    B, X, R, Rt, matvecs = _start(A, B, X0, Rt)
    bnorm = _colnorms(B)
    P = R.copy()
    W = A(R)
    V = W.copy()
    matvecs += 1
    RtH = Rt.conj().T
    hist, k, converged, breakdown = [], 0, False, False
    while True:
        rel = _colnorms(R) / bnorm
        hist.append(float(np.max(rel)))
        if hist[-1] <= tol:
            converged = True
            break
        if k >= maxiter:
            break
        G_RR = RtH @ R
        alpha = np.linalg.solve(RtH @ V, G_RR)
        zeta = np.trace(W.conj().T @ R) / np.trace(W.conj().T @ W)
        S = P - zeta * V
        Ublk = S @ alpha
        Y = A(Ublk)
        X = X + zeta * R + Ublk
        R_new = R - zeta * W - Y
        W_new = A(R_new)
        gamma = np.linalg.solve(G_RR, (RtH @ R_new) / zeta)
        P = R_new + Ublk @ gamma
        V = W_new + Y @ gamma
        R, W = R_new, W_new
        matvecs += 2
        k += 1
        if not (np.all(np.isfinite(alpha)) and np.all(np.isfinite(gamma)) and np.isfinite(zeta)):
            breakdown = True
            break
    return X, dict(iterations=k, matvecs=matvecs, converged=converged, breakdown=breakdown,
                   history=np.array(hist), rec_res=_colnorms(R) / bnorm)
