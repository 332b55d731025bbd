"""Restarted, right-preconditioned GCR (oracle).

Test infrastructure only.  The paper solves the mixed system with GCR (Sec. 4.1 solver
list; Sec. 5.1, outer tolerance 1e-6, following Melvin et al. 2018) and uses the same
solver framework K(A, P, eps) for the pressure system (Eq. solver_notation).  The paper
does not print the GCR recurrences; this is the textbook generalised conjugate residual
method (Eisenstat, Elman & Schultz 1983) with right preconditioning and restart after
``restart`` directions:

    x = 0, r = b
    repeat:  z = P r,  w = A z
             for each stored (z_j, w_j):  beta = <w, w_j>/<w_j, w_j>,
                                          w -= beta w_j,  z -= beta z_j   (modified G-S)
             alpha = <r, w>/<w, w>,  x += alpha z,  r -= alpha w
             store (z, w); clear the store after ``restart`` directions
    until ||r||_2 <= tol ||b||_2.

The recursively updated r is the true residual in exact arithmetic; ``gcr`` also
returns the history of ||r|| / ||b||.
"""
from __future__ import annotations

from typing import Callable

import numpy as np


class GCR:
    """The iteration above, one step at a time: ``step()`` does one GCR iteration and
    returns the new ||r|| / ||b||."""

    def __init__(self, A: Callable, b: np.ndarray, P: Callable | None = None, restart: int = 5):
        self.A = A
        self.P = (lambda v: v) if P is None else P
        self.b = np.asarray(b, dtype=np.float64).ravel()
        self.restart = restart
        self.x = np.zeros_like(self.b)
        self.r = self.b.copy()
        self.nb = np.linalg.norm(self.b)
        self.Z, self.W, self.WW = [], [], []

    def step(self) -> float:
        z = np.asarray(self.P(self.r), dtype=np.float64).ravel().copy()
        w = np.asarray(self.A(z), dtype=np.float64).ravel().copy()
        for zj, wj, wwj in zip(self.Z, self.W, self.WW):
            beta = np.dot(w, wj) / wwj
            w -= beta * wj
            z -= beta * zj
        ww = np.dot(w, w)
        if not np.isfinite(ww) or ww == 0.0:
            raise FloatingPointError("GCR breakdown: <w, w> = %r" % ww)
        alpha = np.dot(self.r, w) / ww
        self.x += alpha * z
        self.r -= alpha * w
        if len(self.Z) + 1 >= self.restart:
            self.Z, self.W, self.WW = [], [], []
        else:
            self.Z.append(z)
            self.W.append(w)
            self.WW.append(ww)
        return np.linalg.norm(self.r) / self.nb


def gcr(A: Callable, b: np.ndarray, P: Callable | None = None, tol: float = 1e-8,
        restart: int = 5, maxiter: int = 500):
    """Solve A x = b; returns (x, iterations, relative residual history)."""
    g = GCR(A, b, P, restart)
    hist = [1.0]
    if g.nb == 0.0:
        return g.x, 0, hist
    it = 0
    while it < maxiter:
        hist.append(g.step())
        it += 1
        if hist[-1] <= tol:
            break
    return g.x, it, hist


def bicgstab(A: Callable, b: np.ndarray, P: Callable | None = None, tol: float = 1e-8,
             maxiter: int = 500):
    """BiCGStab(A, P, eps) of the solver list of Sec. 4.1, used in Table 1 as the pressure solver
    K_H of the "Krylov" and "Krylov-MG" configurations.  The paper does not print the
    recurrences; this is van der Vorst's stabilised biconjugate gradient method (SIAM J. Sci.
    Stat. Comput. 13, 1992) with the preconditioner applied on the right, x0 = 0 and the shadow
    residual r^ = r0 = b:

        rho = <r^, r>;  p = r + (rho / rho_old)(alpha / omega)(p - omega v)   (p = r first)
        p^ = P p,  v = A p^,  alpha = rho / <r^, v>,  s = r - alpha v
        stop with x += alpha p^ if ||s|| <= tol ||b||                          (half step)
        s^ = P s,  t = A s^,  omega = <t, s> / <t, t>
        x += alpha p^ + omega s^,  r = s - omega t,  stop if ||r|| <= tol ||b||

    Each full step applies A and P twice (the cost 2 n_iter (C_H + C_Hz) + C_H of Sec. 3.7).
    Returns (x, iterations with a half step counted as 0.5, history of ||r|| / ||b||)."""
    P = (lambda v: v) if P is None else P
    b = np.asarray(b, dtype=np.float64).ravel()
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    hist = [1.0]
    if nb == 0.0:
        return x, 0.0, hist
    r = b.copy()
    rh = b.copy()
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho_old = alpha = omega = 1.0
    it = 0.0
    for i in range(maxiter):
        rho = np.dot(rh, r)
        if rho == 0.0 or not np.isfinite(rho):
            raise FloatingPointError("BiCGStab breakdown: <r^, r> = %r" % rho)
        p = r.copy() if i == 0 else r + (rho / rho_old) * (alpha / omega) * (p - omega * v)
        ph = np.asarray(P(p), dtype=np.float64).ravel()
        v = np.asarray(A(ph), dtype=np.float64).ravel()
        alpha = rho / np.dot(rh, v)
        s = r - alpha * v
        ns = np.linalg.norm(s) / nb
        if ns <= tol:
            x = x + alpha * ph
            hist.append(ns)
            return x, it + 0.5, hist
        sh = np.asarray(P(s), dtype=np.float64).ravel()
        t = np.asarray(A(sh), dtype=np.float64).ravel()
        omega = np.dot(t, s) / np.dot(t, t)
        if omega == 0.0 or not np.isfinite(omega):
            raise FloatingPointError("BiCGStab breakdown: omega = %r" % omega)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho_old = rho
        it += 1.0
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            break
    return x, it, hist
