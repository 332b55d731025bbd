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
