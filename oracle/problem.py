"""Build the oracle's objects for a synthetic workload (test infrastructure only)."""
from __future__ import annotations

from .geometry import Mesh
from .multigrid import Hierarchy
from .mixed import MixedSystem


def pressure_hierarchy(cfg, inp, levels: int | None = None) -> Hierarchy:
    """Helmholtz hierarchy of the pressure-only workload (Sec. 3.5-3.6)."""
    return Hierarchy(cfg.n, inp["z_if"], cfg.radius, levels or cfg.levels, inp["g"],
                     cfg.cs * cfg.dt)


def mixed_problem(cfg, inp, levels: int | None = None):
    """(MixedSystem, Hierarchy of its Schur-complement Helmholtz operator) (Sec. 3.4)."""
    mesh = Mesh(cfg.n, inp["z_if"], cfg.radius)
    S = MixedSystem(mesh, inp["g"], cfg.cs * cfg.dt, inp["beta_up"], inp["beta_dn"], cfg.eps)
    hier = Hierarchy(cfg.n, inp["z_if"], cfg.radius, levels or cfg.levels, inp["g"],
                     cfg.cs * cfg.dt, mu=S.mu)
    return S, hier
