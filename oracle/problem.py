"""Build the oracle's objects for a synthetic workload (test infrastructure only)."""
from __future__ import annotations

from .geometry import Mesh
from .multigrid import Hierarchy
from .mixed import MixedSystem


def pressure_hierarchy(cfg, inp, levels: int | None = None) -> Hierarchy:
    """Helmholtz hierarchy of the pressure-only workload (Sec. 3.5-3.6)."""
    return Hierarchy(cfg.n, inp["z_if"], cfg.radius, levels or cfg.levels, inp["g"],
                     cfg.cs * cfg.dt, gamma2=cfg.gamma2)


TAU_U = 0.5     # off-centring of the velocity equation (Sec. 3.3, tau_u = 1/2)


def mixed_problem(cfg, inp, levels: int | None = None):
    """(MixedSystem, Hierarchy of its Schur-complement Helmholtz operator) (Sec. 3.4).

    The Coriolis factor of Eq. M2muCdef is f0 = tau_u dt 2 Omega."""
    mesh = Mesh(cfg.n, inp["z_if"], cfg.radius)
    f0 = TAU_U * cfg.dt * 2.0 * cfg.rotation
    S = MixedSystem(mesh, inp["g"], cfg.cs * cfg.dt, inp["beta_up"], inp["beta_dn"], cfg.eps,
                    consistent=cfg.consistent_mass, f0=f0)
    hier = Hierarchy(cfg.n, inp["z_if"], cfg.radius, levels or cfg.levels, inp["g"],
                     cfg.cs * cfg.dt, mu=S.mu, mu_h=S.mu_h)
    return S, hier
