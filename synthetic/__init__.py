"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module only draws random numbers and lays out the input arrays of a workload: it
contains none of the solver's arithmetic (no geometry, no operator coefficients, no
multigrid or Krylov steps).  Both the oracle and the CUDA library receive the arrays it
returns and derive everything else themselves.

Random numbers come from a counter-based splitmix64 generator: value ``i`` of stream
``s`` under seed ``S`` is ``mix64(key(S, s) + (i + 1) * 0x9E3779B97F4A7C15)`` where
``mix64`` is the splitmix64 finaliser (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) and ``key`` mixes the seed and the stream
id the same way.  Uniform doubles take the top 53 bits; normals use the Box-Muller
transform on consecutive pairs of uniforms.

Workloads (cubed sphere C_n, nlev levels):
  * vertical levels are quadratically stretched to a 30 km lid,
    z(s) = H_top (beta s + (1 - beta) s^2), s = k / nlev, beta = 5/29, which gives a
    lowest layer of 200 m at 30 levels (the paper's C192L30 grid, Sec. 5.1) and ~79 m
    at 70 levels;
  * background-state factors g = exp(0.1 xi), xi ~ N(0, 1), one per cell
    (lognormal(0, 0.1));
  * right-hand sides N(0, 1) per cell (and per velocity face for the mixed system,
    zero on the top and bottom boundary faces);
  * mixed-system velocity-mass couplings beta_up, beta_dn ~ U(0, 1) per vertical face.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Config", "CONFIGS", "config", "small_config", "uniform", "normal",
    "z_interfaces", "make_inputs",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 200200756

# stream ids of the fields a workload draws
STREAM_G = 1
STREAM_RHS = 2
STREAM_BETA_UP = 3
STREAM_BETA_DN = 4
STREAM_RHS_U = 5
STREAM_RHS_P = 6


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([(seed * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix64(s + _GOLDEN)[0]


def _raw(seed: int, stream: int, count: int) -> np.ndarray:
    key = _key(seed, stream)
    ctr = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + ctr * _GOLDEN)


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` uniform doubles in [0, 1) from stream ``stream`` of ``seed``."""
    return (_raw(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` standard normal doubles (Box-Muller on consecutive uniform pairs)."""
    m = (count + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:count]


def z_interfaces(nlev: int, top: float = 30.0e3, beta: float = 5.0 / 29.0) -> np.ndarray:
    """nlev+1 level interfaces (metres above the surface), quadratically stretched."""
    s = np.arange(nlev + 1, dtype=np.float64) / nlev
    return top * (beta * s + (1.0 - beta) * s * s)


@dataclasses.dataclass(frozen=True)
class Config:
    """One synthetic workload: a C_n cubed sphere with nlev levels and its solver settings."""
    name: str
    n: int
    nlev: int
    levels: int                 # multigrid levels L
    seed: int
    mixed: bool = False         # full (u, p) system with velocity-mass coupling
    eps: float = 0.05           # strength of the non-symmetric vertical coupling
    consistent_mass: bool = False   # mixed: consistent instead of lumped velocity mass
    rotation: float = 0.0       # mixed: planet angular velocity Omega [1/s] of the Coriolis term
    gamma2: float = 0.0         # > 0: 9-cell stencil, strength of the couplings two levels apart
    cs: float = 340.0           # speed of sound, m/s
    dt: float = 600.0           # time step, s
    radius: float = 6371.0e3    # planet radius, m
    top: float = 30.0e3         # model lid, m
    omega: float = 0.8
    n_pre: int = 2
    n_post: int = 2
    n_coarse: int = 4
    gcr_restart: int = 5

    @property
    def ncol(self) -> int:
        return 6 * self.n * self.n

    @property
    def ncell(self) -> int:
        return self.ncol * self.nlev

    @property
    def n_hface(self) -> int:
        """horizontal velocity faces: 2 per column per level"""
        return 2 * self.ncol * self.nlev

    @property
    def n_vface(self) -> int:
        """vertical velocity faces: nlev+1 per column (bottom and top boundary included)"""
        return self.ncol * (self.nlev + 1)

    @property
    def n_uface(self) -> int:
        return self.n_hface + self.n_vface


CONFIGS = {
    # C12L30, 3-level V-cycle, FP64, Helmholtz system only
    "c12": Config("c12", n=12, nlev=30, levels=3, seed=BASE_SEED + 0),
    # C48L30 mixed (u, p) system, GCR(5) outer, 4 levels
    "c48": Config("c48", n=48, nlev=30, levels=4, seed=BASE_SEED + 1, mixed=True),
    # C192L70 pressure solve (the benchmarked workload)
    "c192": Config("c192", n=192, nlev=70, levels=4, seed=BASE_SEED + 2),
    # C96L70 (differentiable-solve workload)
    "c96": Config("c96", n=96, nlev=70, levels=4, seed=BASE_SEED + 3),
    # C128L70: the headline workload's shape at 44% of its size (each finest-level array still
    # larger than L2), for detailed profiler captures
    "c128": Config("c128", n=128, nlev=70, levels=4, seed=BASE_SEED + 5),
}


def config(name: str) -> Config:
    return CONFIGS[name]


def small_config(n: int, nlev: int, levels: int = 1, seed: int = BASE_SEED + 100,
                 mixed: bool = False, **kw) -> Config:
    return Config(f"c{n}l{nlev}", n=n, nlev=nlev, levels=levels, seed=seed, mixed=mixed, **kw)


def make_inputs(cfg: Config, mixed: bool | None = None) -> dict:
    """All host arrays of a workload, float64, in the library's level-major layouts.

    Cell fields are (nlev, ncol) arrays, flattened as f[k * ncol + col].  Vertical-face
    fields are (nlev + 1, ncol), face kf lying below cell k = kf.
    """
    mixed = cfg.mixed if mixed is None else mixed
    out = {
        "z_if": z_interfaces(cfg.nlev, cfg.top),
        "g": np.exp(0.1 * normal(cfg.seed, STREAM_G, cfg.ncell)).reshape(cfg.nlev, cfg.ncol),
        "rhs": normal(cfg.seed, STREAM_RHS, cfg.ncell),
    }
    if mixed:
        out["beta_up"] = uniform(cfg.seed, STREAM_BETA_UP, cfg.n_vface).reshape(cfg.nlev + 1, cfg.ncol)
        out["beta_dn"] = uniform(cfg.seed, STREAM_BETA_DN, cfg.n_vface).reshape(cfg.nlev + 1, cfg.ncol)
        ru = normal(cfg.seed, STREAM_RHS_U, cfg.n_uface)
        rv = ru[cfg.n_hface:].reshape(cfg.nlev + 1, cfg.ncol)
        rv[0, :] = 0.0
        rv[cfg.nlev, :] = 0.0
        out["rhs_u"] = ru
        out["rhs_p"] = normal(cfg.seed, STREAM_RHS_P, cfg.ncell)
    return out
