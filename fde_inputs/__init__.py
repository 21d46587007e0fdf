"""Seeded synthetic problem generators for the space-fractional diffusion equation.

This module produces *problem data only*: the grid, the diffusion coefficients
d+(x_i), d-(x_i), the initial value u0(x_i) and the source f(x_i, t_n) on the
n = 0..s time levels, plus the BVM scheme name.  It holds none of the solver's
arithmetic (no Grunwald weights, no BVM coefficients, no matrices), so that both
the CPU oracle and the CUDA path can consume the same inputs without sharing any
code of the method.

The problem is the initial-boundary value problem of Sec. 2, eq. (1.1) of
Gu et al., "Strang-type preconditioners for solving fractional diffusion
equations by boundary value methods":

    u_t = d+(x) D^alpha_+ u + d-(x) D^alpha_- u + f,   x in (xL, xR), t in (t0, T],
    u(xL, t) = u(xR, t) = 0,   u(x, t0) = u0(x),   1 < alpha < 2.

Grid (Sec. 2.1): dx = (xR - xL)/(m + 1), x_i = xL + i dx, i = 1..m (interior
points); time levels t_n = t0 + n h, h = (T - t0)/s, n = 0..s (Sec. 2.2).

Workload recipes (all seeded; the paper's Example 4.1 and the manufactured
problems are deterministic):

* ``manufactured``: exact solution u = exp(-t) x^2 (1-x)^2 on (0, 1).  The
  Riemann-Liouville derivatives of the monomial pieces have closed forms
  Gamma(p+1)/Gamma(p+1-alpha) y^(p-alpha), so f = u_t - d+ D+u - d- D-u is
  exact.  Used for the plain-method configurations (m=63/s=32 and
  m=2047/s=256) and the precision study (m=4095/s=128).
* ``random_modes``: f = exp(-c t) sum_{j=1..8} a_j sin(j pi x), a_j ~ N(0,1),
  c ~ U(0.5, 2), constant d ~ U(0.5, 2) on both sides, alpha ~ U(1.1, 1.9);
  optional random initial value u0 = sum_j b_j sin(j pi x).  Used for the
  batched and learned-warm-start workloads.
* ``example_4_1``: Example 4.1 of Sec. 4 (Gaussian pulse, f = 0, d+ = 0.6,
  d- = 0.5, x in [0, 2], T = 1, fifth-order GAM with mu = 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem",
    "SCHEMES",
    "manufactured",
    "manufactured_exact",
    "random_modes",
    "example_4_1",
    "config_small",
    "config_scale",
    "config_batch",
    "config_precision",
    "config_learned_family",
    "instance_seed",
    "check_sample",
]

# Scheme name -> (family, mu).  The family names follow the BVM literature the
# paper relies on (Sec. 2.2, Sec. 4): GBDF = generalised backward
# differentiation formulae, GAM = generalised Adams methods, ETR = extended
# trapezoidal rule (a GAM with an odd number of steps).
SCHEMES = {
    "GBDF1": ("GBDF", 1),
    "GBDF2": ("GBDF", 2),
    "GBDF3": ("GBDF", 3),
    "GBDF4": ("GBDF", 4),
    "GBDF5": ("GBDF", 5),
    "GAM1": ("GAM", 1),
    "GAM2": ("GAM", 2),
    "GAM3": ("GAM", 3),
    "GAM4": ("GAM", 4),
    "GAM5": ("GAM", 5),
    "ETR3": ("ETR", 3),
    "ETR5": ("ETR", 5),
}


@dataclass
class Problem:
    """One instance of eq. (1.1) sampled on the grid of Sec. 2.1 / Sec. 2.2."""

    m: int
    s: int
    alpha: float
    xL: float
    xR: float
    t0: float
    T: float
    dplus: np.ndarray  # (m,) float64, d+(x_i)
    dminus: np.ndarray  # (m,) float64, d-(x_i)
    u0: np.ndarray  # (m,) float64, u0(x_i)
    f: np.ndarray  # (s+1, m) float64, f(x_i, t_n), row n = time level n
    scheme: str  # key of SCHEMES
    name: str = ""
    meta: dict = field(default_factory=dict)
    # time-dependent coefficients d+-(x_i, t_n), (s+1, m), or None; when given, dplus /
    # dminus hold their means over the unknown time levels n = 1..s
    dplus_t: np.ndarray | None = None
    dminus_t: np.ndarray | None = None

    @property
    def family(self) -> str:
        return SCHEMES[self.scheme][0]

    @property
    def mu(self) -> int:
        return SCHEMES[self.scheme][1]

    @property
    def dx(self) -> float:
        return (self.xR - self.xL) / (self.m + 1)

    @property
    def h(self) -> float:
        return (self.T - self.t0) / self.s

    @property
    def x(self) -> np.ndarray:
        return self.xL + self.dx * np.arange(1, self.m + 1, dtype=np.float64)

    @property
    def t(self) -> np.ndarray:
        return self.t0 + self.h * np.arange(0, self.s + 1, dtype=np.float64)

    @property
    def n(self) -> int:
        """Number of unknowns u_1..u_s (u_0 is given)."""
        return self.m * self.s

    def constant_d(self) -> bool:
        return bool(np.all(self.dplus == self.dplus[0]) and np.all(self.dminus == self.dminus[0]))


def instance_seed(index: int) -> int:
    """Per-instance seed of the batched / learned workloads."""
    return 1305 * 1000 + int(index)


def _grid(m: int, xL: float, xR: float) -> np.ndarray:
    dx = (xR - xL) / (m + 1)
    return xL + dx * np.arange(1, m + 1, dtype=np.float64)


def _rl_poly_coeff(p: int, alpha: float) -> float:
    # Riemann-Liouville derivative of y^p (lower terminal 0): Gamma(p+1)/Gamma(p+1-alpha) y^(p-alpha)
    return math.gamma(p + 1) / math.gamma(p + 1 - alpha)


def _rl_profile(y: np.ndarray, alpha: float) -> np.ndarray:
    """D^alpha of y^2 (1-y)^2 = y^2 - 2 y^3 + y^4 with lower terminal 0."""
    return (_rl_poly_coeff(2, alpha) * y ** (2 - alpha)
            - 2.0 * _rl_poly_coeff(3, alpha) * y ** (3 - alpha)
            + _rl_poly_coeff(4, alpha) * y ** (4 - alpha))


def manufactured_exact(x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Exact solution u(x, t) = exp(-t) x^2 (1-x)^2, returned as (len(t), len(x))."""
    return np.exp(-np.asarray(t))[:, None] * (x ** 2 * (1.0 - x) ** 2)[None, :]


def manufactured(m: int, s: int, alpha: float, scheme: str,
                 dplus_fn=lambda x: np.ones_like(x), dminus_fn=lambda x: np.ones_like(x),
                 name: str = "manufactured") -> Problem:
    """Problem on (0,1)x(0,1] whose exact solution is exp(-t) x^2 (1-x)^2.

    The left derivative of x^2(1-x)^2 is _rl_profile(x); by the symmetry
    x -> 1-x of the profile, the right derivative is _rl_profile(1-x).
    """
    xL, xR, t0, T = 0.0, 1.0, 0.0, 1.0
    x = _grid(m, xL, xR)
    t = t0 + (T - t0) / s * np.arange(s + 1, dtype=np.float64)
    dp = np.asarray(dplus_fn(x), dtype=np.float64)
    dm = np.asarray(dminus_fn(x), dtype=np.float64)
    prof = x ** 2 * (1.0 - x) ** 2
    left = _rl_profile(x, alpha)
    right = _rl_profile(1.0 - x, alpha)
    et = np.exp(-t)[:, None]
    # f = u_t - d+ D+ u - d- D- u with u_t = -u
    f = -et * prof[None, :] - et * (dp * left + dm * right)[None, :]
    u0 = prof.copy()
    return Problem(m=m, s=s, alpha=float(alpha), xL=xL, xR=xR, t0=t0, T=T,
                   dplus=dp, dminus=dm, u0=u0, f=np.ascontiguousarray(f),
                   scheme=scheme, name=name)


def manufactured_time_varying(m: int, s: int, alpha: float, scheme: str,
                              name: str = "manufactured_tv") -> Problem:
    """As manufactured(), with coefficients that vary in space and time (eq. (1.1)
    allows d+-(x, t)): d+(x,t) = (1+x)(1 + sin(pi t)/2), d-(x,t) = (2-x)(1 + t/2)."""
    xL, xR, t0, T = 0.0, 1.0, 0.0, 1.0
    x = _grid(m, xL, xR)
    t = t0 + (T - t0) / s * np.arange(s + 1, dtype=np.float64)
    dpt = (1.0 + x)[None, :] * (1.0 + 0.5 * np.sin(np.pi * t))[:, None]
    dmt = (2.0 - x)[None, :] * (1.0 + 0.5 * t)[:, None]
    prof = x ** 2 * (1.0 - x) ** 2
    left = _rl_profile(x, alpha)
    right = _rl_profile(1.0 - x, alpha)
    et = np.exp(-t)[:, None]
    f = -et * prof[None, :] - et * (dpt * left[None, :] + dmt * right[None, :])
    return Problem(m=m, s=s, alpha=float(alpha), xL=xL, xR=xR, t0=t0, T=T,
                   dplus=dpt[1:].mean(axis=0), dminus=dmt[1:].mean(axis=0), u0=prof.copy(),
                   f=np.ascontiguousarray(f), scheme=scheme, name=name,
                   dplus_t=np.ascontiguousarray(dpt), dminus_t=np.ascontiguousarray(dmt))


def random_modes(m: int, s: int, scheme: str, seed: int, *, random_u0: bool = False,
                 alpha: float | None = None, name: str = "random_modes") -> Problem:
    """Smooth random source (8 sine modes times exp(-c t)) on (0,1)x(0,1]."""
    rng = np.random.default_rng(seed)
    a_alpha = rng.uniform(1.1, 1.9)
    d = rng.uniform(0.5, 2.0)
    c = rng.uniform(0.5, 2.0)
    a = rng.standard_normal(8)
    b = rng.standard_normal(8)
    if alpha is not None:
        a_alpha = float(alpha)
    xL, xR, t0, T = 0.0, 1.0, 0.0, 1.0
    x = _grid(m, xL, xR)
    t = t0 + (T - t0) / s * np.arange(s + 1, dtype=np.float64)
    j = np.arange(1, 9, dtype=np.float64)
    modes = np.sin(np.pi * np.outer(x, j))  # (m, 8)
    f = np.exp(-c * t)[:, None] * (modes @ a)[None, :]
    u0 = modes @ b if random_u0 else np.zeros(m)
    return Problem(m=m, s=s, alpha=float(a_alpha), xL=xL, xR=xR, t0=t0, T=T,
                   dplus=np.full(m, d), dminus=np.full(m, d), u0=u0,
                   f=np.ascontiguousarray(f), scheme=scheme, name=name,
                   meta={"seed": seed, "d": d, "c": c, "a": a, "b": b if random_u0 else None})


def example_4_1(alpha: float, n: int, s: int) -> Problem:
    """Example 4.1 of Sec. 4: Gaussian pulse, f = 0, d+ = 0.6, d- = 0.5, GAM with mu = 4."""
    xL, xR, t0, T = 0.0, 2.0, 0.0, 1.0
    x = _grid(n, xL, xR)
    xc, xi = 1.2, 0.08
    u0 = np.exp(-((x - xc) ** 2) / (2.0 * xi ** 2))
    return Problem(m=n, s=s, alpha=float(alpha), xL=xL, xR=xR, t0=t0, T=T,
                   dplus=np.full(n, 0.6), dminus=np.full(n, 0.5), u0=u0,
                   f=np.zeros((s + 1, n)), scheme="GAM4", name=f"ex41_a{alpha}_n{n}_s{s}")


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def config_small() -> Problem:
    """Plain method, FP64: m=63, s=32, alpha=1.5, d+=d-=1, 3-step GBDF; 2016 unknowns."""
    return manufactured(63, 32, 1.5, "GBDF3", name="small_m63_s32")


def config_scale(m: int = 2047, s: int = 256) -> Problem:
    """Plain method at scale: alpha=1.8, d+=1+x, d-=2-x, 5-step GBDF; m=2047, s=256."""
    return manufactured(m, s, 1.8, "GBDF5", dplus_fn=lambda x: 1.0 + x,
                        dminus_fn=lambda x: 2.0 - x, name=f"scale_m{m}_s{s}")


def config_precision(m: int = 4095, s: int = 128) -> Problem:
    """Precision study: m=4095, s=128, alpha=1.9, d+=d-=1, 3-step GBDF."""
    return manufactured(m, s, 1.9, "GBDF3", name=f"precision_m{m}_s{s}")


def config_batch(count: int = 64, m_choices=(255, 511, 1023, 2047), s_choices=(64, 128, 256),
                 schemes=("ETR3", "GBDF3", "GAM4"), base: int = 0) -> list[Problem]:
    """Batch of independent instances with uneven m, s, alpha and scheme."""
    out = []
    for i in range(count):
        seed = instance_seed(base + i)
        rng = np.random.default_rng(seed + 7_000_000)
        m = int(rng.choice(m_choices))
        s = int(rng.choice(s_choices))
        scheme = str(rng.choice(schemes))
        out.append(random_modes(m, s, scheme, seed, name=f"batch{base + i}"))
    return out


def config_many_rhs(count: int = 16, m: int = 2047, s: int = 256, base_seed: int = 0) -> list[Problem]:
    """Many right-hand sides of the benchmark operator (m, s, alpha = 1.8, d+ = 1+x,
    d- = 2-x, GBDF5): instance r keeps the operator and takes the manufactured source
    scaled by (1 + r/4) plus a seeded smooth source e^{-ct} sum_j a_j sin(j pi x),
    and the manufactured u0 scaled by (1 - r/(2 count))."""
    import dataclasses
    base = config_scale(m, s)
    x, t = base.x, base.t
    modes = np.sin(np.pi * np.outer(x, np.arange(1, 9, dtype=np.float64)))
    out = []
    for r in range(count):
        rng = np.random.default_rng(instance_seed(base_seed + r) + 9_000_000)
        c = rng.uniform(0.5, 2.0)
        a = rng.standard_normal(8)
        f = base.f * (1.0 + 0.25 * r) + np.exp(-c * t)[:, None] * (modes @ a)[None, :]
        out.append(dataclasses.replace(base, f=np.ascontiguousarray(f), u0=base.u0 * (1.0 - 0.5 * r / count),
                                       name=f"rhs{r}_m{m}_s{s}", meta={"c": c, "a": a}))
    return out


def check_sample(n: int, seed: int, count: int = 128, projections: int = 8):
    """Seeded positions and probe vectors for comparing two length-n solutions that are
    too large to store: `count` distinct indices in [0, n) and `projections` standard
    normal vectors of length n (E <g, v>^2 = |v|^2, so the probes estimate the 2-norm
    of a difference).  Plain random numbers; no arithmetic of the method."""
    rng = np.random.default_rng(seed + 11_000_000)
    idx = np.sort(rng.choice(n, size=min(count, n), replace=False))
    probes = rng.standard_normal((projections, n))
    return idx, probes


def config_learned_family(seed: int, m: int = 1023, s: int = 256) -> Problem:
    """Learned-warm-start family member: random alpha, d, u0 and source; 3-step GBDF."""
    return random_modes(m, s, "GBDF3", seed, random_u0=True, name=f"family{seed}")
