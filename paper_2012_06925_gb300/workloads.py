"""Seeded synthetic particle sets for the BLDTT workloads.

This module only draws random inputs; it holds none of the method's
arithmetic.  It is the one piece of code that both the CUDA path's callers and
the CPU oracle's callers share, so both sides always see the same inputs.

Distributions follow the experiments of Wilson, Vaughn & Krasny (Sec. 4):
uniform points in the cube [-1,1]^3 with charges uniform in [-1,1]
(Sec. 4, opening paragraph and Sec. 4.1), points on the surface of the unit
sphere (Sec. 4.4), and a Plummer sphere (Sec. 4.3).  The Plummer sphere used
by the unequal-set workload is the truncated one with scale radius 0.1 and
cut-off radius 1 (cumulative mass m(r) = r^3 / (r^2 + a^2)^{3/2}), not the
paper's a=1, +/-100 cube variant.

Arrays are float64 and structure-of-arrays: positions have shape (3, n).
"""
from __future__ import annotations

import math

import numpy as np


def uniform_cube(n: int, rng: np.random.Generator) -> np.ndarray:
    """n points uniform in [-1,1]^3, shape (3, n)."""
    return rng.uniform(-1.0, 1.0, size=(3, n))


def sphere_surface(n: int, rng: np.random.Generator) -> np.ndarray:
    """n points uniform on the unit sphere (normalised Gaussian 3-vectors)."""
    g = rng.standard_normal(size=(3, n))
    norm = np.sqrt((g * g).sum(axis=0))
    norm[norm == 0.0] = 1.0
    return g / norm


def plummer(n: int, rng: np.random.Generator, a: float = 0.1, rmax: float = 1.0) -> np.ndarray:
    """n points of a Plummer sphere with scale radius a, truncated at rmax.

    The radius is drawn by inverting m(r) = r^3/(r^2+a^2)^{3/2} on
    u ~ U(0, m(rmax)); the direction is uniform on the sphere.
    """
    mmax = rmax ** 3 / (rmax * rmax + a * a) ** 1.5
    u = rng.uniform(0.0, mmax, size=n)
    u = np.maximum(u, 1e-300)
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    return sphere_surface(n, rng) * r


def gaussian(n: int, rng: np.random.Generator) -> np.ndarray:
    """n points with each coordinate normal(0, 3) (Sec. 4.3, Gaussian case)."""
    return rng.normal(0.0, math.sqrt(3.0), size=(3, n))


def uniform_charges(n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, size=n)


def normal_charges(n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal(size=n)


# Kernel identifiers (same numbering as the C ABI).
COULOMB = 0
YUKAWA = 1
OSCILLATORY = 2
REG_COULOMB = 3
TEST_POLY = 99


def make_problem(kind: str, n_targets: int, n_sources: int | None = None, seed: int = 0,
                 charges: str = "uniform", sources_kind: str | None = None):
    """Return (targets, sources, charges) for a named particle distribution.

    When n_sources is None the targets and the sources are the same set
    (the default in the paper's experiments, Sec. 4); otherwise two
    independent sets are drawn, the sources from ``sources_kind`` if given.
    """
    rng = np.random.default_rng(seed)
    gen = {"uniform": uniform_cube, "sphere": sphere_surface,
           "plummer": plummer, "gaussian": gaussian}
    tgt = gen[kind](n_targets, rng)
    if n_sources is None:
        src = tgt
        ns = n_targets
    else:
        src = gen[sources_kind or kind](n_sources, rng)
        ns = n_sources
    q = uniform_charges(ns, rng) if charges == "uniform" else normal_charges(ns, rng)
    return np.ascontiguousarray(tgt), np.ascontiguousarray(src), q


# The five workloads.  Sizes are the full ones; tests scale them down.
CONFIGS = {
    "plain_fp64_n2e4": dict(kind="uniform", M=20_000, N=None, seed=0, kernel=COULOMB,
                             kappa=0.0, n=4, theta=0.7, N0=500, M0=500),
    "uniform_n1e6": dict(kind="uniform", M=1_000_000, N=None, seed=2, kernel=COULOMB,
                          kappa=0.0, n=8, theta=0.7, N0=2000, M0=2000),
    "unequal_yukawa": dict(kind="uniform", M=10_000_000, N=5_000_000, seed=3,
                            sources_kind="plummer", kernel=YUKAWA, kappa=0.5,
                            n=7, theta=0.8, N0=2000, M0=2000),
    "uniform_n1e8": dict(kind="uniform", M=100_000_000, N=None, seed=5, kernel=COULOMB,
                          kappa=0.0, n=8, theta=0.7, N0=2000, M0=2000),
}


def batched_problems(count: int = 512, seed: int = 4, nmin: float = 1e3, nmax: float = 1e5):
    """The batched workload: `count` independent problems.

    N_p is log-uniform in [nmin, nmax]; even problems are uniform in the cube,
    odd ones lie on the unit sphere; charges are normal(0,1); the kernel is
    Coulomb or Yukawa with equal probability, kappa ~ U[0.1, 2].
    """
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        u = rng.uniform()
        npts = int(round(10 ** (math.log10(nmin) + u * (math.log10(nmax) - math.log10(nmin)))))
        pts = uniform_cube(npts, rng) if p % 2 == 0 else sphere_surface(npts, rng)
        q = normal_charges(npts, rng)
        yuk = rng.uniform() < 0.5
        kappa = float(rng.uniform(0.1, 2.0)) if yuk else 0.0
        out.append(dict(points=pts, charges=q, kernel=YUKAWA if yuk else COULOMB, kappa=kappa))
    return out
