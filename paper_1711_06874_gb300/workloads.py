"""Seeded synthetic workloads (parameters only, none of the method's arithmetic).

The paper's experiments use analytically defined functions on tensor grids
(Sec. 3.7), so every input here is a parameter set: kernel kind, smoothness
nu, length scale ell, variance sigma2, grid size n, box b and tolerance eps.
Both the CUDA path and the CPU oracle consume these; this module computes no
covariance value and no part of the decomposition.
"""
from __future__ import annotations

import dataclasses

import numpy as np

MATERN, SLATER_P, GAUSSIAN, MATERN_SD = 0, 1, 2, 3
CELL, VERTEX = 0, 1


@dataclasses.dataclass(frozen=True)
class Problem:
    kind: int = MATERN
    nu: float = 0.5
    ell: tuple = (1.0, 1.0, 1.0)
    sigma2: float = 1.0
    p: float = 1.0
    n: tuple = (64, 64, 64)
    b: tuple = (1.0, 1.0, 1.0)
    grid: int = CELL
    eps: float = 1e-6
    rmax: tuple = (64, 64, 64)

    @property
    def isotropic(self) -> bool:
        return len(set(self.ell)) == 1 and len(set(self.n)) == 1 and len(set(self.b)) == 1


def _t3(v, cast=float):
    if np.isscalar(v):
        return (cast(v),) * 3
    return tuple(cast(x) for x in v)


def problem(kind=MATERN, nu=0.5, ell=1.0, sigma2=1.0, p=1.0, n=64, b=1.0, grid=CELL, eps=1e-6,
            rmax=64) -> Problem:
    return Problem(int(kind), float(nu), _t3(ell), float(sigma2), float(p), _t3(n, int), _t3(b),
                   int(grid), float(eps), _t3(rmax, int))


# Named configurations: the small FP64 Slater case, the single n=256 solve the
# throughput metric is quoted on, the large n=512 solve.
def slater_n64(eps=1e-8):
    return problem(MATERN, nu=0.5, ell=0.3, n=64, eps=eps, rmax=20)


def matern_n256(eps=1e-6):
    return problem(MATERN, nu=1.2, ell=0.2, n=256, eps=eps, rmax=64)


def matern_n512(eps=1e-6):
    return problem(MATERN, nu=2.5, ell=0.1, n=512, eps=eps, rmax=64)


def sweep(count=256, n=128, eps=1e-6, seed=1711):
    """Likelihood-surrogate parameter sweep: nu ~ U[0.3, 2.5], ell ~ logU[0.05, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nus = rng.uniform(0.3, 2.5, size=count)
    ells = np.exp(rng.uniform(np.log(0.05), np.log(1.0), size=count))
    return [problem(MATERN, nu=float(a), ell=float(b), n=n, eps=eps, rmax=64) for a, b in zip(nus, ells)]


def serving_stream(count=2000, rate_hz=200.0, seed=6874):
    """Poisson arrivals; n uniform over {64, 128, 256, 384}; eps over {1e-4, 1e-6, 1e-8}.

    Returns a list of (arrival_seconds, Problem).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps)
    ns = rng.choice([64, 128, 256, 384], size=count)
    nus = rng.uniform(0.3, 2.5, size=count)
    ells = np.exp(rng.uniform(np.log(0.05), np.log(1.0), size=count))
    epss = rng.choice([1e-4, 1e-6, 1e-8], size=count)
    return [(float(t[i]), problem(MATERN, nu=float(nus[i]), ell=float(ells[i]), n=int(ns[i]),
                                  eps=float(epss[i]), rmax=64)) for i in range(count)]


def oracle_kernel(prob: Problem, oracle_mod):
    return oracle_mod.make_kernel(prob.kind, nu=prob.nu, ell=list(prob.ell), sigma2=prob.sigma2, p=prob.p)


def oracle_grid(prob: Problem, oracle_mod):
    return oracle_mod.make_grid(list(prob.n), b=list(prob.b), kind=prob.grid)
