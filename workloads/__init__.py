"""Seeded synthetic inputs for the entropic-OT solver and its oracle.

This module only draws random problem data (point clouds, weights, regularisation
levels, arrival times).  It holds none of the solver's arithmetic: no cost
matrix, no transform, no coupling.  Both the CUDA path (through the C ABI) and
the CPU oracle read their inputs from here, so that the two sides see exactly
the same numbers.

Every generator takes a ``seed`` and uses NumPy's PCG64 (``default_rng``).
Point clouds are returned as float32 (the device input format; the oracle
promotes the very same values to float64) and weights as float64 vectors that
are positive and sum to one (the problem statement of Sec. 2 asks for
probability vectors alpha, beta).

Workload shapes follow the paper's experiments (Sec. 5) and the measured
configurations of this library:

* ``uniform_square``      n = m = 256 points uniform in [0,1]^2, uniform weights.
* ``gaussian_mixture``    n = m = 4096 points in R^3 from a 4-component mixture
                          (sigma = 0.1, means uniform in [0,1]^3), Dirichlet(1)
                          weights.
* ``gaussian_cloud``      n x m points in R^d ~ N(0, I)/8, uniform weights.
* ``gaussians_2d``        Sec. 5 first experiment: 200 points ~ N(0, I) against
                          400 points ~ N((4,4), [[1,-.8],[-.8,1]]), uniform.
* ``batch_problems``      many problems of uneven n, m, d and epsilon.
* ``served_stream``       Poisson arrivals of problems of mixed size.
* ``random_cost``         a dense positive cost matrix (kernel edge cases).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "Problem",
    "uniform_square",
    "gaussian_mixture",
    "gaussian_cloud",
    "gaussians_2d",
    "random_cost",
    "random_potentials",
    "batch_problems",
    "served_stream",
]


@dataclass
class Problem:
    """One discrete EOT problem: clouds X (n x d), Y (m x d) or a cost C, weights a, b."""

    a: np.ndarray                      # (n,) float64, positive, sums to 1
    b: np.ndarray                      # (m,) float64, positive, sums to 1
    X: Optional[np.ndarray] = None     # (n, d) float32
    Y: Optional[np.ndarray] = None     # (m, d) float32
    C: Optional[np.ndarray] = None     # (n, m) float32 when the cost is given directly
    eps: float = 1e-2
    normalize_cost: bool = False
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.a.shape[0])

    @property
    def m(self) -> int:
        return int(self.b.shape[0])

    @property
    def d(self) -> int:
        return 0 if self.X is None else int(self.X.shape[1])


def _simplex_uniform(k: int) -> np.ndarray:
    return np.full(k, 1.0 / k, dtype=np.float64)


def _dirichlet_ones(rng: np.random.Generator, k: int) -> np.ndarray:
    w = rng.dirichlet(np.ones(k))
    w = np.maximum(w, np.finfo(np.float64).tiny)
    return w / w.sum()


def uniform_square(n: int = 256, m: int = 256, d: int = 2, seed: int = 0,
                   eps: float = 1e-2) -> Problem:
    """Points uniform in [0,1]^d with uniform weights; cost normalised to max 1."""
    rng = np.random.default_rng(seed)
    X = rng.random((n, d)).astype(np.float32)
    Y = rng.random((m, d)).astype(np.float32)
    return Problem(a=_simplex_uniform(n), b=_simplex_uniform(m), X=X, Y=Y, eps=eps,
                   normalize_cost=True, name=f"uniform_square_{n}x{m}_d{d}")


def gaussian_mixture(n: int = 4096, m: int = 4096, d: int = 3, k: int = 4,
                     sigma: float = 0.1, seed: int = 0, eps: float = 1e-3) -> Problem:
    """X and Y are independent samples of the same equal-weight Gaussian mixture.

    The k means are uniform in [0,1]^d, each component is N(mu, sigma^2 I).
    Weights a, b are independent Dirichlet(1) draws.  The cost is meant to be
    normalised to max 1.
    """
    rng = np.random.default_rng(seed)
    mu = rng.random((k, d))
    cx = rng.integers(0, k, size=n)
    cy = rng.integers(0, k, size=m)
    X = (mu[cx] + sigma * rng.standard_normal((n, d))).astype(np.float32)
    Y = (mu[cy] + sigma * rng.standard_normal((m, d))).astype(np.float32)
    a = _dirichlet_ones(rng, n)
    b = _dirichlet_ones(rng, m)
    return Problem(a=a, b=b, X=X, Y=Y, eps=eps, normalize_cost=True,
                   name=f"gaussian_mixture_{n}x{m}_d{d}")


def gaussian_cloud(n: int = 20000, m: int = 30000, d: int = 64, seed: int = 0,
                   eps: float = 1e-3, scale: float = 1.0 / 8.0) -> Problem:
    """Points ~ N(0, I_d) * scale with uniform weights; raw (unnormalised) cost."""
    rng = np.random.default_rng(seed)
    X = (scale * rng.standard_normal((n, d))).astype(np.float32)
    Y = (scale * rng.standard_normal((m, d))).astype(np.float32)
    return Problem(a=_simplex_uniform(n), b=_simplex_uniform(m), X=X, Y=Y, eps=eps,
                   normalize_cost=False, name=f"gaussian_cloud_{n}x{m}_d{d}")


def gaussians_2d(n: int = 200, seed: int = 0, eps: float = 1e-1) -> Problem:
    """Sec. 5, 2-D experiment: n points ~ N(0, I) against 2n points ~ N((4,4), S).

    S = [[1, -0.8], [-0.8, 1]]; both measures uniform; squared Euclidean cost,
    not normalised.
    """
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 2))
    L = np.linalg.cholesky(np.array([[1.0, -0.8], [-0.8, 1.0]]))
    Y = np.array([4.0, 4.0]) + rng.standard_normal((2 * n, 2)) @ L.T
    return Problem(a=_simplex_uniform(n), b=_simplex_uniform(2 * n),
                   X=X.astype(np.float32), Y=Y.astype(np.float32), eps=eps,
                   normalize_cost=False, name=f"gaussians_2d_{n}x{2 * n}")


def square_annulus(n: int = 200, m: int = 200, seed: int = 0, eps: float = 0.064) -> Problem:
    """Sec. 3 (spectral stability): uniform measure on the unit square against
    the uniform measure on an annulus (radii 0.25 and 0.5, centred at
    (0.5, 0.5)); uniform weights; squared Euclidean cost, not normalised."""
    rng = np.random.default_rng(seed)
    X = rng.random((n, 2))
    r = np.sqrt(rng.uniform(0.25 ** 2, 0.5 ** 2, m))     # uniform in area
    th = rng.uniform(0.0, 2.0 * np.pi, m)
    Y = np.stack([0.5 + r * np.cos(th), 0.5 + r * np.sin(th)], axis=1)
    return Problem(a=_simplex_uniform(n), b=_simplex_uniform(m), X=X.astype(np.float32),
                   Y=Y.astype(np.float32), eps=eps, normalize_cost=False,
                   name=f"square_annulus_{n}x{m}")


def random_cost(n: int, m: int, seed: int = 0, scale: float = 1.0,
                dirichlet: bool = True) -> Problem:
    """A dense cost with entries uniform in [0, scale), float32, plus weights."""
    rng = np.random.default_rng(seed)
    C = (scale * rng.random((n, m))).astype(np.float32)
    if dirichlet:
        a, b = _dirichlet_ones(rng, n), _dirichlet_ones(rng, m)
    else:
        a, b = _simplex_uniform(n), _simplex_uniform(m)
    return Problem(a=a, b=b, C=C, name=f"random_cost_{n}x{m}")


def random_potentials(n: int, m: int, seed: int = 0, spread: float = 1.0):
    """Arbitrary float64 potentials f (n,), g (m,) for single half-step tests."""
    rng = np.random.default_rng(seed)
    return (spread * rng.standard_normal(n), spread * rng.standard_normal(m))


def batch_problems(count: int = 512, seed: int = 0, n_lo: int = 64, n_hi: int = 4096,
                   eps_lo: float = 1e-3, eps_hi: float = 1e-1) -> list:
    """Problems with n, m log-uniform in [n_lo, n_hi], d in {2, 3}, points uniform
    in [0,1]^d, Dirichlet(1) weights, eps log-uniform in [eps_lo, eps_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        m = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        d = int(rng.integers(2, 4))
        eps = float(np.exp(rng.uniform(np.log(eps_lo), np.log(eps_hi))))
        X = rng.random((n, d)).astype(np.float32)
        Y = rng.random((m, d)).astype(np.float32)
        out.append(Problem(a=_dirichlet_ones(rng, n), b=_dirichlet_ones(rng, m), X=X, Y=Y,
                           eps=eps, normalize_cost=True, name=f"batch_{k}_{n}x{m}_d{d}"))
    return out


def served_stream(seed: int = 0, rate_per_s: float = 2000.0, duration_s: float = 1.0,
                  n_lo: int = 128, n_hi: int = 16384, dims=(2, 3, 64),
                  eps_set=(1e-1, 1e-2, 1e-3), reuse_fraction: float = 0.5,
                  max_requests: Optional[int] = None) -> list:
    """Poisson arrivals of problems of mixed size for the serving loop.

    Each request is a dict with ``t`` (arrival time in seconds), ``problem``
    and ``cloud_id`` (requests that re-use an earlier cloud with another eps carry
    the same id, so that potentials resident on the device can warm-start them).
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    clouds = []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t > duration_s or (max_requests is not None and len(reqs) >= max_requests):
            break
        eps = float(rng.choice(eps_set))
        if clouds and rng.random() < reuse_fraction:
            cid, base = clouds[int(rng.integers(0, len(clouds)))]
            prob = Problem(a=base.a, b=base.b, X=base.X, Y=base.Y, eps=eps,
                           normalize_cost=base.normalize_cost, name=base.name)
        else:
            n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
            m = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
            d = int(rng.choice(dims))
            if d == 64:
                X = (rng.standard_normal((n, d)) / 8.0).astype(np.float32)
                Y = (rng.standard_normal((m, d)) / 8.0).astype(np.float32)
            else:
                X = rng.random((n, d)).astype(np.float32)
                Y = rng.random((m, d)).astype(np.float32)
            prob = Problem(a=_dirichlet_ones(rng, n), b=_dirichlet_ones(rng, m), X=X, Y=Y,
                           eps=eps, normalize_cost=True, name=f"served_{n}x{m}_d{d}")
            cid = len(clouds) + 1
            clouds.append((cid, prob))
        reqs.append({"t": t, "problem": prob, "cloud_id": cid})
    return reqs
