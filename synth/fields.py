"""Analytic data and seeded per-cell coefficient fields.

Each *problem* bundles a pressure p, the flux u = -K grad p (for constant K),
the source f = div u and the Dirichlet datum g_D = p, as vectorised functions
of an (N, 3) array of points.  The numerical methods only ever see the values
of f and g_D at the quadrature points they ask for.
"""

from __future__ import annotations

from dataclasses import dataclass
from functools import partial
from typing import Callable

import numpy as np

Fn = Callable[[np.ndarray], np.ndarray]


@dataclass
class Problem:
    name: str
    p: Fn          # exact pressure
    u: Fn          # exact flux (for K = 1 unless stated)
    f: Fn          # source f = div u
    gD: Fn         # Dirichlet datum on the boundary


# The data are module-level functions (bound to their parameters with
# functools.partial), so problems can be sent to worker processes.
_PI = np.pi


def _sine_p(x):
    return np.sin(_PI * x[:, 0]) * np.sin(_PI * x[:, 1]) * np.sin(_PI * x[:, 2])


def _sine_u(x):
    s = np.sin(_PI * x)
    c = np.cos(_PI * x)
    return -_PI * np.stack([c[:, 0] * s[:, 1] * s[:, 2],
                            s[:, 0] * c[:, 1] * s[:, 2],
                            s[:, 0] * s[:, 1] * c[:, 2]], 1)


def _sine_f(x):
    return 3.0 * _PI * _PI * _sine_p(x)


def sine_problem() -> Problem:
    """p = sin(pi x) sin(pi y) sin(pi z), K = 1: f = 3 pi^2 p, g_D = 0."""
    return Problem("sine", _sine_p, _sine_u, _sine_f, _sine_p)


def _lin_p(x, a0, a):
    return a0 + x @ a


def _lin_u(x, a, K):
    return np.broadcast_to(-K * a, x.shape).copy()


def _zero(x):
    return np.zeros(x.shape[0])


def linear_problem(a0: float = 0.3, a=(1.0, -2.0, 0.5), K: float = 1.0) -> Problem:
    """p = a0 + a.x with constant K: u = -K a, f = 0."""
    a = np.asarray(a, dtype=np.float64)
    p = partial(_lin_p, a0=a0, a=a)
    return Problem("linear", p, partial(_lin_u, a=a, K=K), _zero, p)


def _quad_p(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return X * X - 2 * Y * Y + 0.5 * Z * Z + X * Y - Y * Z + 0.3 * X


def _quad_u(x, K):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return -K * np.stack([2 * X + Y + 0.3, -4 * Y + X - Z, Z - Y], 1)


def _quad_f(x, K):
    # div u = -K (2 - 4 + 1)
    return np.full(x.shape[0], K * 1.0)


def quadratic_problem(K: float = 1.0) -> Problem:
    """p = x^2 - 2 y^2 + z^2/2 + xy - yz + 0.3 x, constant K: u linear, f const."""
    return Problem("quadratic", _quad_p, partial(_quad_u, K=K), partial(_quad_f, K=K), _quad_p)


def _poly_p(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return X ** 5 + 6 * Y ** 4 + 9 * Z ** 3 + X * Y ** 2 * Z ** 3


def _poly_u(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return np.stack([-5 * X ** 4 - Y ** 2 * Z ** 3,
                     -24 * Y ** 3 - 2 * X * Y * Z ** 3,
                     -27 * Z ** 2 - 3 * X * Y ** 2 * Z ** 2], 1)


def _poly_f(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return -(20 * X ** 3 + 2 * X * Z ** 3 + 72 * Y ** 2 + 54 * Z + 6 * X * Y ** 2 * Z)


def paper_polynomial_problem() -> Problem:
    """The polynomial exact solution of the paper's convergence test (Sec. 4.4),
    nu = 1: q = x^5 + 6y^4 + 9z^3 + x y^2 z^3 and v = -grad q."""
    return Problem("paper_poly", _poly_p, _poly_u, _poly_f, _poly_p)


def _fourier(x, ks, ph):
    return np.cos(2 * np.pi * (x @ ks.T) + ph).sum(axis=1)


def fourier_source(seed: int, n_modes: int = 8) -> Fn:
    """f = sum_m cos(2 pi k_m . x + phi_m), k_m in {0..3}^3 \\ {0}, phi ~ U[0, 2pi)."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(0, 4, size=3)
        if np.any(k != 0):
            ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    ph = rng.uniform(0.0, 2 * np.pi, size=n_modes)
    return partial(_fourier, ks=ks, ph=ph)


def K_uniform(n_cells: int, value: float = 1.0) -> np.ndarray:
    return np.full(n_cells, value, dtype=np.float64)


def K_high_contrast(n_cells: int, seed: int = 1, decades: float = 4.0) -> np.ndarray:
    """K = 10^U per cell, U ~ U[-decades, decades] i.i.d."""
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(-decades, decades, size=n_cells)


def K_lognormal(n_cells: int, seed: int, sigma: float = 2.0) -> np.ndarray:
    """K = exp(sigma * xi) per cell, xi ~ N(0, 1) i.i.d."""
    rng = np.random.default_rng(seed)
    return np.exp(sigma * rng.standard_normal(n_cells))
