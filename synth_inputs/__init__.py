"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and bench.py.

This module holds only input generation: problem sizes, right-hand sides and the random
draws of the workloads. It performs none of the HHL method's arithmetic (no operator,
no normalisation, no T0 rule, no angles), so that the oracle and the CUDA path stay
independent and merely see identical inputs.

Workloads (all synthetic; the paper uses no public dataset):

* ``poiseuille_16``  - N = 16 interior points, b = 1 (constant pressure gradient), n_c = 6.
* ``couette_1024``   - N = 1024, b = e_N / h^2 (moving wall u = 1 carried on the last
  entry), n_c = 12.
* ``batch_256``      - 256 instances: n_s ~ U{6..12}, n_c ~ U{8..12}, flow ~ Bernoulli(1/2),
  b ~ U[0,1)^N, T0 multiplier 10^U(-1,1) applied to each side's own power-law T0.
* ``poiseuille_2p18`` - N = 2^18, b = 1, n_c = 13 (32 qubits).
* ``qft_random``     - complex Gaussian random states (the random initial states of the
  paper's QFT-IQFT scaling experiment, Fig. 1c).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 230700391


def rng(offset: int = 0) -> np.random.Generator:
    """PCG64 generator seeded with ``BASE_SEED + offset``."""
    return np.random.default_rng(BASE_SEED + offset)


def grid_spacing(n_points: int) -> float:
    """h = 1/(N+1) for N interior points between walls at y = 0 and y = 1."""
    return 1.0 / (n_points + 1)


def rhs(flow: str, n_points: int, wall_hi: float = 1.0) -> np.ndarray:
    """Right-hand side b of the steady 1-D channel problem for N interior points.

    ``poiseuille``: b_i = 1 (constant forcing, in units of Re * (-dp/dx)).
    ``couette``: b = e_N * wall_hi / h^2, the moving-wall Dirichlet value carried on the
    last interior equation.
    """
    if flow == "poiseuille":
        return np.ones(n_points, dtype=np.float64)
    if flow == "couette":
        h = grid_spacing(n_points)
        b = np.zeros(n_points, dtype=np.float64)
        b[-1] = wall_hi / (h * h)
        return b
    raise ValueError(f"unknown flow {flow!r}")


def walls(flow: str, wall_hi: float = 1.0) -> tuple[float, float]:
    """Dirichlet wall velocities (u(0), u(1))."""
    return (0.0, 0.0) if flow == "poiseuille" else (0.0, wall_hi)


def random_state(n_qubits: int, seed_offset: int = 0, count: int = 1) -> np.ndarray:
    """``count`` complex Gaussian states of 2^n amplitudes, each normalised, complex128."""
    g = rng(1000 + seed_offset)
    dim = 1 << n_qubits
    z = g.standard_normal((count, dim)) + 1j * g.standard_normal((count, dim))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    return z if count > 1 else z[0]


def random_rhs(n_points: int, seed_offset: int = 0) -> np.ndarray:
    """b ~ U[0,1)^N (float64)."""
    return rng(2000 + seed_offset).random(n_points)


def batch_instances(count: int = 256, seed_offset: int = 0,
                    ns_range=(6, 12), nc_range=(8, 12)) -> list[dict]:
    """Uneven batch: per instance n_s, n_c, flow, b ~ U[0,1)^N and a T0 multiplier.

    Draws are made in instance order from one generator so that any prefix of the batch is
    reproducible on its own.
    """
    g = rng(3000 + seed_offset)
    out = []
    for i in range(count):
        n_s = int(g.integers(ns_range[0], ns_range[1] + 1))
        n_c = int(g.integers(nc_range[0], nc_range[1] + 1))
        flow = "couette" if g.random() < 0.5 else "poiseuille"
        n = 1 << n_s
        b = g.random(n)
        t0_mult = float(10.0 ** g.uniform(-1.0, 1.0))
        out.append(dict(index=i, n_s=n_s, n_c=n_c, flow=flow, b=b, t0_mult=t0_mult))
    return out


def uniform_draws(count: int, seed_offset: int = 0) -> np.ndarray:
    """U[0,1) draws handed to measurement sampling (shots) as explicit inputs."""
    return rng(4000 + seed_offset).random(count)


WORKLOADS = {
    "poiseuille_16": dict(flow="poiseuille", n_s=4, n_c=6, nu=0.1),
    "couette_1024": dict(flow="couette", n_s=10, n_c=12, nu=0.1),
    "poiseuille_2p18": dict(flow="poiseuille", n_s=18, n_c=13, nu=0.1),
}
