"""T0 - Q_PE phase-diagram scans and re-fits (Sec. VI; Figs. 3b-d, 4b) from the batched engine.

Sec. VI sweeps the Hamiltonian-simulation time T0 and the clock count Q_PE (= n_c) and fits
(i) the error floor against Q_PE, (ii) the smallest Q_PE that reaches a target error and
(iii) the optimal T0* against kappa (the "power law" T0*_per_unit = e^0.918 kappa^-0.363 of the
T0 rule). Here the same scans run on the GPU through ``HHLBatch`` (one instance per problem,
clock count and T0 scale; fidelity of the postselected solution against the classical one),
and the fits are redone on the measured grid:

* ``fit_t0_kappa``: least squares of ln T0*_per_unit = a + b ln kappa over every
  (problem, n_c) optimum, with the coefficient of determination;
* ``eps_floor_slope``: ln eps_min(n_c) = alpha + beta n_c per problem (eps = 1 - F, the
  error at the best T0), and the mean slope beta;
* ``qpe_min``: per problem, the smallest n_c whose best error is at most a target.
"""
from __future__ import annotations

import math

import numpy as np

from . import t0_model


def kappa_tridiag(diag: float, off: float, n_points: int) -> float:
    """kappa of the Toeplitz tridiagonal (diag, off): eigenvalues diag + 2 off cos(k pi/(N+1))."""
    lam = diag + 2.0 * off * np.cos(np.arange(1, n_points + 1) * math.pi / (n_points + 1))
    lam = np.abs(lam)
    return float(lam.max() / lam.min())


def t0_power_law_per_unit(kappa: float) -> float:
    """The T0 rule's per-unit T0 (the Sec. VI fit read as a power law)."""
    return math.exp(0.918) * kappa ** (-0.363)


def scan(n_problems: int = 60, n_clocks=(4, 5, 6, 7), scales=None, seed: int = 5, ns_range=(3, 6)) -> dict:
    """Run the sweep on the GPU: problems (shifted channel operators spanning decades of
    kappa), fidelities F[p, c, s] for clock counts ``n_clocks`` and T0 = scale x power law."""
    problems = t0_model.sweep_problems(n_problems, seed=seed, ns_range=ns_range)
    if scales is None:
        scales = 10.0 ** np.linspace(-1.5, 1.5, 25)
    sweep = t0_model.run_sweep(problems, n_clocks=n_clocks, scales=scales)
    sweep["kappa"] = np.array([kappa_tridiag(p["diag"], p["off"], p["N"]) for p in problems])
    sweep["problems"] = problems
    return sweep


def fit_t0_kappa(sweep: dict) -> dict:
    """ln T0*_per_unit = a + b ln kappa over every (problem, n_c) optimum of the scan."""
    F, scales, kappa = sweep["F"], np.asarray(sweep["scales"]), np.asarray(sweep["kappa"])
    xs, ys = [], []
    for p in range(F.shape[0]):
        for c in range(F.shape[1]):
            s_best = scales[int(np.argmax(F[p, c]))]
            xs.append(math.log(kappa[p]))
            ys.append(math.log(s_best * t0_power_law_per_unit(kappa[p])))
    x, y = np.array(xs), np.array(ys)
    b, a = np.polyfit(x, y, 1)
    resid = y - (a + b * x)
    r2 = 1.0 - float(resid @ resid) / float(((y - y.mean()) ** 2).sum()) if len(y) > 2 else float("nan")
    return dict(a=float(a), b=float(b), r2=r2, points=len(y))


def eps_floor_slope(sweep: dict) -> dict:
    """Per problem, ln eps_min(n_c) = alpha + beta n_c (eps_min: 1 - the best fidelity over
    T0); the mean and spread of beta over the problems."""
    F, ncs = sweep["F"], np.asarray(sweep["n_clocks"], dtype=float)
    betas = []
    for p in range(F.shape[0]):
        eps = np.maximum(1.0 - F[p].max(axis=1), 1e-12)
        betas.append(np.polyfit(ncs, np.log(eps), 1)[0])
    betas = np.array(betas)
    return dict(beta_mean=float(betas.mean()), beta_std=float(betas.std()), betas=betas)


def qpe_min(sweep: dict, eps_target: float) -> np.ndarray:
    """Per problem, the smallest n_c whose best error 1 - F is <= eps_target (0 if none)."""
    F, ncs = sweep["F"], list(sweep["n_clocks"])
    out = np.zeros(F.shape[0], dtype=int)
    for p in range(F.shape[0]):
        best = 1.0 - F[p].max(axis=1)
        ok = [nc for nc, e in zip(ncs, best) if e <= eps_target]
        out[p] = ok[0] if ok else 0
    return out
