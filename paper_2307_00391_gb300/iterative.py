"""The iterative backward-Euler hybrid loop (Sec. II; Fig. 2a-b): once per time step the
system A_be1 u^{j+1} = b_be1, A_be1 = I - A dt, b_be1 = u^j + f dt, is loaded (QSP-1 tree,
App. C), solved by the HHL circuit, read out in full, and the classical side checks the
residue max_i |u^{j+1} - u^j| against a tolerance (1e-6 in the paper) before the next step.

A_be1 of the channel flow is the Toeplitz tridiagonal tridiag(-r, 1 + 2r, -r), r = nu dt/h^2:
one plan serves every step (only the right-hand side changes). The read-out here is the
exact postselected amplitude vector of the simulated state (no shot noise):
u^{j+1} = |b| Re(v) / (C lambda_ub).
"""
from __future__ import annotations

import numpy as np


def be1_tridiagonal(n_points: int, nu: float, dt: float) -> tuple[np.ndarray, np.ndarray]:
    """Diagonal and off-diagonal of I - dt nu (u_{i+1} - 2 u_i + u_{i-1}) / h^2."""
    r = nu * dt * (n_points + 1) ** 2
    return np.full(n_points, 1.0 + 2.0 * r), np.full(n_points - 1, -r)


def iterative_be(n_points: int, nu: float, f, u0, dt: float, n_clock: int, max_steps: int,
                 tol: float = 1e-6, precision: str = "c64", prep: str = "qsp1", t0_rule: str = "range_fill",
                 on_step=None) -> dict:
    """Run the loop on the GPU. ``prep``: "qsp1" (gate-level tree; b_be1 >= 0 for the flows
    here) or "amplitude". ``on_step(j, b, u_next)`` is called after every step (for checks).
    Returns the fields u^0 .. u^J, the residues and the plan info."""
    import torch

    from . import HHLPlan

    diag, off = be1_tridiagonal(n_points, nu, dt)
    n_s = int(np.log2(n_points))
    if (1 << n_s) != n_points:
        raise ValueError("n_points must be a power of two")
    plan = HHLPlan(n_s, n_clock, diag=diag, off=off, precision=precision, t0_rule=t0_rule)
    info = plan.info
    st = plan.new_state()
    f = np.asarray(f, dtype=float)
    us, res = [np.array(u0, dtype=float)], []
    for j in range(max_steps):
        b = us[-1] + dt * f
        if prep == "qsp1":
            if np.any(b < 0):
                raise ValueError("QSP-1 encodes magnitudes: b_be1 must be >= 0 (use prep='amplitude')")
            plan.prepare_rhs_qsp1(torch.tensor(b, dtype=torch.float64, device="cuda"), st)
        else:
            plan.prepare_rhs_host(b, st)
        plan.apply_circuit(st)
        meas = plan.measure(st)
        v = meas["xhat"] * np.sqrt(meas["p_success"])
        u_next = np.linalg.norm(b) * v.real / (info["C"] * info["lambda_ub"])
        if on_step is not None:
            on_step(j, b, u_next)
        res.append(float(np.max(np.abs(u_next - us[-1]))))
        us.append(u_next)
        if res[-1] <= tol:
            break
    return dict(fields=us, residues=res, info=info)
