"""Nonlinear transform of the QPP protocol (App. D): sum_k z_k |k> -> ~ sum_k z_k^2 |k>.

The amplitudes z_k of a state |zeta> = U_V |0> (real, normalised) are converted to binary on a
clock register by phase estimation of an amplitude-estimation iterate (QADC), an ancilla is
rotated by an angle that depends on the clock value (sin(theta_y / 2) = c sin^2(pi y / 2^r),
so that its amplitude becomes c z_k^2), and the conversion is undone (QDAC). This is the HHL
circuit with the phase estimation of a given unitary in place of exp(i Ahat t) and a caller
rotation table in place of the eigenvalue inversion, so it runs on the library's kernels
through a UNITARY plan (controlled Q^(2^k) as dense GEMMs, the fused clock block, the
uncompute and the Hadamard layer).

Registers of the plan's system part (2a qubits for 2^a amplitudes): data (low a bits) and
address (high a bits); the address starts uniform, the data in |zeta>. After postselection
the address register carries c z_k^2 / sqrt(2^a) (with the data back in |zeta>).
"""
from __future__ import annotations

import numpy as np


def iterate(zeta: np.ndarray) -> np.ndarray:
    """Block-diagonal Q over the address: block k = -U_V S_0 U_V^T S_k on the data register
    (U_V: the Householder reflection taking |0> to |zeta>; S_j flips the sign of |j>)."""
    z = np.asarray(zeta, dtype=float)
    n = len(z)
    w = np.eye(n)[0] - z
    uv = np.eye(n) if w @ w < 1e-300 else np.eye(n) - 2.0 * np.outer(w, w) / (w @ w)
    refl0 = np.diag(np.r_[-1.0, np.ones(n - 1)])
    core = -uv @ refl0 @ uv.T
    blocks = [core @ np.diag(np.where(np.arange(n) == k, -1.0, 1.0)) for k in range(n)]
    out = np.zeros((n * n, n * n))
    for k, blk in enumerate(blocks):
        out[k * n:(k + 1) * n, k * n:(k + 1) * n] = blk
    return out


def rotation_table(n_clock: int, c: float = 1.0) -> np.ndarray:
    """theta_y = 2 arcsin(c sin^2(pi y / 2^r)), y < 2^r."""
    y = np.arange(1 << n_clock, dtype=float)
    return 2.0 * np.arcsin(c * np.square(np.sin(np.pi * y / float(1 << n_clock))))


def square_amplitudes(zeta, n_clock: int, c: float = 1.0, precision: str = "c64", gemm: str = "simt") -> dict:
    """Run the transform on the GPU; returns the postselected [address | data] vector ``v``,
    the address amplitudes (the data register projected on |zeta>) ``squares`` ~ c z^2 /
    sqrt(2^a), the success probability and the final ``state``."""
    from . import HHLPlan

    z = np.asarray(zeta, dtype=float)
    n = len(z)
    a = int(np.log2(n))
    if (1 << a) != n:
        raise ValueError("len(zeta) must be a power of two")
    plan = HHLPlan(2 * a, n_clock, unitary=iterate(z), theta_table=rotation_table(n_clock, c),
                   precision=precision, gemm=gemm)
    st = plan.new_state()
    plan.prepare_rhs_host(np.kron(np.full(n, 1.0 / np.sqrt(n)), z), st)
    plan.apply_circuit(st)
    meas = plan.measure(st)
    v = meas["xhat"] * np.sqrt(meas["p_success"])
    return dict(v=v, squares=(v.reshape(n, n) @ z), p_success=meas["p_success"], state=st, plan=plan)
