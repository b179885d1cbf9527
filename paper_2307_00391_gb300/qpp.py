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

``form="swap"`` runs the conversion the way App. D prints it (STEPS 1-5): per address s the
data register ua, a clone a1 of the address and a swap-test qubit a2 (system index
ua + N a1 + N^2 a2 + 2 N^2 s, 3a + 1 qubits); the swap test of ua against a1 puts weight
sin^2(pi beta) = (1 + z_s^2) / 2 on a2 = 0, phase estimation of its amplitude-estimation
iterate reads beta or 1 - beta, and the rotation uses z_s^2 = 2 sin^2(pi beta) - 1. Its
system register holds 2 N^3 amplitudes, so the dense UNITARY plan (at most 256) takes N <= 4.
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


def swap_register_state(zeta: np.ndarray) -> np.ndarray:
    """The state after STEPS 1-3 (uniform address, clone, U_V, swap test without measurement):
    amplitude (z_i [j = s] +- [i = s] z_j) / (2 sqrt N) at ua = i, a1 = j, address s, with +
    for a2 = 0 and - for a2 = 1."""
    z = np.asarray(zeta, dtype=float)
    n = len(z)
    eye = np.eye(n)
    out = np.zeros((n, 2, n, n))                          # [s, a2, a1 = j, ua = i]
    for s in range(n):
        sym = np.outer(eye[s], z)                         # z_i [j = s]
        out[s, 0] = sym + sym.T
        out[s, 1] = sym - sym.T
    return out.reshape(-1) / (2.0 * np.sqrt(n))


def swap_iterate(zeta: np.ndarray) -> np.ndarray:
    """Block-diagonal Q over the address: block s = -A S_s A^T S_good on [ua | a1 | a2], with
    A = (H on a2) (SWAP(ua, a1) controlled by a2) (H on a2) (U_V on ua), S_good = -Z on a2 (a
    sign flip of a2 = 0) and S_s the sign flip of |0>_ua |s>_a1 |0>_a2."""
    z = np.asarray(zeta, dtype=float)
    n = len(z)
    w = np.eye(n)[0] - z
    uv = np.eye(n) if w @ w < 1e-300 else np.eye(n) - 2.0 * np.outer(w, w) / (w @ w)
    nn = n * n
    swap = np.zeros((nn, nn))
    idx = np.arange(nn)
    swap[(idx % n) * n + idx // n, idx] = 1.0              # |i>_ua |j>_a1 -> |j>_ua |i>_a1
    cswap = np.zeros((2 * nn, 2 * nn))
    cswap[:nn, :nn] = np.eye(nn)
    cswap[nn:, nn:] = swap
    h2 = np.kron(np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0), np.eye(nn))
    amat = h2 @ cswap @ h2 @ np.kron(np.eye(2 * n), uv)
    s_good = np.diag(np.r_[-np.ones(nn), np.ones(nn)])
    out = np.zeros((n * 2 * nn, n * 2 * nn))
    for s in range(n):
        s_s = np.eye(2 * nn)
        s_s[n * s, n * s] = -1.0
        out[s * 2 * nn:(s + 1) * 2 * nn, s * 2 * nn:(s + 1) * 2 * nn] = -amat @ s_s @ amat.T @ s_good
    return out


def swap_rotation_table(n_clock: int, c: float = 1.0) -> np.ndarray:
    """theta_y = 2 arcsin(c (2 sin^2(pi y / 2^r) - 1)), y < 2^r."""
    y = np.arange(1 << n_clock, dtype=float)
    return 2.0 * np.arcsin(c * (2.0 * np.square(np.sin(np.pi * y / float(1 << n_clock))) - 1.0))


def square_amplitudes(zeta, n_clock: int, c: float = 1.0, precision: str = "c64", gemm: str = "simt",
                      form: str = "ae") -> dict:
    """Run the transform on the GPU; returns the postselected system vector ``v``, the address
    amplitudes ``squares`` ~ c z^2 / sqrt(2^a) (each address block projected on its starting
    state: |zeta> for ``form="ae"``, the STEPS 1-3 state for ``form="swap"``), the success
    probability and the final ``state``."""
    from . import HHLPlan

    z = np.asarray(zeta, dtype=float)
    n = len(z)
    a = int(np.log2(n))
    if (1 << a) != n:
        raise ValueError("len(zeta) must be a power of two")
    if form == "ae":
        n_sys, q, table = 2 * a, iterate(z), rotation_table(n_clock, c)
        b = np.kron(np.full(n, 1.0 / np.sqrt(n)), z)
    elif form == "swap":
        n_sys, q, table = 3 * a + 1, swap_iterate(z), swap_rotation_table(n_clock, c)
        b = swap_register_state(z)
    else:
        raise ValueError("form must be 'ae' or 'swap'")
    plan = HHLPlan(n_sys, n_clock, unitary=q, theta_table=table, precision=precision, gemm=gemm)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    meas = plan.measure(st)
    v = meas["xhat"] * np.sqrt(meas["p_success"])
    start = b.reshape(n, -1) * np.sqrt(n)
    return dict(v=v, squares=np.einsum("sk,sk->s", start, v.reshape(n, -1)), p_success=meas["p_success"],
                state=st, plan=plan)
