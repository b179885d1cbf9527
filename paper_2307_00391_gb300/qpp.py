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

This module only marshals: the iterate, the rotation tables, the start states and the
projection of the result are the library's host calls hhl_qpp_iterate, hhl_qpp_rotation_table,
hhl_qpp_start_state and hhl_qpp_project (include/hhl.h).
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._ffi import check, load

_FORM = {"ae": 0, "swap": 1}


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _bits(zeta) -> tuple[np.ndarray, int]:
    z = np.ascontiguousarray(zeta, dtype=np.float64)
    a = int(np.log2(len(z)))
    if (1 << a) != len(z):
        raise ValueError("len(zeta) must be a power of two")
    return z, a


def _dim(a: int, form: str) -> int:
    n = 1 << a
    return n * n if form == "ae" else 2 * n ** 3


def iterate(zeta: np.ndarray, form: str = "ae") -> np.ndarray:
    """The iterate Q (hhl_qpp_iterate): block diagonal over the address, block k =
    -U_V S_0 U_V^T S_k on the data register (U_V the Householder reflection taking |0> to
    |zeta>; S_j flips the sign of |j>)."""
    z, a = _bits(zeta)
    d = _dim(a, form)
    q = np.zeros((d, d), dtype=np.float64)
    check(load().hhl_qpp_iterate(_ptr(z), a, _FORM[form], _ptr(q)), "hhl_qpp_iterate")
    return q


def rotation_table(n_clock: int, c: float = 1.0, form: str = "ae") -> np.ndarray:
    """theta_y = 2 arcsin(c sin^2(pi y / 2^r)) (form "ae") or 2 arcsin(c (2 sin^2 - 1)) ("swap")."""
    t = np.zeros(1 << n_clock, dtype=np.float64)
    check(load().hhl_qpp_rotation_table(n_clock, float(c), _FORM[form], _ptr(t)), "hhl_qpp_rotation_table")
    return t


def swap_register_state(zeta: np.ndarray) -> np.ndarray:
    """The state after STEPS 1-3 (uniform address, clone, U_V, swap test without measurement)."""
    z, a = _bits(zeta)
    b = np.zeros(_dim(a, "swap"), dtype=np.float64)
    check(load().hhl_qpp_start_state(_ptr(z), a, 1, _ptr(b)), "hhl_qpp_start_state")
    return b


def swap_iterate(zeta: np.ndarray) -> np.ndarray:
    """The swap-test iterate: block s = -A S_s A^T S_good on [ua | a1 | a2]."""
    return iterate(zeta, form="swap")


def swap_rotation_table(n_clock: int, c: float = 1.0) -> np.ndarray:
    """theta_y = 2 arcsin(c (2 sin^2(pi y / 2^r) - 1)), y < 2^r."""
    return rotation_table(n_clock, c, form="swap")


def square_amplitudes(zeta, n_clock: int, c: float = 1.0, precision: str = "c64", gemm: str = "simt",
                      form: str = "ae") -> dict:
    """Run the transform on the GPU; returns the postselected system vector ``v``, the address
    amplitudes ``squares`` ~ c z^2 / sqrt(2^a) (each address block projected on its starting
    state: |zeta> for ``form="ae"``, the STEPS 1-3 state for ``form="swap"``), the success
    probability and the final ``state``."""
    from . import HHLPlan

    if form not in _FORM:
        raise ValueError("form must be 'ae' or 'swap'")
    z, a = _bits(zeta)
    n_sys = 2 * a if form == "ae" else 3 * a + 1
    q = iterate(z, form)
    table = rotation_table(n_clock, c, form)
    b = np.zeros(_dim(a, form), dtype=np.float64)
    check(load().hhl_qpp_start_state(_ptr(z), a, _FORM[form], _ptr(b)), "hhl_qpp_start_state")
    plan = HHLPlan(n_sys, n_clock, unitary=q, theta_table=table, precision=precision, gemm=gemm)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    meas = plan.measure(st)
    # v: the anc = 1, clock = 0 row of the final state
    v = st.view(2, 1 << n_clock, -1)[1, 0].cpu().numpy().astype(np.complex128)
    sq = np.zeros(2 << a, dtype=np.float64)
    check(load().hhl_qpp_project(_ptr(v), _ptr(b), a, _FORM[form], _ptr(sq)), "hhl_qpp_project")
    return dict(v=v, squares=sq[0::2] + 1j * sq[1::2], p_success=meas["p_success"], state=st, plan=plan)
