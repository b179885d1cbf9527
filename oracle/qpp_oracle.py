"""Plain FP64 oracle of the quantum post-processing (QPP) of App. D: the dissipation rate by a
linear combination of unitaries (LCU derivative) and the nonlinear transform of amplitudes
(QADC, squaring rotation, QDAC) in its amplitude-estimation and swap-test forms. TEST
INFRASTRUCTURE ONLY: only ``tests/`` may import it; it shares no code with the library.

The finite-difference derivative of the velocity field with its Dirichlet walls is written
as the difference of two unitaries on a register of 2N points that holds the interior
velocities u_1 .. u_N at positions 0 .. N-1, the wall value u_{N+1} at position N, the wall
value u_0 at position 2N-1 and zeros elsewhere (w): with P the cyclic increment,
(w - P w)_j = w_j - w_{j-1} gives every forward difference u_{i+1} - u_i, i = 0 .. N, plus two
spurious terms -u_{N+1} (position N+1) and u_0 (position 2N-1) that involve only the known
wall values. The LCU circuit (one ancilla, the most significant qubit): prepare the ancilla
with H (the coefficients 1, 1 of I and -P), apply Z on the ancilla and P controlled by it,
undo with H; the probability of ancilla 0 is ||(w~ - P w~) / 2||^2 for the normalised w~, so
sum_i (u_{i+1} - u_i)^2 = 4 p0 |w|^2 - u_0^2 - u_{N+1}^2 and eps = nu / h times that
(h = 1/(N+1)): the dissipation of Sec. VII read from one probability instead of the whole
vector.
"""
from __future__ import annotations

import numpy as np

from oracle import hhl_oracle as o


def lcu_register(u: np.ndarray, wall_lo: float, wall_hi: float) -> np.ndarray:
    """w: u at 0 .. N-1, wall_hi at N, wall_lo at 2N-1, zeros elsewhere."""
    n = len(u)
    w = np.zeros(2 * n)
    w[:n] = u
    w[n] = wall_hi
    w[2 * n - 1] = wall_lo
    return w


def lcu_probability(w: np.ndarray) -> float:
    """Run the LCU circuit gate by gate on [ancilla | data] and return P(ancilla = 0)."""
    m = int(round(np.log2(len(w))))
    n_q = m + 1
    psi = np.zeros(2 * len(w), dtype=np.complex128)
    psi[:len(w)] = w / np.linalg.norm(w)
    o.apply_1q(psi, n_q, m, o.H_GATE)
    o.apply_1q(psi, n_q, m, np.array([[1.0, 0.0], [0.0, -1.0]]))    # Z: the coefficient -1 of P
    perm = np.zeros((len(w), len(w)))
    for j in range(len(w)):
        perm[(j + 1) % len(w), j] = 1.0                               # P |j> = |j + 1 mod 2N>
    o.apply_register_unitary(psi, n_q, 0, m, perm, control=m)
    o.apply_1q(psi, n_q, m, o.H_GATE)
    return float(np.sum(np.abs(psi[:len(w)]) ** 2))


def qpp_dissipation(u: np.ndarray, wall_lo: float, wall_hi: float, nu: float) -> tuple[float, float]:
    """(eps, p0): the dissipation rate from the LCU circuit's ancilla-0 probability."""
    w = lcu_register(u, wall_lo, wall_hi)
    p0 = lcu_probability(w)
    h = 1.0 / (len(u) + 1)
    sq = 4.0 * p0 * float(w @ w) - wall_lo ** 2 - wall_hi ** 2
    return nu * sq / h, p0


# ---------------------------------------------------------------------------------------
# QADC - squaring rotation - QDAC (App. D nonlinear transform): sum_k z_k |k> -> ~ sum_k z_k^2 |k>
# ---------------------------------------------------------------------------------------


def state_prep_unitary(zeta: np.ndarray) -> np.ndarray:
    """A real orthogonal U_V with U_V |0> = |zeta> (the Householder reflection that swaps e_0
    and zeta; the identity when zeta = e_0)."""
    n = len(zeta)
    v = -np.asarray(zeta, dtype=float).copy()
    v[0] += 1.0
    nv = float(v @ v)
    if nv < 1e-300:
        return np.eye(n)
    return np.eye(n) - 2.0 * np.outer(v, v) / nv


def amplitude_estimation_iterate(zeta: np.ndarray) -> np.ndarray:
    """Q = sum_k |k><k|_address (x) G_k on [address | data] (system index d + k N, address the
    high half): G_k = -U_V S_0 U_V^T S_k, S_0 / S_k the reflections flipping |0> / |k> of the
    data register. G_k rotates by 2 theta_k in the plane of |zeta>, sin theta_k = |zeta_k|,
    so phase estimation of Q from |k>|zeta> reads +- theta_k / pi (amplitude estimation,
    the analog-to-digital conversion of the amplitudes)."""
    n = len(zeta)
    uv = state_prep_unitary(zeta)
    s0 = np.eye(n)
    s0[0, 0] = -1.0
    q = np.zeros((n * n, n * n))
    for k in range(n):
        sk = np.eye(n)
        sk[k, k] = -1.0
        q[k * n:(k + 1) * n, k * n:(k + 1) * n] = -uv @ s0 @ uv.T @ sk
    return q


def squaring_angles(n_clock: int, c: float) -> np.ndarray:
    """theta_y with sin(theta_y / 2) = c sin^2(pi y / 2^n_c): the ancilla amplitude becomes
    c sin^2 theta_k = c zeta_k^2 for either estimated phase +- theta_k / pi."""
    y = np.arange(1 << n_clock)
    return 2.0 * np.arcsin(c * np.sin(np.pi * y / (1 << n_clock)) ** 2)


def qadc_square(zeta: np.ndarray, n_clock: int, c: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Run the HHL-shaped circuit (address uniform, data |zeta>; phase estimation of Q, the
    squaring rotation, the inverse) gate by gate in the oracle; return (the final state, the
    postselected [address | data] vector)."""
    n = len(zeta)
    a = int(round(np.log2(n)))
    q = amplitude_estimation_iterate(zeta)
    evolutions = []
    u = q.copy()
    for _ in range(n_clock):
        evolutions.append(u.astype(np.complex128))
        u = u @ u
    b = np.kron(np.full(n, 1.0 / np.sqrt(n)), np.asarray(zeta, dtype=float))
    pl = dict(n_clock=n_clock, theta=squaring_angles(n_clock, c), t0=2.0 * np.pi)
    psi = o.hhl_circuit(b, 2 * a, pl, evolutions=evolutions)
    return psi, o.postselect(psi, 2 * a, n_clock)["v"]


# ---------------------------------------------------------------------------------------
# The swap-test form of the QADC (App. D, STEPS 1-5): registers ua (the data, a qubits),
# a1 (the clone of the address, a qubits), a2 (the swap-test qubit) and the address
# (a qubits), laid out low to high in the system index ua + N a1 + N^2 a2 + 2 N^2 s.
# ---------------------------------------------------------------------------------------

X_GATE = np.array([[0.0, 1.0], [1.0, 0.0]])


def _controlled_swap(psi: np.ndarray, n_q: int, c: int, x: int, y: int) -> None:
    """Fredkin gate (SWAP of qubits x and y when qubit c is 1) as CNOT(y -> x),
    Toffoli(c, x -> y), CNOT(y -> x)."""
    o.apply_1q(psi, n_q, x, X_GATE, controls=(y,))
    o.apply_1q(psi, n_q, y, X_GATE, controls=(c, x))
    o.apply_1q(psi, n_q, x, X_GATE, controls=(y,))


def _swap_test_block(psi: np.ndarray, n_q: int, a: int, zeta: np.ndarray, inverse: bool = False) -> None:
    """A = V (U_V on ua): U_V, then the swap test without measurement (H on a2, ua and a1
    swapped qubit by qubit under control of a2, H on a2); ``inverse`` applies A^T (every
    gate is real and self-inverse except U_V, a reflection, so the reversed order is A^T)."""
    uv = state_prep_unitary(zeta)
    gates = [("uv",), ("h",)] + [("cswap", j) for j in range(a)] + [("h",)]
    for g in (reversed(gates) if inverse else gates):
        if g[0] == "uv":
            o.apply_register_unitary(psi, n_q, 0, a, uv)
        elif g[0] == "h":
            o.apply_1q(psi, n_q, 2 * a, o.H_GATE)
        else:
            _controlled_swap(psi, n_q, 2 * a, g[1], a + g[1])


def swap_test_prepare(zeta: np.ndarray) -> np.ndarray:
    """STEPS 1-3 gate by gate from |0>: Hadamards on the address, CNOTs cloning each address
    qubit into a1, then A on [ua | a1 | a2]. Returns the 2 N^3 state."""
    n = len(zeta)
    a = int(round(np.log2(n)))
    n_q = 3 * a + 1
    psi = np.zeros(1 << n_q, dtype=np.complex128)
    psi[0] = 1.0
    for j in range(a):
        o.apply_1q(psi, n_q, 2 * a + 1 + j, o.H_GATE)
    for j in range(a):
        o.apply_1q(psi, n_q, a + j, X_GATE, controls=(2 * a + 1 + j,))
    _swap_test_block(psi, n_q, a, zeta)
    return psi


def swap_test_iterate(zeta: np.ndarray) -> np.ndarray:
    """Q = sum_s |s><s|_address (x) P_s with P_s = -A S_s A^T S_good on [ua | a1 | a2]:
    S_good flips the sign of a2 = 0 (the component whose weight the swap test makes
    (1 + zeta_s^2) / 2), S_s the sign of the start state |0>_ua |s>_a1 |0>_a2 (the
    conditional phase shift of STEP 4). Built column by column by running the gates on
    basis states."""
    n = len(zeta)
    a = int(round(np.log2(n)))
    n_q = 2 * a + 1
    dim = 1 << n_q
    good = np.where(np.arange(dim) < n * n, -1.0, 1.0)        # a2 = 0 is the low N^2 block
    q = np.zeros((n * dim, n * dim))
    for s in range(n):
        start = n * s                                          # |0>_ua |s>_a1 |0>_a2
        blk = np.zeros((dim, dim))
        for col in range(dim):
            psi = np.zeros(dim, dtype=np.complex128)
            psi[col] = good[col]
            _swap_test_block(psi, n_q, a, zeta, inverse=True)
            psi[start] = -psi[start]
            _swap_test_block(psi, n_q, a, zeta)
            blk[:, col] = -psi.real
        q[s * dim:(s + 1) * dim, s * dim:(s + 1) * dim] = blk
    return q


def swap_squaring_angles(n_clock: int, c: float) -> np.ndarray:
    """theta_y with sin(theta_y / 2) = c (2 sin^2(pi y / 2^n_c) - 1): for an estimate of
    sin^2(pi beta) = (1 + zeta_s^2) / 2 (either of beta, 1 - beta) the ancilla amplitude
    becomes c zeta_s^2."""
    y = np.arange(1 << n_clock)
    return 2.0 * np.arcsin(c * (2.0 * np.sin(np.pi * y / (1 << n_clock)) ** 2 - 1.0))


def qadc_swap_square(zeta: np.ndarray, n_clock: int, c: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """The HHL-shaped circuit on the swap-test register (STEPS 1-3 state, phase estimation
    of Q, the squaring rotation, the inverse), gate by gate; returns (the final state, the
    postselected system vector)."""
    n = len(zeta)
    a = int(round(np.log2(n)))
    n_s = 3 * a + 1
    q = swap_test_iterate(zeta)
    evolutions = []
    u = q.copy()
    for _ in range(n_clock):
        evolutions.append(u.astype(np.complex128))
        u = u @ u
    b = swap_test_prepare(zeta)
    pl = dict(n_clock=n_clock, theta=swap_squaring_angles(n_clock, c), t0=2.0 * np.pi)
    psi = o.hhl_circuit(b, n_s, pl, evolutions=evolutions)
    return psi, o.postselect(psi, n_s, n_clock)["v"]


def swap_squares(v: np.ndarray, zeta: np.ndarray) -> np.ndarray:
    """The address amplitudes of a postselected swap-register vector: each address block
    projected on its STEPS 1-3 state A |0>_ua |s>_a1 |0>_a2 (undoing A and the clone)."""
    n = len(zeta)
    prep = swap_test_prepare(zeta).reshape(n, -1) * np.sqrt(n)
    return np.einsum("sk,sk->s", prep.conj(), np.asarray(v).reshape(n, -1))
