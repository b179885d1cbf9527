"""Plain FP64 CPU oracle of the HHL (QLSA-1) state-vector path of QFlowS.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm
may import or run it. It shares no code, table or constant generator with the CUDA
library; the two meet only through the seeded inputs of ``synth_inputs``.

What it computes, step by step, in complex128 with index loops or one numpy/scipy
library call per step (no blocking, fusion or reordering):

* the steady channel operator, Sec. II Eq. (poiseuille flow) with the central-difference
  Laplacian of App. A.1 Eq. (CDS): A = tridiag(-1, 2, -1)/h^2, h = 1/(N+1);
* a direct classical solve of A x = b (Thomas algorithm) as the target of the method;
* the gate-level HHL circuit of Sec. IV / VI: amplitude-encoded right-hand side, Hadamards
  on the clock, clock-bit-controlled U_k = exp(i Ahat t_k), inverse QFT, clock-controlled
  RY on the ancilla (eigenvalue inversion), then the mirror image (QFT, controlled U_k^dagger,
  Hadamards), and postselection on ancilla = 1, clock = 0;
* the viscous dissipation rate eps = nu <(du/dy)^2> of Sec. VII / App. D, evaluated with
  the same finite-difference post-processing as the classical solution;
* the Grover-Rudolph binary-tree state preparation QSP-1 of App. C, and QSP-2 (Sec. III,
  App. C): the same rotations only on the nodes of the decision tree that lie on a path to a
  nonzero leaf, as multi-controlled gates (X gates around the controls that must read 0);
* the second-order (Strang) Trotter product for exp(i Ahat t) on a tridiagonal Ahat, gate
  by gate (paper silent; reading below).

Register layout (shared with the library's interface, not with its code): amplitude
index = sys | clk << n_s | anc << (n_s + n_c); qubit q is index bit q (q = 0 is the least
significant bit). The two-qubit example of App. B (U = H_1 (x) X_0 equals kron(H, X))
fixes that the qubit with the larger label is the more significant bit.

Readings where the paper is silent or ambiguous (each one is also listed in the design
notes of the repository):

* Ahat = A / lambda_ub with lambda_ub the Gershgorin bound max_i sum_j |A_ij| (4/h^2 for the
  Laplacian).
* U_k = exp(+i Ahat T0 2^k / 2^n_c) ("total" T0 convention); the clock then reads
  y ~ lambda T0 / (2 pi). A "per-unit" T0 is converted by T0_total = 2^n_c T0_per_unit.
* QFT|x> = 2^(-m/2) sum_y exp(+2 pi i x y / 2^m)|y>; the inverse QFT is its inverse.
* C = 2 pi / T0 unless given; theta_y = 2 arcsin(min(1, C / lambda~_y)), lambda~_y =
  2 pi y / T0, theta_0 = 0; RY(theta) = exp(-i theta Y / 2).
* T0 rules: "range_fill" T0 = 2 pi (2^n_c - 1) maps Ahat's bound 1 to the top clock value;
  "power_law" T0_per_unit = exp(0.918) kappa^(-0.363) (the fit of Sec. VI read as a power
  law; parity unpinned, a fallback only).
* Denormalisation: the postselected vector v approximates C Ahat^{-1} bhat, so the velocity
  is u = |b| v / (C lambda_ub).
* Dissipation: forward differences including both walls, eps = nu h sum_{i=0}^{N}
  ((u_{i+1} - u_i)/h)^2.
* Trotter: Ahat = E + O with E the 2x2 blocks on pairs (2i, 2i+1) carrying the whole
  diagonal and O the couplings of pairs (2i+1, 2i+2); one step S(tau) = E(tau/2) O(tau)
  E(tau/2) with E(s) = exp(i s E); r_k = clamp(ceil(t_k / dt), 1, r_max) steps for U_k.

Parity unpinned: the power-law T0 rule (the paper's own fit does not reproduce its printed
T0* at its printed kappa under any reading).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

# ---------------------------------------------------------------------------------------
# Problem: App. A.1 Eq. (CDS) and Sec. II Eq. (poiseuille flow)
# ---------------------------------------------------------------------------------------


def laplacian_tridiag(n_points: int) -> tuple[np.ndarray, np.ndarray]:
    """(diag, off) of A = tridiag(-1, 2, -1)/h^2 with h = 1/(N+1) (App. A.1 Eq. CDS)."""
    h = 1.0 / (n_points + 1)
    diag = np.full(n_points, 2.0 / (h * h))
    off = np.full(n_points - 1, -1.0 / (h * h))
    return diag, off


def dense_from_tridiag(diag: np.ndarray, off: np.ndarray) -> np.ndarray:
    """Dense symmetric matrix with the given diagonal and first off-diagonals."""
    n = len(diag)
    a = np.zeros((n, n))
    for i in range(n):
        a[i, i] = diag[i]
    for i in range(n - 1):
        a[i, i + 1] = off[i]
        a[i + 1, i] = off[i]
    return a


def thomas_solve(diag: np.ndarray, off: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Direct solve of a symmetric tridiagonal system (Thomas algorithm), the classical
    target the quantum solution is compared with (Sec. V: fidelity |u_Q . u_C|)."""
    n = len(diag)
    c = np.zeros(n)
    d = np.zeros(n, dtype=np.result_type(b, np.float64))
    beta = diag[0]
    c[0] = (off[0] / beta) if n > 1 else 0.0
    d[0] = b[0] / beta
    for i in range(1, n):
        beta = diag[i] - off[i - 1] * c[i - 1]
        if i < n - 1:
            c[i] = off[i] / beta
        d[i] = (b[i] - off[i - 1] * d[i - 1]) / beta
    x = np.zeros_like(d)
    x[n - 1] = d[n - 1]
    for i in range(n - 2, -1, -1):
        x[i] = d[i] - c[i] * x[i + 1]
    return x


def gershgorin_bound(a: np.ndarray) -> float:
    """max_i sum_j |a_ij|: an upper bound of the spectral radius, used as lambda_ub."""
    return float(np.max(np.sum(np.abs(a), axis=1)))


def condition_number(a: np.ndarray) -> float:
    """kappa = |lambda|_max / |lambda|_min of a Hermitian matrix (library eigvalsh)."""
    w = np.abs(np.linalg.eigvalsh(a))
    return float(w.max() / w.min())


def wolkowicz_bounds(a: np.ndarray) -> tuple[float, float, float, float]:
    """Eigenvalue bounds quoted in Sec. VI: with b1 = Tr A / N and
    b2 = (Tr A^2 / N - b1^2)^(1/2): b1 - b2 sqrt(N-1) <= lambda_min <= b1 - b2/sqrt(N-1) and
    b1 + b2/sqrt(N-1) <= lambda_max <= b1 + b2 sqrt(N-1).
    Returns (lmin_lo, lmin_hi, lmax_lo, lmax_hi)."""
    n = a.shape[0]
    b1 = np.trace(a).real / n
    b2 = math.sqrt(max(np.trace(a @ a).real / n - b1 * b1, 0.0))
    r = math.sqrt(n - 1)
    return b1 - b2 * r, b1 - b2 / r, b1 + b2 / r, b1 + b2 * r


# ---------------------------------------------------------------------------------------
# Planning scalars (Sec. VI: T0, least count, eigenvalue inversion)
# ---------------------------------------------------------------------------------------


def t0_total(rule: str, n_clock: int, kappa: float | None = None, t0: float | None = None,
             convention: str = "total") -> float:
    """Hamiltonian-simulation time T0 in the "total" convention (U_k = exp(i Ahat T0 2^k/2^n_c))."""
    if rule == "range_fill":
        return 2.0 * math.pi * ((1 << n_clock) - 1)
    if rule == "range_fill_signed":
        # signed clock: lambdahat = +-1 maps to the clock values +-(2^(n_c-1) - 1)
        return 2.0 * math.pi * ((1 << (n_clock - 1)) - 1)
    if rule == "power_law":
        per_unit = math.exp(0.918) * kappa ** (-0.363)
        return per_unit * (1 << n_clock)
    if rule == "user":
        return t0 * (1 << n_clock) if convention == "per_unit" else t0
    raise ValueError(rule)


def rotation_angles(n_clock: int, t0: float, c_const: float | None = None,
                    signed: bool = False) -> np.ndarray:
    """theta_y for clock values y = 0 .. 2^n_c - 1: the ancilla amplitude after the
    controlled RY is sin(theta_y/2) = min(1, C / lambda~_y), lambda~_y = 2 pi y / T0,
    and theta_0 = 0 (Sec. IV/VI eigenvalue inversion, reading of C and y = 0).

    signed: the clock value is read in two's complement, y_s = y - 2^n_c for
    y >= 2^(n_c-1), so that a negative eigenvalue (an indefinite A, such as the Hermitian
    dilation of a one-shot time-stepping system) gets lambda~ = 2 pi y_s / T0 < 0 and a
    negative amplitude, sin(theta_y/2) = max(-1, min(1, C / lambda~))."""
    if c_const is None:
        c_const = 2.0 * math.pi / t0
    th = np.zeros(1 << n_clock)
    half = 1 << (n_clock - 1)
    for y in range(1, 1 << n_clock):
        ys = y - (1 << n_clock) if (signed and y >= half) else y
        lam = 2.0 * math.pi * ys / t0
        th[y] = 2.0 * math.asin(max(-1.0, min(1.0, c_const / lam)))
    return th


# ---------------------------------------------------------------------------------------
# Gates on a flat complex128 state (App. B: gates act algebraically on amplitude pairs)
# ---------------------------------------------------------------------------------------

H_GATE = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
X_GATE = np.array([[0.0, 1.0], [1.0, 0.0]])


def ry(theta: float) -> np.ndarray:
    """RY(theta) = exp(-i theta Y/2) = [[cos, -sin], [sin, cos]](theta/2)."""
    c, s = math.cos(theta / 2.0), math.sin(theta / 2.0)
    return np.array([[c, -s], [s, c]])


def _pair_view(psi: np.ndarray, n: int, qa: int, qb: int) -> tuple[np.ndarray, bool]:
    """5-D view of psi with separate length-2 axes for qubits qa != qb. Returns the view
    and whether axis 1 is qa (True) or qb (False); axis 1 is always the higher qubit."""
    hi, lo = max(qa, qb), min(qa, qb)
    v = psi.reshape((1 << (n - 1 - hi), 2, 1 << (hi - lo - 1), 2, 1 << lo))
    return v, hi == qa


def apply_1q(psi: np.ndarray, n: int, q: int, u: np.ndarray, controls=()) -> None:
    """Apply the 2x2 matrix u to qubit q, conditioned on every qubit in ``controls``
    being 1. psi[i] pairs with psi[i + 2^q] (bit q clear / set)."""
    t = psi.reshape((1 << (n - 1 - q), 2, 1 << q))
    if not controls:
        a0 = t[:, 0, :].copy()
        a1 = t[:, 1, :].copy()
        t[:, 0, :] = u[0, 0] * a0 + u[0, 1] * a1
        t[:, 1, :] = u[1, 0] * a0 + u[1, 1] * a1
        return
    idx = np.arange(1 << n).reshape(t.shape)[:, 0, :]
    mask = np.ones(idx.shape, dtype=bool)
    for c in controls:
        mask &= ((idx >> c) & 1) == 1
    v0 = t[:, 0, :]
    v1 = t[:, 1, :]
    a0 = v0[mask].copy()
    a1 = v1[mask].copy()
    v0[mask] = u[0, 0] * a0 + u[0, 1] * a1
    v1[mask] = u[1, 0] * a0 + u[1, 1] * a1


def apply_cphase(psi: np.ndarray, n: int, q1: int, q2: int, phi: float) -> None:
    """Controlled phase: multiply amplitudes whose bits q1 and q2 are both 1 by e^{i phi}."""
    v, _ = _pair_view(psi, n, q1, q2)
    v[:, 1, :, 1, :] *= np.exp(1j * phi)


def apply_swap(psi: np.ndarray, n: int, q1: int, q2: int) -> None:
    """SWAP of qubits q1 and q2 (exchange the amplitudes whose two bits are 10 and 01)."""
    if q1 == q2:
        return
    v, _ = _pair_view(psi, n, q1, q2)
    tmp = v[:, 1, :, 0, :].copy()
    v[:, 1, :, 0, :] = v[:, 0, :, 1, :]
    v[:, 0, :, 1, :] = tmp


def apply_register_unitary(psi: np.ndarray, n: int, lo: int, m: int, u: np.ndarray,
                           control: int | None = None) -> None:
    """Apply the 2^m x 2^m matrix u to the register of bits [lo, lo+m), conditioned on
    qubit ``control`` (outside the register) being 1 if given:
    |rest>|x> -> |rest> u|x> for every selected value of the remaining bits."""
    t = psi.reshape((1 << (n - lo - m), 1 << m, 1 << lo))
    outer = np.arange(1 << (n - lo - m))[:, None] << (lo + m)
    inner = np.arange(1 << lo)[None, :]
    rest = outer | inner
    sel = np.ones(rest.shape, dtype=bool) if control is None else ((rest >> control) & 1) == 1
    tt = np.moveaxis(t, 1, 2)            # (rest_hi, rest_lo, register) view
    vecs = tt[sel]                       # one register vector per selected row
    tt[sel] = vecs @ u.T


def qft(psi: np.ndarray, n: int, lo: int, m: int, inverse: bool = False) -> None:
    """QFT on the register of bits [lo, lo+m) as a gate sequence: for each qubit from the
    most significant down, a Hadamard then controlled phases pi/2^(j-l) from every lower
    qubit l, then the bit-reversal swap layer. Implements
    QFT|x> = 2^(-m/2) sum_y exp(+2 pi i x y / 2^m)|y>; ``inverse`` applies the exact inverse
    (the same gates in reverse order with conjugated phases)."""
    gates = []
    for j in range(m - 1, -1, -1):
        gates.append(("h", j))
        for l in range(j - 1, -1, -1):
            gates.append(("cp", j, l, math.pi / (1 << (j - l))))
    for i in range(m // 2):
        gates.append(("swap", i, m - 1 - i))
    if inverse:
        gates = gates[::-1]
    for g in gates:
        if g[0] == "h":
            apply_1q(psi, n, lo + g[1], H_GATE)
        elif g[0] == "cp":
            apply_cphase(psi, n, lo + g[1], lo + g[2], -g[3] if inverse else g[3])
        else:
            apply_swap(psi, n, lo + g[1], lo + g[2])


def apply_clock_controlled_ry(psi: np.ndarray, n_s: int, n_c: int, theta: np.ndarray,
                              adjoint: bool = False) -> None:
    """For every clock value y, RY(theta_y) on the ancilla conditioned on clock == y
    (a uniformly controlled rotation)."""
    s = psi.reshape((2, 1 << n_c, 1 << n_s))
    for y in range(1 << n_c):
        u = ry(-theta[y] if adjoint else theta[y])
        a0 = s[0, y, :].copy()
        a1 = s[1, y, :].copy()
        s[0, y, :] = u[0, 0] * a0 + u[0, 1] * a1
        s[1, y, :] = u[1, 0] * a0 + u[1, 1] * a1


# ---------------------------------------------------------------------------------------
# Hamiltonian simulation: dense exponential (Sec. VI) and Strang-Trotter product
# ---------------------------------------------------------------------------------------


def evolution_dense(a_hat: np.ndarray, t: float) -> np.ndarray:
    """exp(i Ahat t) by the library matrix exponential."""
    return scipy.linalg.expm(1j * t * a_hat)


def trotter_steps(t: float, dt: float, r_max: int) -> int:
    """r = clamp(ceil(t/dt), 1, r_max) Strang steps for an evolution time t."""
    r = int(math.ceil(t / dt)) if dt > 0 else 1
    r = max(r, 1)
    if r_max > 0:
        r = min(r, r_max)
    return r


def trotter_unitary(diag_hat: np.ndarray, off_hat: np.ndarray, t: float, r: int) -> np.ndarray:
    """S(t/r)^r with S(tau) = E(tau/2) O(tau) E(tau/2) as a dense matrix (small N only).
    E(s) = exp(i s E): 2x2 blocks [[d_2i, o_2i], [o_2i, d_2i+1]] on pairs (2i, 2i+1).
    O(s) = exp(i s O): blocks [[0, o_2i+1], [o_2i+1, 0]] on pairs (2i+1, 2i+2)."""
    n = len(diag_hat)
    tau = t / r

    def layer(start: int, s: float, with_diag: bool) -> np.ndarray:
        g = np.eye(n, dtype=complex)
        for i in range(start, n - 1, 2):
            blk = np.array([[diag_hat[i] if with_diag else 0.0, off_hat[i]],
                            [off_hat[i], diag_hat[i + 1] if with_diag else 0.0]])
            g[i:i + 2, i:i + 2] = scipy.linalg.expm(1j * s * blk)
        return g

    e_half = layer(0, tau / 2.0, True)
    o_full = layer(1, tau, False)
    step = e_half @ o_full @ e_half
    u = np.eye(n, dtype=complex)
    for _ in range(r):
        u = step @ u
    return u


def _pair_blocks(diag_hat: np.ndarray, off_hat: np.ndarray, start: int, s: float,
                 with_diag: bool) -> np.ndarray:
    """exp(i s M_i) for the 2x2 blocks M_i = [[d_i, o_i], [o_i, d_i+1]] (or without the
    diagonal) of the pairs (i, i+1), i = start, start+2, ...; equal blocks share one
    library exponential."""
    n = len(diag_hat)
    cache: dict = {}
    out = []
    for i in range(start, n - 1, 2):
        key = (diag_hat[i] if with_diag else 0.0, off_hat[i], diag_hat[i + 1] if with_diag else 0.0)
        if key not in cache:
            blk = np.array([[key[0], key[1]], [key[1], key[2]]])
            cache[key] = scipy.linalg.expm(1j * s * blk)
        out.append(cache[key])
    return np.array(out).reshape(-1, 2, 2)


def apply_trotter_controlled(psi: np.ndarray, n: int, n_s: int, control: int,
                             diag_hat: np.ndarray, off_hat: np.ndarray, t: float, r: int) -> None:
    """Gate by gate: r Strang steps of exp(i Ahat t) on the system register, each 2x2 block
    a two-level gate on basis states (i, i+1), all conditioned on qubit ``control``. The
    gates of one layer act on disjoint pairs and commute, so a layer is applied at once."""
    nsys = 1 << n_s
    tau = t / r
    rows = psi.reshape((-1, nsys))
    ridx = np.arange(rows.shape[0]) << n_s
    sel = ((ridx >> control) & 1) == 1

    def two_level_layer(start: int, s: float, with_diag: bool) -> None:
        g = _pair_blocks(diag_hat, off_hat, start, s, with_diag)
        if g.shape[0] == 0:
            return
        i0 = np.arange(start, nsys - 1, 2)
        sub = rows[sel]
        a0 = sub[:, i0].copy()
        a1 = sub[:, i0 + 1].copy()
        sub[:, i0] = g[:, 0, 0] * a0 + g[:, 0, 1] * a1
        sub[:, i0 + 1] = g[:, 1, 0] * a0 + g[:, 1, 1] * a1
        rows[sel] = sub

    for _ in range(r):
        two_level_layer(0, tau / 2.0, True)
        two_level_layer(1, tau, False)
        two_level_layer(0, tau / 2.0, True)


# ---------------------------------------------------------------------------------------
# The HHL circuit (Sec. IV QLSA-1; Sec. VI phase estimation with exp(i A T0))
# ---------------------------------------------------------------------------------------


def plan(a: np.ndarray, n_clock: int, t0_rule: str = "range_fill", t0: float | None = None,
         t0_convention: str = "total", c_const: float | None = None, signed: bool = False) -> dict:
    """Classical pre-computation (Sec. II.A): Ahat, lambda_ub, kappa, T0, C and theta_y.
    signed: two's-complement clock reading for an indefinite A ("range_fill" then maps
    lambdahat = +-1 to +-(2^(n_c-1) - 1))."""
    lam_ub = gershgorin_bound(a)
    a_hat = a / lam_ub
    kappa = condition_number(a)
    rule = "range_fill_signed" if (signed and t0_rule == "range_fill") else t0_rule
    t0_tot = t0_total(rule, n_clock, kappa=kappa, t0=t0, convention=t0_convention)
    c = (2.0 * math.pi / t0_tot) if c_const is None else c_const
    return dict(lam_ub=lam_ub, a_hat=a_hat, kappa=kappa, t0=t0_tot, C=c,
                theta=rotation_angles(n_clock, t0_tot, c, signed=signed), n_clock=n_clock)


def prepare_state(b: np.ndarray, n_s: int, n_c: int) -> np.ndarray:
    """|0>_anc |0>_clk |bhat>, then a Hadamard on every clock qubit."""
    n = n_s + n_c + 1
    psi = np.zeros(1 << n, dtype=np.complex128)
    bh = np.asarray(b, dtype=np.complex128)
    psi[: 1 << n_s] = bh / np.linalg.norm(bh)
    for q in range(n_s, n_s + n_c):
        apply_1q(psi, n, q, H_GATE)
    return psi


def hhl_circuit(b: np.ndarray, n_s: int, pl: dict, evolutions: list[np.ndarray] | None = None,
                trotter: dict | None = None) -> np.ndarray:
    """Run the whole circuit and return the final 2^(n_s+n_c+1) state.

    ``evolutions[k]`` is U_k (dense path); with ``trotter`` = dict(diag, off, dt, r_max)
    each U_k is instead the Strang product applied gate by gate."""
    n_c = pl["n_clock"]
    n = n_s + n_c + 1
    psi = prepare_state(b, n_s, n_c)
    t_k = [pl["t0"] * (1 << k) / (1 << n_c) for k in range(n_c)]
    if evolutions is None and trotter is None:
        evolutions = [evolution_dense(pl["a_hat"], t) for t in t_k]

    def controlled_u(k: int, adjoint: bool) -> None:
        ctrl = n_s + k
        if trotter is None:
            u = evolutions[k].conj().T if adjoint else evolutions[k]
            apply_register_unitary(psi, n, 0, n_s, u, control=ctrl)
        else:
            r = trotter_steps(t_k[k], trotter["dt"], trotter["r_max"])
            apply_trotter_controlled(psi, n, n_s, ctrl, trotter["diag"], trotter["off"],
                                     -t_k[k] if adjoint else t_k[k], r)

    for k in range(n_c):
        controlled_u(k, False)
    qft(psi, n, n_s, n_c, inverse=True)
    apply_clock_controlled_ry(psi, n_s, n_c, pl["theta"])
    qft(psi, n, n_s, n_c, inverse=False)
    for k in range(n_c - 1, -1, -1):
        controlled_u(k, True)
    for q in range(n_s, n_s + n_c):
        apply_1q(psi, n, q, H_GATE)
    return psi


def postselect(psi: np.ndarray, n_s: int, n_c: int) -> dict:
    """Measurement statistics of the final state: v = amplitudes with ancilla = 1 and
    clock = 0; P_success = |v|^2; xhat = v/|v|; P(anc = 1) = total weight of the anc = 1 half."""
    s = psi.reshape((2, 1 << n_c, 1 << n_s))
    v = s[1, 0, :].copy()
    p_succ = float(np.vdot(v, v).real)
    p_anc1 = float(np.vdot(s[1], s[1]).real)
    norm = float(np.vdot(psi, psi).real)
    xhat = v / math.sqrt(p_succ) if p_succ > 0 else v
    return dict(v=v, p_success=p_succ, p_anc1=p_anc1, norm=norm, xhat=xhat)


def sample_counts(v: np.ndarray, uniforms: np.ndarray) -> np.ndarray:
    """Shots of the system register after postselection (Sec. II.A: the solution is read by
    repeated measurement): outcome j has probability |v_j|^2 / sum |v|^2; shot s with the
    uniform u_s in [0, 1) lands in the bin j with cdf_{j-1} <= u_s * total < cdf_j, where cdf
    is the running sum of |v|^2 (inverse-transform sampling). Returns the N counts."""
    p = np.abs(np.asarray(v, dtype=np.complex128)) ** 2
    cdf = np.cumsum(p)
    idx = np.searchsorted(cdf, np.asarray(uniforms, dtype=np.float64) * cdf[-1], side="right")
    return np.bincount(np.minimum(idx, len(p) - 1), minlength=len(p)).astype(np.int64)


def velocity(v: np.ndarray, b_norm: float, c_const: float, lam_ub: float) -> np.ndarray:
    """Denormalised velocity at the interior nodes: u = |b| Re(v) / (C lambda_ub)."""
    return b_norm * np.real(v) / (c_const * lam_ub)


def dissipation(u: np.ndarray, wall_lo: float, wall_hi: float, nu: float) -> float:
    """eps = nu <(du/dy)^2> (Sec. VII, App. D) by forward differences over the N+1 cells
    between the walls: eps = nu h sum_{i=0}^{N} ((u_{i+1} - u_i)/h)^2."""
    n = len(u)
    h = 1.0 / (n + 1)
    full = np.concatenate(([wall_lo], u, [wall_hi]))
    acc = 0.0
    for i in range(n + 1):
        g = (full[i + 1] - full[i]) / h
        acc += g * g
    return nu * h * acc


def fidelity(x_q: np.ndarray, x_c: np.ndarray) -> float:
    """|<xhat_C | xhat_Q>| of the normalised vectors (Sec. V)."""
    a = x_q / np.linalg.norm(x_q)
    c = x_c / np.linalg.norm(x_c)
    return float(abs(np.vdot(c, a)))


# ---------------------------------------------------------------------------------------
# QSP-1: Grover-Rudolph binary tree (App. C)
# ---------------------------------------------------------------------------------------


def qsp1_angles(prob: np.ndarray) -> list[np.ndarray]:
    """Per tree level l (0 = root), one angle per node: theta = arccos sqrt(p_zero-child /
    p_node) in the paper's R_y convention (R_y(theta)|0> = cos theta|0> + sin theta|1>)."""
    n = int(round(math.log2(len(prob))))
    levels = [np.asarray(prob, dtype=float)]
    for _ in range(n):
        p = levels[0]
        levels.insert(0, p[0::2] + p[1::2])
    out = []
    for l in range(n):
        parent = levels[l]
        child = levels[l + 1]
        ang = np.zeros(len(parent))
        for i in range(len(parent)):
            ang[i] = math.acos(math.sqrt(min(1.0, child[2 * i] / parent[i]))) if parent[i] > 0 else 0.0
        out.append(ang)
    return out


def qsp1_prepare(amplitudes: np.ndarray) -> np.ndarray:
    """Prepare sum_i a_i |i> for real a_i >= 0 with the binary-tree circuit: level l rotates
    qubit n-1-l by R_y(theta) (paper convention, i.e. our RY(2 theta)) conditioned on the
    values of the l more significant qubits."""
    a = np.asarray(amplitudes, dtype=float)
    n = int(round(math.log2(len(a))))
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    angles = qsp1_angles(a * a)
    for l in range(n):
        target = n - 1 - l
        for node in range(1 << l):
            # condition: qubits n-1 .. n-l hold the bits of ``node`` (MSB first)
            idx = np.arange(1 << n)
            prefix = idx >> (target + 1)
            sel_rows = prefix == node
            u = ry(2.0 * angles[l][node])
            t0 = idx[sel_rows & (((idx >> target) & 1) == 0)]
            t1 = t0 | (1 << target)
            a0 = psi[t0].copy()
            a1 = psi[t1].copy()
            psi[t0] = u[0, 0] * a0 + u[0, 1] * a1
            psi[t1] = u[1, 0] * a0 + u[1, 1] * a1
    return psi


# ---------------------------------------------------------------------------------------
# The QFT-then-inverse-QFT circuit of the paper's scaling experiment (Fig. 1c)
# ---------------------------------------------------------------------------------------


def qft_then_iqft(psi: np.ndarray, n: int) -> np.ndarray:
    """QFT on all n qubits followed by the inverse QFT (returns a new array)."""
    out = psi.astype(np.complex128).copy()
    qft(out, n, 0, n, inverse=False)
    qft(out, n, 0, n, inverse=True)
    return out


def qft_register(psi: np.ndarray, n: int, lo: int, m: int, inverse: bool) -> np.ndarray:
    """QFT (or inverse) on bits [lo, lo+m) of a copy of psi."""
    out = psi.astype(np.complex128).copy()
    qft(out, n, lo, m, inverse=inverse)
    return out


# ---------------------------------------------------------------------------------------
# QSP-2 (Sec. III, App. C): sparse state preparation along the paths of a decision diagram
# ---------------------------------------------------------------------------------------


def qsp2_paths(idx: np.ndarray, val: np.ndarray, n: int) -> list[tuple[int, int, float]]:
    """The branch nodes of the binary decision tree of a sparse real vector (nonzero values
    ``val`` at positions ``idx``), root first: one (level l, prefix, theta) per node that lies
    on a path to a nonzero leaf, where the node holds the l most significant bits ``prefix``
    and theta = arccos sqrt(p(zero child) / p(node)) in the paper's R_y convention. Nodes off
    every path (zero subtrees) get no gate; a node with a single nonzero child gets theta 0
    (zero child) or pi/2 (one child)."""
    order = np.argsort(idx)
    idx = np.asarray(idx)[order]
    prob = np.asarray(val, dtype=float)[order] ** 2
    out = []
    for l in range(n):
        shift = n - l
        prefixes = sorted(set(int(i) >> shift for i in idx))
        for pre in prefixes:
            mask = (idx >> shift) == pre
            p_node = float(prob[mask].sum())
            p_zero = float(prob[mask & (((idx >> (shift - 1)) & 1) == 0)].sum())
            theta = math.acos(math.sqrt(min(1.0, p_zero / p_node))) if p_node > 0 else 0.0
            out.append((l, pre, theta))
    return out


def qsp2_prepare(idx: np.ndarray, val: np.ndarray, n: int) -> np.ndarray:
    """Prepare sum_k val_k |idx_k> / |val| from |0>: for every branch node, a rotation
    R_y(theta) (our RY(2 theta)) on qubit n-1-l controlled by the l more significant qubits
    holding ``prefix`` (X gates around the controls that must read 0), then the sign of each
    negative value by a Z on its path (paper silent on signs: a Z on the last qubit
    controlled by the leaf's other n-1 bits)."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for l, pre, theta in qsp2_paths(idx, val, n):
        target = n - 1 - l
        ctrls = list(range(target + 1, n))
        zeros = [q for q in ctrls if ((pre >> (q - target - 1)) & 1) == 0]
        for q in zeros:
            apply_1q(psi, n, q, X_GATE)
        apply_1q(psi, n, target, ry(2.0 * theta), controls=ctrls)
        for q in zeros:
            apply_1q(psi, n, q, X_GATE)
    z = np.array([[1.0, 0.0], [0.0, -1.0]])
    for i, v in zip(idx, val):
        if v < 0:
            ctrls = list(range(1, n))
            zeros = [q for q in ctrls if ((int(i) >> q) & 1) == 0]
            for q in zeros:
                apply_1q(psi, n, q, X_GATE)
            if int(i) & 1:
                apply_1q(psi, n, 0, z, controls=ctrls)
            else:
                apply_1q(psi, n, 0, X_GATE, controls=ctrls)
                apply_1q(psi, n, 0, z, controls=ctrls)
                apply_1q(psi, n, 0, X_GATE, controls=ctrls)
            for q in zeros:
                apply_1q(psi, n, q, X_GATE)
    return psi
