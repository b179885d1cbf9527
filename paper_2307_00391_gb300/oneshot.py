"""One-shot time-stepping flow systems on the HHL path (App. A, Eqs. FE_OBM / BE_OBM).

The unsteady channel flow du/dt = A u + f (A the central-difference Laplacian of App. A
Eq. CDS, f the constant forcing) marched over m steps of size dt and held p more steps is
one linear system for all fields u^0 .. u^{m+p} at once: block lower-bidiagonal, identity (or
I - A dt for the implicit scheme) on the diagonal, -(I + A dt) (explicit) or -I below. It is
not Hermitian, so the HHL plan takes its Hermitian dilation [[0, M], [M^T, 0]] with the right-
hand side [b; 0], read with a signed (two's-complement) clock because the dilation has the
eigenvalues +- the singular values of M; the solution sits in the second block, and its last
N_g entries are the final field u^{m+p}.

Host-side construction only (numpy, Kronecker products); every step of the circuit runs in
the library's kernels through ``HHLPlan``.
"""
from __future__ import annotations

import numpy as np


def unsteady_operator(n_points: int, nu: float = 1.0) -> np.ndarray:
    """nu (u_{i+1} - 2 u_i + u_{i-1}) / h^2 with h = 1/(N_g + 1), homogeneous walls."""
    h = 1.0 / (n_points + 1)
    lap = -2.0 * np.eye(n_points) + np.eye(n_points, k=1) + np.eye(n_points, k=-1)
    return nu * lap / (h * h)


def one_shot_system(a: np.ndarray, f: np.ndarray, u_in: np.ndarray, dt: float, m: int, p: int,
                    scheme: str = "fe") -> tuple[np.ndarray, np.ndarray]:
    """(M, b) of the one-shot forward-Euler ("fe") or backward-Euler ("be") scheme."""
    n = a.shape[0]
    t = m + p + 1
    eye_n, eye_t = np.eye(n), np.eye(t)
    marched = np.zeros(t)
    marched[1:m + 1] = 1.0                       # block rows that take a time step
    below = np.eye(t, k=-1)                       # block (i, i-1)
    if scheme == "fe":
        mat = np.kron(eye_t, eye_n) - np.kron(below * marched[:, None], eye_n + dt * a) \
            - np.kron(below * (1.0 - marched)[:, None], eye_n)
    elif scheme == "be":
        mat = np.kron(np.diag(1.0 - marched), eye_n) + np.kron(np.diag(marched), eye_n - dt * a) \
            - np.kron(below, eye_n)
    else:
        raise ValueError(scheme)
    first = np.zeros(t)
    first[0] = 1.0
    rhs = np.kron(first, np.asarray(u_in, dtype=float)) + np.kron(marched, dt * np.asarray(f, dtype=float))
    return mat, rhs


def hermitian_dilation(mat: np.ndarray, rhs: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """[[0, M], [M^T, 0]] and [b; 0], zero-padded to a power-of-two size with an identity
    block on the padding (eigenvalue 1, no right-hand side there)."""
    k = mat.shape[0]
    size = 1 << int(np.ceil(np.log2(2 * k)))
    h = np.eye(size)
    h[:2 * k, :2 * k] = np.block([[np.zeros((k, k)), mat], [mat.T, np.zeros((k, k))]])
    r = np.zeros(size)
    r[:k] = rhs
    return h, r


def final_field(x_dilated: np.ndarray, k: int, n_points: int) -> np.ndarray:
    """u^{m+p} from the dilated solution [0; u^0 .. u^{m+p}; padding] (k = (m+p+1) N_g)."""
    return np.asarray(x_dilated)[2 * k - n_points:2 * k]


def solve_one_shot(a, f, u_in, dt: float, m: int, p: int, n_clock: int, scheme: str = "fe",
                   precision: str = "c64", gemm: str = "auto", t0_rule: str = "range_fill",
                   t0: float = 0.0, prep: str = "amplitude") -> dict:
    """Plan the dilated system with a signed clock, run the whole circuit on the GPU and read
    the result: ``fields`` (all u^j estimated, (m+p+1) x N_g), ``final`` (u^{m+p}),
    ``p_success``, the plan ``info`` and the dilated problem (``h``, ``r``). ``prep``:
    "amplitude" (hhl_prepare_rhs) or "qsp2" (the sparse gate-level preparation of the
    right-hand side, whose nonzeros are u_in and the m forcing blocks)."""
    from . import HHLPlan

    mat, rhs = one_shot_system(a, f, u_in, dt, m, p, scheme)
    h, r = hermitian_dilation(mat, rhs)
    n_s = int(np.log2(h.shape[0]))
    plan = HHLPlan(n_s, n_clock, dense=h, precision=precision, gemm=gemm, t0_rule=t0_rule, t0=t0,
                   signed_clock=True)
    st = plan.new_state()
    if prep == "qsp2":
        import torch
        nz = np.nonzero(r)[0]
        plan.prepare_rhs_qsp2(torch.tensor(nz, dtype=torch.int64, device="cuda"),
                              torch.tensor(r[nz], dtype=torch.float64, device="cuda"), st)
    elif prep == "amplitude":
        plan.prepare_rhs_host(r, st)
    else:
        raise ValueError(prep)
    plan.apply_circuit(st)
    meas = plan.measure(st)
    info = plan.info
    # postselected v ~ C Hhat^{-1} rhat, so x = |r| v / (C lambda_ub)
    v = meas["xhat"] * np.sqrt(meas["p_success"])
    x = np.linalg.norm(r) * v.real / (info["C"] * info["lambda_ub"])
    k = mat.shape[0]
    n = a.shape[0]
    return dict(fields=x[k:2 * k].reshape(m + p + 1, n), final=final_field(x, k, n), p_success=meas["p_success"],
                info=info, h=h, r=r, state=st, plan=plan)
