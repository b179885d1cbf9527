"""Plain FP64 oracle of the one-shot time-stepping flow systems (App. A, finite differences).

TEST INFRASTRUCTURE ONLY: only ``tests/`` may import it; it shares no code with the
library or with the library's own builder of these systems.

The unsteady channel flow du/dt = A u + f (App. A: A the central-difference Laplacian
operator, f the constant forcing) is marched over m time steps of size dt and then held for
p more steps (copies of the last field, which raise the postselection probability). The
one-shot schemes stack all T = m + p + 1 fields u^0 .. u^{m+p} into one vector and one
block lower-bidiagonal system of size T N_g:

* forward Euler (App. A, Eq. FE_OBM): block row 0 is u^0 = u_in; block row i <= m is
  u^i - (I + A dt) u^{i-1} = f dt; block row i > m is u^i - u^{i-1} = 0;
* backward Euler (App. A, Eq. BE_OBM): block row i <= m is (I - A dt) u^i - u^{i-1} = f dt,
  the other rows as above.

Reading (the prose of App. A writes the BE diagonal blocks as -(I + A dt) and the
right-hand side as -f dt, which contradicts both the displayed block matrix and the
backward-Euler recurrence it stands for): the displayed matrix and the recurrence
(I - A dt) u^{j+1} = u^j + f dt are taken.

The block matrix is not Hermitian; HHL takes its Hermitian dilation
H = [[0, M], [M^T, 0]] with right-hand side [b; 0], whose solution is [0; M^{-1} b]
(paper silent on the embedding; the dilation is the standard one), padded to a power of two
with an identity block (eigenvalue 1, zero right-hand side there).
"""
from __future__ import annotations

import numpy as np


def time_operator(n_points: int, nu: float = 1.0) -> np.ndarray:
    """nu * tridiag(1, -2, 1) / h^2, h = 1/(N_g + 1): the Laplacian of App. A Eq. (CDS) with the
    sign of du/dt = A u + f (negative definite)."""
    h = 1.0 / (n_points + 1)
    a = np.zeros((n_points, n_points))
    for i in range(n_points):
        a[i, i] = -2.0
        if i > 0:
            a[i, i - 1] = 1.0
        if i + 1 < n_points:
            a[i, i + 1] = 1.0
    return nu * a / (h * h)


def fe_system(a: np.ndarray, f: np.ndarray, u_in: np.ndarray, dt: float, m: int, p: int):
    """Forward-Euler one-shot block system (matrix, right-hand side), block by block."""
    n = a.shape[0]
    t = m + p + 1
    big = np.zeros((t * n, t * n))
    rhs = np.zeros(t * n)
    eye = np.eye(n)
    for i in range(t):
        big[i * n:(i + 1) * n, i * n:(i + 1) * n] = eye
        if i > 0:
            big[i * n:(i + 1) * n, (i - 1) * n:i * n] = -(eye + a * dt) if i <= m else -eye
    rhs[:n] = u_in
    for i in range(1, m + 1):
        rhs[i * n:(i + 1) * n] = f * dt
    return big, rhs


def be_system(a: np.ndarray, f: np.ndarray, u_in: np.ndarray, dt: float, m: int, p: int):
    """Backward-Euler one-shot block system (matrix, right-hand side), block by block."""
    n = a.shape[0]
    t = m + p + 1
    big = np.zeros((t * n, t * n))
    rhs = np.zeros(t * n)
    eye = np.eye(n)
    for i in range(t):
        big[i * n:(i + 1) * n, i * n:(i + 1) * n] = (eye - a * dt) if 1 <= i <= m else eye
        if i > 0:
            big[i * n:(i + 1) * n, (i - 1) * n:i * n] = -eye
    rhs[:n] = u_in
    for i in range(1, m + 1):
        rhs[i * n:(i + 1) * n] = f * dt
    return big, rhs


def fe_march(a, f, u_in, dt, m, p) -> list[np.ndarray]:
    """The forward-Euler fields u^0 .. u^{m+p} step by step (then held)."""
    us = [np.array(u_in, dtype=float)]
    for _ in range(m):
        us.append(us[-1] + dt * (a @ us[-1] + f))
    us += [us[-1].copy() for _ in range(p)]
    return us


def be_march(a, f, u_in, dt, m, p) -> list[np.ndarray]:
    """The backward-Euler fields u^0 .. u^{m+p} step by step (one library solve per step)."""
    n = a.shape[0]
    us = [np.array(u_in, dtype=float)]
    for _ in range(m):
        us.append(np.linalg.solve(np.eye(n) - dt * a, us[-1] + dt * f))
    us += [us[-1].copy() for _ in range(p)]
    return us


def dilation(big: np.ndarray) -> np.ndarray:
    """[[0, M], [M^T, 0]]: Hermitian, eigenvalues +- the singular values of M."""
    k = big.shape[0]
    h = np.zeros((2 * k, 2 * k))
    h[:k, k:] = big
    h[k:, :k] = big.T
    return h


def padded(h: np.ndarray, rhs: np.ndarray):
    """Embed H (and its right-hand side) in the next power of two, identity on the padding."""
    k = h.shape[0]
    size = 1
    while size < k:
        size *= 2
    hp = np.eye(size)
    hp[:k, :k] = h
    r = np.zeros(size)
    r[:k] = rhs
    return hp, r


def dilated_problem(big: np.ndarray, rhs: np.ndarray):
    """The padded dilation and its right-hand side [b; 0; 0...]."""
    k = big.shape[0]
    r = np.zeros(2 * k)
    r[:k] = rhs
    return padded(dilation(big), r)


def solution_part(x_dilated: np.ndarray, k: int) -> np.ndarray:
    """M^{-1} b from the dilated solution [0; M^{-1} b; padding]."""
    return x_dilated[k:2 * k]


def final_slice(x: np.ndarray, n_points: int, m: int, p: int) -> np.ndarray:
    """u^{m+p}: the last field of the stacked one-shot solution."""
    return x[(m + p) * n_points:(m + p + 1) * n_points]


# ---------------------------------------------------------------------------------------
# Iterative backward Euler (Sec. II: A_be1 u^{j+1} = b_be1 solved once per time step)
# ---------------------------------------------------------------------------------------


def be1_operator(a: np.ndarray, dt: float) -> np.ndarray:
    """A_be1 = -(A dt - I) = I - A dt (symmetric positive definite for the Laplacian A)."""
    return np.eye(a.shape[0]) - dt * a


def iterative_be(a, f, u0, dt: float, max_steps: int, tol: float, solve) -> tuple[list, list]:
    """u^{j+1} = solve(A_be1, u^j + f dt) until max_i |u^{j+1} - u^j| <= tol (the classical
    residue check of the hybrid loop) or max_steps; returns (fields, residues)."""
    a1 = be1_operator(a, dt)
    us, res = [np.array(u0, dtype=float)], []
    for _ in range(max_steps):
        u_next = solve(a1, us[-1] + dt * np.asarray(f, dtype=float))
        res.append(float(np.max(np.abs(u_next - us[-1]))))
        us.append(u_next)
        if res[-1] <= tol:
            break
    return us, res
