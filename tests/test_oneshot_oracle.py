"""Pins of the one-shot time-stepping systems (App. A, Eqs. FE_OBM / BE_OBM) and of the
two's-complement clock reading used for their indefinite Hermitian dilations: against the
time-marching recurrences, closed forms, the steady limit, library SVD / solves, and an
exact (on-grid) HHL run with negative eigenvalues."""
import math

import numpy as np
import pytest

from oracle import hhl_oracle as o
from oracle import oneshot_oracle as os1


def _setup(n_points=4, seed=3):
    rng = np.random.default_rng(seed)
    a = os1.time_operator(n_points, nu=1.0)
    f = np.full(n_points, 8.0)
    u_in = rng.uniform(0.0, 1.0, n_points)
    return a, f, u_in


@pytest.mark.parametrize("m,p", [(1, 0), (5, 2), (9, 6)])
def test_fe_one_shot_solve_is_the_forward_euler_march(m, p):
    a, f, u_in = _setup()
    dt = 0.25 * (1.0 / 5) ** 2          # Courant number 0.25 at N_g = 4
    big, rhs = os1.fe_system(a, f, u_in, dt, m, p)
    x = np.linalg.solve(big, rhs)
    us = os1.fe_march(a, f, u_in, dt, m, p)
    np.testing.assert_allclose(x, np.concatenate(us), rtol=1e-12, atol=1e-12)
    # closed form of the march: u^m = G^m u_in + sum_{j<m} G^j f dt, G = I + A dt
    g = np.eye(4) + a * dt
    um = np.linalg.matrix_power(g, m) @ u_in + sum(np.linalg.matrix_power(g, j) for j in range(m)) @ f * dt
    np.testing.assert_allclose(os1.final_slice(x, 4, m, p), um, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m,p", [(1, 1), (6, 1), (12, 3)])
def test_be_one_shot_solve_is_the_backward_euler_march(m, p):
    a, f, u_in = _setup(seed=5)
    dt = 0.01
    big, rhs = os1.be_system(a, f, u_in, dt, m, p)
    x = np.linalg.solve(big, rhs)
    np.testing.assert_allclose(x, np.concatenate(os1.be_march(a, f, u_in, dt, m, p)), rtol=1e-12, atol=1e-12)
    # each block row is the implicit step itself
    n = 4
    for i in range(1, m + 1):
        lhs = (np.eye(n) - dt * a) @ x[i * n:(i + 1) * n] - x[(i - 1) * n:i * n]
        np.testing.assert_allclose(lhs, f * dt, atol=1e-12)


def test_be_one_shot_reaches_the_steady_channel_flow():
    """Many implicit steps: the last field solves A u + f = 0, i.e. the steady Poiseuille
    profile of the discrete operator (Thomas solve of the SPD system -A u = f)."""
    n = 8
    a = os1.time_operator(n)
    f = np.full(n, 2.0)
    big, rhs = os1.be_system(a, f, np.zeros(n), 0.05, 400, 0)
    u_last = os1.final_slice(np.linalg.solve(big, rhs), n, 400, 0)
    diag, off = o.laplacian_tridiag(n)
    steady = o.thomas_solve(diag, off, f)
    np.testing.assert_allclose(u_last, steady, rtol=1e-9)
    y = np.arange(1, n + 1) / (n + 1)
    np.testing.assert_allclose(steady, y * (1 - y), rtol=1e-12)  # -u'' = 2: exact on the grid


def test_dilation_spectrum_and_solution():
    a, f, u_in = _setup(seed=7)
    big, rhs = os1.fe_system(a, f, u_in, 0.01, 3, 1)
    h = os1.dilation(big)
    np.testing.assert_array_equal(h, h.T)
    sv = np.linalg.svd(big, compute_uv=False)
    ev = np.sort(np.linalg.eigvalsh(h))
    np.testing.assert_allclose(ev, np.sort(np.concatenate([sv, -sv])), rtol=1e-11, atol=1e-12)
    hp, rp = os1.dilated_problem(big, rhs)
    assert hp.shape[0] == 64 and np.allclose(hp[40:, 40:], np.eye(24))
    xd = np.linalg.solve(hp, rp)
    k = big.shape[0]
    np.testing.assert_allclose(xd[:k], 0.0, atol=1e-12)
    np.testing.assert_allclose(xd[2 * k:], 0.0, atol=1e-12)
    np.testing.assert_allclose(os1.solution_part(xd, k), np.linalg.solve(big, rhs), rtol=1e-11)


def test_signed_rotation_angles():
    n_c, t0 = 4, 2 * math.pi * 7
    th = o.rotation_angles(n_c, t0, signed=True)
    for y in range(16):
        ys = y - 16 if y >= 8 else y
        want = 0.0 if ys == 0 else 2 * math.asin(max(-1.0, min(1.0, 1.0 / (ys * 1.0))))
        assert th[y] == pytest.approx(want, abs=1e-15)
    assert o.t0_total("range_fill_signed", 6) == pytest.approx(2 * math.pi * 31)
    # the unsigned reading is unchanged
    np.testing.assert_allclose(o.rotation_angles(n_c, t0)[1:8], th[1:8])


def test_signed_hhl_is_exact_on_the_clock_grid():
    """An indefinite A whose eigenvalues sit on the two's-complement clock grid: phase
    estimation is exact, so the postselected vector is C Ahat^{-1} bhat to rounding."""
    rng = np.random.default_rng(11)
    lam = np.array([3.0, -5.0, 7.0, -2.0])
    q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    a = q @ np.diag(lam) @ q.T
    lub = o.gershgorin_bound(a)
    n_s, n_c = 2, 5
    pl = o.plan(a, n_c, t0_rule="user", t0=2 * math.pi * lub, signed=True)  # y_j = lambda_j
    b = rng.uniform(0.0, 1.0, 4)
    psi = o.hhl_circuit(b, n_s, pl)
    v = o.postselect(psi, n_s, n_c)["v"]
    bh = b / np.linalg.norm(b)
    want = pl["C"] * np.linalg.solve(a / lub, bh)
    np.testing.assert_allclose(v, want, atol=1e-10)
    # the unsigned reading of the same clock gets the negative eigen-components wrong
    pl_u = o.plan(a, n_c, t0_rule="user", t0=2 * math.pi * lub)
    v_u = o.postselect(o.hhl_circuit(b, n_s, pl_u), n_s, n_c)["v"]
    assert np.abs(v_u - want).max() > 1e-2


@pytest.mark.parametrize("scheme", ["fe", "be"])
def test_library_builder_matches_the_oracle_systems(scheme):
    """The library's host-side construction (Kronecker products) against the oracle's
    block-by-block one (host logic; no GPU)."""
    from paper_2307_00391_gb300 import oneshot as lib1
    a, f, u_in = _setup(seed=9)
    np.testing.assert_allclose(lib1.unsteady_operator(4, 1.0), a, rtol=1e-15)
    dt, m, p = 0.01, 5, 2
    mat, rhs = lib1.one_shot_system(a, f, u_in, dt, m, p, scheme)
    big, brhs = (os1.fe_system if scheme == "fe" else os1.be_system)(a, f, u_in, dt, m, p)
    np.testing.assert_allclose(mat, big, rtol=1e-15, atol=0)
    np.testing.assert_allclose(rhs, brhs, rtol=1e-15, atol=0)
    h, r = lib1.hermitian_dilation(mat, rhs)
    hp, rp = os1.dilated_problem(big, brhs)
    np.testing.assert_array_equal(h, hp)
    np.testing.assert_array_equal(r, rp)
    x = np.linalg.solve(hp, rp)
    np.testing.assert_allclose(lib1.final_field(x, big.shape[0], 4),
                               os1.final_slice(os1.solution_part(x, big.shape[0]), 4, m, p), rtol=1e-14)


def test_qsp2_prepares_the_sparse_vector_and_counts_path_nodes():
    """QSP-2 along decision-tree paths: the prepared state is the amplitude encoding of the
    sparse vector (signs included), only nodes on paths get gates (at most n per nonzero),
    and on a dense vector its angles are the QSP-1 tree's."""
    rng = np.random.default_rng(21)
    n = 7
    idx = np.sort(rng.choice(1 << n, size=9, replace=False))
    val = rng.uniform(0.2, 1.0, 9) * rng.choice([-1.0, 1.0], 9)
    psi = o.qsp2_prepare(idx, val, n)
    want = np.zeros(1 << n)
    want[idx] = val / np.linalg.norm(val)
    np.testing.assert_allclose(psi, want, atol=1e-13)
    nodes = o.qsp2_paths(idx, val, n)
    assert len(nodes) <= 9 * n
    levels = {}
    for l, pre, th in nodes:
        levels.setdefault(l, []).append(pre)
    assert levels[0] == [0] and all(len(v) <= 9 for v in levels.values())
    # a dense vector: every node is on a path and the angles are QSP-1's
    b = rng.uniform(0.1, 1.0, 16)
    ang1 = o.qsp1_angles(b * b)
    for l, pre, th in o.qsp2_paths(np.arange(16), b, 4):
        assert th == pytest.approx(ang1[l][pre], abs=1e-14)
    np.testing.assert_allclose(o.qsp2_prepare(np.arange(16), b, 4), b / np.linalg.norm(b), atol=1e-14)


def test_qsp2_on_the_one_shot_right_hand_side():
    """The dilated one-shot right-hand side [b_fe; 0] is sparse: u_in and m copies of f dt in
    a 2^7 register; QSP-2 prepares it with at most n gates per nonzero."""
    a, f, u_in = _setup(n_points=8, seed=4)
    big, rhs = os1.fe_system(a, f, u_in, 0.003, 3, 4)
    hp, rp = os1.dilated_problem(big, rhs)
    nz = np.nonzero(rp)[0]
    n = int(math.log2(len(rp)))
    psi = o.qsp2_prepare(nz, rp[nz], n)
    np.testing.assert_allclose(psi, rp / np.linalg.norm(rp), atol=1e-13)
    assert len(nz) == 8 * 4 and len(o.qsp2_paths(nz, rp[nz], n)) <= len(nz) * n


def test_iterative_be_with_exact_solves_is_the_march_and_converges():
    """The hybrid loop with exact linear solves reproduces the backward-Euler march and stops
    at the steady channel flow once the residue reaches 1e-6."""
    n = 16
    a = os1.time_operator(n)
    f = np.full(n, 2.0)
    u0 = np.zeros(n)
    us, res = os1.iterative_be(a, f, u0, 0.01, 5000, 1e-6, np.linalg.solve)
    march = os1.be_march(a, f, u0, 0.01, len(us) - 1, 0)
    np.testing.assert_allclose(np.array(us), np.array(march), rtol=1e-12, atol=1e-14)
    assert res[-1] <= 1e-6 < res[-2]
    assert all(r2 < r1 for r1, r2 in zip(res, res[1:]))            # monotone approach
    y = np.arange(1, n + 1) / (n + 1)
    np.testing.assert_allclose(us[-1], y * (1 - y), atol=2e-4)     # steady parabola
    # the HHL read-out as the linear solve (oracle circuit, 10 clock qubits) tracks it
    def hhl_solve(a1, b):
        pl = o.plan(a1, 10)
        psi = o.hhl_circuit(b, 4, pl)
        v = o.postselect(psi, 4, 10)["v"]
        return o.velocity(v, np.linalg.norm(b), pl["C"], pl["lam_ub"])
    uq, rq = os1.iterative_be(a, f, u0, 0.01, 3, 0.0, hhl_solve)
    np.testing.assert_allclose(np.array(uq), np.array(march[:4]), atol=0.05 * np.abs(march[3]).max())
