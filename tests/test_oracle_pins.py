"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values printed in the
paper (tests/golden/), closed forms, invariants, special cases that reduce to a textbook
result, and brute force on tiny inputs (dense Kronecker-product circuit matrices).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import hhl_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kron_1q(n, q, u):
    """Full 2^n matrix of a one-qubit gate on qubit q (qubit n-1 leftmost in kron order)."""
    return np.kron(np.kron(np.eye(1 << (n - 1 - q)), u), np.eye(1 << q))


def _proj(n, q, bit):
    p = np.array([[1.0, 0.0], [0.0, 0.0]]) if bit == 0 else np.array([[0.0, 0.0], [0.0, 1.0]])
    return _kron_1q(n, q, p)


# ----------------------------------------------------------------------------- golden


def test_gate_example_h1_x0_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "gate_example_h1_x0.json")))
    expect = np.array(g["matrix_times_sqrt2"], dtype=float) / math.sqrt(2.0)
    cols = []
    for x in range(4):
        psi = np.zeros(4, dtype=complex)
        psi[x] = 1.0
        o.apply_1q(psi, 2, 0, o.X_GATE)
        o.apply_1q(psi, 2, 1, o.H_GATE)
        cols.append(psi)
    got = np.array(cols).T
    np.testing.assert_allclose(got, expect, atol=1e-15)
    u = np.array([0.3, -1.1, 0.7, 2.0], dtype=complex)
    out = u.copy()
    o.apply_1q(out, 2, 0, o.X_GATE)
    o.apply_1q(out, 2, 1, o.H_GATE)
    m = np.array([u[1] + u[3], u[0] + u[2], u[1] - u[3], u[0] - u[2]]) / math.sqrt(2.0)
    np.testing.assert_allclose(out, m, atol=1e-15)


def test_qsp1_worked_example_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "qsp1_worked_example.json")))
    p = np.array(g["leaf_probabilities"])
    ang = o.qsp1_angles(p)
    # root rotation alone: sqrt(0.75)|0> + sqrt(0.25)|1> on the most significant qubit
    root = o.ry(2.0 * ang[0][0]) @ np.array([1.0, 0.0])
    np.testing.assert_allclose(root ** 2, [g["after_first_rotation"]["msb0"],
                                           g["after_first_rotation"]["msb1"]], atol=1e-15)
    psi = o.qsp1_prepare(np.sqrt(p))
    np.testing.assert_allclose(np.abs(psi) ** 2, g["final_amplitudes_squared"], atol=1e-15)
    np.testing.assert_allclose(psi.imag, 0.0, atol=1e-15)


def test_qsp1_constant_vector_is_hadamard_layer():
    n = 5
    psi = o.qsp1_prepare(np.full(1 << n, 1.0 / math.sqrt(1 << n)))
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = 1.0
    for q in range(n):
        o.apply_1q(ref, n, q, o.H_GATE)
    np.testing.assert_allclose(psi, ref, atol=1e-14)


def test_qsp1_random_log_concave_profile():
    y = (np.arange(1, 17)) / 17.0
    a = np.sqrt(y * (1 - y))
    a /= np.linalg.norm(a)
    np.testing.assert_allclose(o.qsp1_prepare(a).real, a, atol=1e-14)


# ----------------------------------------------------------------------------- QFT


@pytest.mark.parametrize("n,lo,m", [(3, 0, 3), (5, 1, 3), (6, 2, 4), (7, 0, 6), (8, 3, 5)])
def test_qft_closed_form_on_basis_states(n, lo, m):
    dim = 1 << m
    for rest in (0, (1 << n) - 1 - (((1 << m) - 1) << lo)):
        for x in range(dim):
            psi = np.zeros(1 << n, dtype=complex)
            psi[rest | (x << lo)] = 1.0
            o.qft(psi, n, lo, m)
            exp = np.zeros(1 << n, dtype=complex)
            for y in range(dim):
                exp[rest | (y << lo)] = np.exp(2j * np.pi * x * y / dim) / math.sqrt(dim)
            np.testing.assert_allclose(psi, exp, atol=1e-13)


def test_inverse_qft_is_inverse_dft_and_roundtrip():
    n, lo, m = 9, 2, 5
    psi = np.random.default_rng(5).standard_normal(1 << n) + 0j
    out = o.qft_register(psi, n, lo, m, inverse=True)
    t = psi.reshape((1 << (n - lo - m), 1 << m, 1 << lo))
    ref = np.fft.fft(t, axis=1) / math.sqrt(1 << m)     # sum_x e^{-2 pi i x y / 2^m}
    np.testing.assert_allclose(out.reshape(t.shape), ref, atol=1e-13)
    back = o.qft_register(out, n, lo, m, inverse=False)
    np.testing.assert_allclose(back, psi, atol=1e-13)


def test_qft_then_iqft_identity_random_states():
    for seed in range(3):
        psi = np.random.default_rng(seed).standard_normal(1 << 10) * (1 + 0.5j)
        np.testing.assert_allclose(o.qft_then_iqft(psi, 10), psi, atol=1e-12)


# ----------------------------------------------------------------------------- gates


def test_gate_primitives_against_kronecker_products():
    n = 5
    rng = np.random.default_rng(11)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    u = np.linalg.qr(rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)))[0]
    for q in range(n):
        got = psi.copy()
        o.apply_1q(got, n, q, u)
        np.testing.assert_allclose(got, _kron_1q(n, q, u) @ psi, atol=1e-14)
    # controlled on qubits 0 and 3, target 2
    got = psi.copy()
    o.apply_1q(got, n, 2, u, controls=(0, 3))
    full = np.eye(1 << n) - _proj(n, 0, 1) @ _proj(n, 3, 1) + \
        _proj(n, 0, 1) @ _proj(n, 3, 1) @ _kron_1q(n, 2, u)
    np.testing.assert_allclose(got, full @ psi, atol=1e-14)
    # controlled phase and swap
    got = psi.copy()
    o.apply_cphase(got, n, 1, 4, 0.7)
    d = np.array([np.exp(0.7j) if ((i >> 1) & 1 and (i >> 4) & 1) else 1.0 for i in range(1 << n)])
    np.testing.assert_allclose(got, d * psi, atol=1e-14)
    got = psi.copy()
    o.apply_swap(got, n, 1, 3)
    perm = [i ^ (((i >> 1) & 1) ^ ((i >> 3) & 1)) * 0b1010 for i in range(1 << n)]
    np.testing.assert_allclose(got, psi[perm], atol=1e-14)
    # register unitary on bits [1, 4) controlled by qubit 4
    v = np.linalg.qr(rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)))[0]
    got = psi.copy()
    o.apply_register_unitary(got, n, 1, 3, v, control=4)
    full = _proj(n, 4, 0) + _proj(n, 4, 1) @ np.kron(np.kron(np.eye(2), v), np.eye(2))
    np.testing.assert_allclose(got, full @ psi, atol=1e-13)


def _brute_force_hhl(b, n_s, pl):
    """Whole HHL circuit as a product of dense 2^n x 2^n matrices, built from Kronecker
    products and the DFT matrix, then applied to |0>|0>|bhat>."""
    n_c = pl["n_clock"]
    n = n_s + n_c + 1
    dim_c = 1 << n_c
    f = np.array([[np.exp(2j * np.pi * x * y / dim_c) for x in range(dim_c)]
                  for y in range(dim_c)]) / math.sqrt(dim_c)
    qft_full = np.kron(np.kron(np.eye(2), f), np.eye(1 << n_s))
    hh = np.eye(1 << n)
    for q in range(n_s, n_s + n_c):
        hh = _kron_1q(n, q, o.H_GATE) @ hh
    mats = []
    for k in range(n_c):
        t = pl["t0"] * (1 << k) / dim_c
        u = o.evolution_dense(pl["a_hat"], t)
        sys_u = np.kron(np.eye(1 << (n_c + 1)), u)
        mats.append(_proj(n, n_s + k, 0) + _proj(n, n_s + k, 1) @ sys_u)
    rot = np.zeros((1 << n, 1 << n), dtype=complex)
    for y in range(dim_c):
        py = np.zeros((dim_c, dim_c))
        py[y, y] = 1.0
        rot += np.kron(np.kron(o.ry(pl["theta"][y]), py), np.eye(1 << n_s))
    circuit = hh
    for m in mats:
        circuit = m @ circuit
    circuit = rot @ qft_full.conj().T @ circuit
    circuit = qft_full @ circuit
    for m in reversed(mats):
        circuit = m.conj().T @ circuit
    circuit = hh @ circuit
    psi0 = np.zeros(1 << n, dtype=complex)
    psi0[: 1 << n_s] = b / np.linalg.norm(b)
    return circuit @ psi0


@pytest.mark.parametrize("n_s,n_c,rule", [(2, 3, "range_fill"), (3, 4, "power_law"), (2, 5, "range_fill")])
def test_hhl_circuit_against_brute_force_matrices(n_s, n_c, rule):
    diag, off = o.laplacian_tridiag(1 << n_s)
    a = o.dense_from_tridiag(diag, off)
    pl = o.plan(a, n_c, t0_rule=rule)
    b = np.random.default_rng(n_s * 10 + n_c).random(1 << n_s)
    got = o.hhl_circuit(b, n_s, pl)
    ref = _brute_force_hhl(b, n_s, pl)
    np.testing.assert_allclose(got, ref, atol=1e-12)


# ----------------------------------------------------------------------------- HHL closed forms


def _laplacian_eigen(n):
    """Analytic eigenpairs of tridiag(-1,2,-1)/h^2 (discrete sine transform, DST-I)."""
    h = 1.0 / (n + 1)
    k = np.arange(1, n + 1)
    lam = (4.0 / h ** 2) * np.sin(k * np.pi / (2 * (n + 1))) ** 2
    i = np.arange(1, n + 1)
    v = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, k) * np.pi / (n + 1))
    return lam, v


def _fejer(d, m):
    s = np.sin(np.pi * d)
    out = np.where(np.abs(s) < 1e-300, 1.0, 0.0)
    nz = np.abs(s) >= 1e-300
    out[nz] = np.sin(np.pi * (1 << m) * d[nz]) ** 2 / ((1 << (2 * m)) * s[nz] ** 2)
    return out


@pytest.mark.parametrize("flow,n_s,n_c,rule", [("poiseuille", 4, 6, "power_law"),
                                                ("poiseuille", 4, 6, "range_fill"),
                                                ("couette", 5, 7, "range_fill")])
def test_hhl_matches_eigendecomposition_closed_form(flow, n_s, n_c, rule):
    """v = sum_j beta_j u_j sum_y K(phi_j - y/2^n_c) sin(theta_y/2), K the Fejer kernel,
    phi_j = lambdahat_j T0 / (2 pi 2^n_c), with the analytic sine eigenbasis."""
    from synth_inputs import rhs
    n = 1 << n_s
    diag, off = o.laplacian_tridiag(n)
    a = o.dense_from_tridiag(diag, off)
    pl = o.plan(a, n_c, t0_rule=rule)
    b = rhs(flow, n)
    res = o.postselect(o.hhl_circuit(b, n_s, pl), n_s, n_c)
    lam, v = _laplacian_eigen(n)
    h = 1.0 / (n + 1)
    lam_hat = lam / (4.0 / h ** 2)
    beta = v.T @ (b / np.linalg.norm(b))
    phi = lam_hat * pl["t0"] / (2 * np.pi * (1 << n_c))
    ys = np.arange(1 << n_c)
    w = np.array([np.sum(_fejer(p - ys / (1 << n_c), n_c) * np.sin(pl["theta"] / 2)) for p in phi])
    closed = v @ (beta * w)
    np.testing.assert_allclose(res["v"], closed, atol=1e-13)


def test_on_grid_spectrum_gives_exact_inverse():
    """If every lambdahat_j T0/(2 pi) is an integer >= 1 the postselected vector is exactly
    C Ahat^{-1} bhat (= A^{-1} bhat with T0 = 2 pi lambda_ub)."""
    n_s, n_c = 3, 5
    rng = np.random.default_rng(3)
    q = np.linalg.qr(rng.standard_normal((8, 8)))[0]
    lam = np.array([1.0, 2.0, 3.0, 5.0, 8.0, 13.0, 21.0, 30.0])
    a = q @ np.diag(lam) @ q.T
    a = 0.5 * (a + a.T)
    lam_ub = o.gershgorin_bound(a)
    pl = o.plan(a, n_c, t0_rule="user", t0=2 * np.pi * lam_ub)
    b = rng.random(8)
    res = o.postselect(o.hhl_circuit(b, n_s, pl), n_s, n_c)
    exact = np.linalg.solve(a, b / np.linalg.norm(b))
    np.testing.assert_allclose(res["v"], exact, atol=1e-12)
    assert o.fidelity(res["v"], exact) == pytest.approx(1.0, abs=1e-13)


def test_norm_and_probability_invariants():
    n_s, n_c = 4, 6
    diag, off = o.laplacian_tridiag(16)
    pl = o.plan(o.dense_from_tridiag(diag, off), n_c)
    psi = o.hhl_circuit(np.ones(16), n_s, pl)
    res = o.postselect(psi, n_s, n_c)
    assert res["norm"] == pytest.approx(1.0, abs=1e-13)
    s = psi.reshape(2, 1 << n_c, 16)
    assert float(np.vdot(s[0], s[0]).real) + res["p_anc1"] == pytest.approx(1.0, abs=1e-13)
    assert 0.0 < res["p_success"] <= res["p_anc1"]


def test_prepare_state_is_clock_uniform():
    b = np.random.default_rng(1).random(8)
    psi = o.prepare_state(b, 3, 4).reshape(2, 16, 8)
    for c in range(16):
        np.testing.assert_allclose(psi[0, c], b / np.linalg.norm(b) / 4.0, atol=1e-15)
    assert np.all(psi[1] == 0)


# ----------------------------------------------------------------------------- classical targets


@pytest.mark.parametrize("n", [16, 1024])
def test_thomas_poiseuille_and_couette_profiles(n):
    from synth_inputs import rhs
    diag, off = o.laplacian_tridiag(n)
    y = np.arange(1, n + 1) / (n + 1)
    # steady limit of Sec. IV Eq. (analytical) with Re * (-dp/dx) = 1: u = y(1-y)/2
    np.testing.assert_allclose(o.thomas_solve(diag, off, rhs("poiseuille", n)), y * (1 - y) / 2,
                               atol=1e-12)
    np.testing.assert_allclose(o.thomas_solve(diag, off, rhs("couette", n)), y, atol=1e-10)


def test_analytical_series_steady_limit():
    """Sec. IV Eq. (analytical): as t -> infinity the series decays and
    u -> -(Re/2)(dp/dx) y(1-y); at t = 0 it reproduces u_in = 1 in the interior."""
    re, dpdx = 10.0, -2.0
    y = np.linspace(0.05, 0.95, 19)

    def u(t, kmax=4001):
        s = np.zeros_like(y)
        for k in range(1, kmax):
            s += (2 * (1 - (-1) ** k) / (k * np.pi)) * (1 + dpdx * re / (k * np.pi) ** 2) * \
                np.sin(k * np.pi * y) * np.exp(-t / re * (k * np.pi) ** 2)
        return s - re / 2 * dpdx * y * (1 - y)

    np.testing.assert_allclose(u(200.0), -re / 2 * dpdx * y * (1 - y), atol=1e-12)
    np.testing.assert_allclose(u(0.0), 1.0, atol=2e-3)
    diag, off = o.laplacian_tridiag(19)
    yy = np.arange(1, 20) / 20.0
    steady = o.thomas_solve(diag, off, np.full(19, re * -dpdx))
    np.testing.assert_allclose(steady, -re / 2 * dpdx * yy * (1 - yy), atol=1e-10)


def test_laplacian_spectrum_and_condition_numbers():
    for n, kappa in ((16, 116.46), (1024, 4.258e5)):
        diag, off = o.laplacian_tridiag(n)
        a = o.dense_from_tridiag(diag, off)
        lam, _ = _laplacian_eigen(n)
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(a)), np.sort(lam), rtol=1e-10)
        assert o.condition_number(a) == pytest.approx(kappa, rel=1e-3)
        assert o.gershgorin_bound(a) == pytest.approx(4.0 * (n + 1) ** 2, rel=1e-14)
        lo1, hi1, lo2, hi2 = o.wolkowicz_bounds(a)
        assert lo1 <= lam.min() <= hi1 and lo2 <= lam.max() <= hi2


# ----------------------------------------------------------------------------- dissipation


@pytest.mark.parametrize("n", [8, 16, 1024])
def test_dissipation_closed_forms(n):
    h = 1.0 / (n + 1)
    y = np.arange(1, n + 1) * h
    nu = 0.37
    # u = y(1-y): h sum (du/h)^2 = 1/3 - h^2/3
    assert o.dissipation(y * (1 - y), 0.0, 0.0, nu) == pytest.approx(nu * (1 / 3 - h * h / 3), rel=1e-12)
    # Couette u = y: eps = nu exactly
    assert o.dissipation(y, 0.0, 1.0, nu) == pytest.approx(nu, rel=1e-12)


def test_velocity_denormalisation_on_grid():
    """With an on-grid spectrum v = C Ahat^{-1} bhat, so |b| v / (C lambda_ub) = A^{-1} b."""
    rng = np.random.default_rng(9)
    q = np.linalg.qr(rng.standard_normal((4, 4)))[0]
    a = q @ np.diag([2.0, 3.0, 6.0, 7.0]) @ q.T
    a = 0.5 * (a + a.T)
    pl = o.plan(a, 4, t0_rule="user", t0=2 * np.pi * o.gershgorin_bound(a))
    b = rng.random(4) * 3.0
    res = o.postselect(o.hhl_circuit(b, 2, pl), 2, 4)
    u = o.velocity(res["v"], np.linalg.norm(b), pl["C"], pl["lam_ub"])
    np.testing.assert_allclose(u, np.linalg.solve(a, b), atol=1e-12)


# ----------------------------------------------------------------------------- planning


def test_rotation_angles_and_t0_rules():
    th = o.rotation_angles(4, 2 * np.pi * 15)
    assert th[0] == 0.0
    np.testing.assert_allclose(np.sin(th[1:] / 2), 1.0 / np.arange(1, 16), atol=1e-15)
    assert o.t0_total("range_fill", 6) == pytest.approx(2 * np.pi * 63)
    assert o.t0_total("user", 5, t0=1.5, convention="per_unit") == pytest.approx(48.0)
    # power-law fallback (parity unpinned): only its monotone decrease with kappa is checked
    assert o.t0_total("power_law", 6, kappa=10.0) > o.t0_total("power_law", 6, kappa=100.0)


# ----------------------------------------------------------------------------- Trotter


def test_trotter_converges_second_order_and_is_unitary():
    n = 16
    diag, off = o.laplacian_tridiag(n)
    lam_ub = 4.0 * (n + 1) ** 2
    dh, oh = diag / lam_ub, off / lam_ub
    t = 3.0
    exact = o.evolution_dense(o.dense_from_tridiag(dh, oh), t)
    errs = []
    for r in (8, 16, 32):
        u = o.trotter_unitary(dh, oh, t, r)
        np.testing.assert_allclose(u @ u.conj().T, np.eye(n), atol=1e-13)
        errs.append(np.linalg.norm(u - exact, 2))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4
    # S(tau) is symmetric: S(-tau) S(tau) = I
    np.testing.assert_allclose(o.trotter_unitary(dh, oh, -t, 4) @ o.trotter_unitary(dh, oh, t, 4),
                               np.eye(n), atol=1e-13)


def test_trotter_two_points_is_exact():
    dh = np.array([0.5, 0.5])
    oh = np.array([-0.25])
    np.testing.assert_allclose(o.trotter_unitary(dh, oh, 2.0, 1),
                               o.evolution_dense(o.dense_from_tridiag(dh, oh), 2.0), atol=1e-14)


def test_trotter_gate_sequence_matches_dense_product():
    n_s, n = 3, 6
    rng = np.random.default_rng(4)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    dh = rng.random(8)
    oh = rng.random(7) - 0.5
    got = psi.copy()
    o.apply_trotter_controlled(got, n, n_s, 4, dh, oh, 1.3, 3)
    u = o.trotter_unitary(dh, oh, 1.3, 3)
    ref = psi.copy()
    o.apply_register_unitary(ref, n, 0, n_s, u, control=4)
    np.testing.assert_allclose(got, ref, atol=1e-13)
    assert o.trotter_steps(10.0, 3.0, 0) == 4
    assert o.trotter_steps(10.0, 3.0, 2) == 2


def test_stage_cuts_reproduce_whole_circuit():
    from tests.oracle_stages import run_stages
    diag, off = o.laplacian_tridiag(16)
    pl = o.plan(o.dense_from_tridiag(diag, off), 5, t0_rule="power_law")
    b = np.random.default_rng(2).random(16)
    st = run_stages(b, 4, pl)
    np.testing.assert_allclose(st["final_h"], o.hhl_circuit(b, 4, pl), atol=1e-13)
    tro = dict(diag=diag / o.gershgorin_bound(o.dense_from_tridiag(diag, off)),
               off=off / o.gershgorin_bound(o.dense_from_tridiag(diag, off)), dt=2.0, r_max=5)
    st2 = run_stages(b, 4, pl, trotter=tro)
    np.testing.assert_allclose(st2["final_h"], o.hhl_circuit(b, 4, pl, trotter=tro), atol=1e-13)


# ----------------------------------------------------------------------------- T0 network


def test_mlp_oracle_gradient_matches_central_differences():
    from oracle import mlp_oracle as m
    rng = np.random.default_rng(12)
    p = rng.standard_normal(m.N_PARAMS) * 0.2
    x = rng.standard_normal((5, 6))
    t = rng.standard_normal((5, 2))
    loss, g = m.loss_and_grad(p, x, t)
    idx = rng.choice(m.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 767, 768, 895, 896, 17279, 17280, 17407, 17408, 17663, 17664, 17665]])
    for i in idx:
        e = np.zeros(m.N_PARAMS)
        e[i] = 1e-6
        fd = (m.loss_and_grad(p + e, x, t)[0] - m.loss_and_grad(p - e, x, t)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), i


def test_mlp_oracle_special_cases():
    from oracle import mlp_oracle as m
    assert m.N_PARAMS == 17666
    p = np.zeros(m.N_PARAMS)
    p[-2:] = [0.5, -1.5]                      # only b3: the output is the bias
    y, _ = m.forward(p, np.ones((3, 6)))
    np.testing.assert_allclose(y, [[0.5, -1.5]] * 3)
    loss, g = m.loss_and_grad(p, np.ones((3, 6)), np.zeros((3, 2)))
    assert loss == pytest.approx((0.25 + 2.25) / 2)
    np.testing.assert_allclose(g[-2:], [0.5, -1.5])   # d/db3 of mean (b3)^2 over 2 outputs
    np.testing.assert_allclose(g[:-2], 0.0)


def test_sampler_counts_on_a_uniform_grid_match_the_probabilities():
    """Inverse-transform sampling with the S grid uniforms (s + 1/2)/S puts floor or ceil of
    p_j S shots in bin j (the cdf steps are p_j): a deterministic pin of the sampler."""
    p = np.array([0.1, 0.25, 0.0, 0.3, 0.35])
    v = np.sqrt(p) * np.exp(1j * np.array([0.3, -1.0, 0.0, 2.0, 0.5]))
    S = 1000
    u = (np.arange(S) + 0.5) / S
    counts = o.sample_counts(v, u)
    assert counts.sum() == S
    assert np.all(np.abs(counts - p * S) <= 1.0)
    assert counts[2] == 0
    # a single bin takes every shot; the last bin takes u -> 1
    assert o.sample_counts(np.array([0, 0, 1.0]), u).tolist() == [0, 0, S]
    assert o.sample_counts(np.array([1.0, 1.0]), np.array([0.0, 0.4999, 0.5, 0.999999])).tolist() == [2, 2]
