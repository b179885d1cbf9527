"""Pins of the LCU post-processing of the dissipation rate (App. D): the circuit's ancilla
probability against the forward-difference formula, closed forms and brute force."""
import numpy as np
import pytest

from oracle import hhl_oracle as o
from oracle import qpp_oracle as q


@pytest.mark.parametrize("n,walls", [(8, (0.0, 0.0)), (16, (0.0, 1.0)), (32, (0.3, -0.7))])
def test_lcu_dissipation_equals_the_forward_difference_formula(n, walls):
    rng = np.random.default_rng(n)
    u = rng.normal(size=n)
    eps, p0 = q.qpp_dissipation(u, walls[0], walls[1], 0.1)
    assert eps == pytest.approx(o.dissipation(u, walls[0], walls[1], 0.1), rel=1e-12)
    assert 0.0 <= p0 <= 1.0


def test_lcu_closed_forms():
    """Poiseuille y(1-y): eps = nu (1/3 - h^2/3); Couette y: eps = nu; a constant field with
    zero walls has only the two wall jumps."""
    n, nu = 64, 0.5
    y = np.arange(1, n + 1) / (n + 1)
    h = 1.0 / (n + 1)
    assert q.qpp_dissipation(y * (1 - y), 0.0, 0.0, nu)[0] == pytest.approx(nu * (1.0 / 3 - h * h / 3), rel=1e-12)
    assert q.qpp_dissipation(y, 0.0, 1.0, nu)[0] == pytest.approx(nu, rel=1e-12)
    assert q.qpp_dissipation(np.ones(n), 0.0, 0.0, nu)[0] == pytest.approx(nu * 2.0 / h, rel=1e-12)


def test_lcu_probability_brute_force():
    """The circuit is (I - P)/2 on the ancilla-0 block: against the explicit matrix."""
    rng = np.random.default_rng(2)
    w = rng.normal(size=16)
    perm = np.roll(np.eye(16), 1, axis=0)
    d = (np.eye(16) - perm) / 2 @ (w / np.linalg.norm(w))
    assert q.lcu_probability(w) == pytest.approx(float(d @ d), rel=1e-12)


def test_amplitude_estimation_iterate_eigenphases():
    """Each block G_k of Q rotates by 2 theta_k with sin theta_k = |zeta_k| (eigenvalues
    e^{+-2 i theta_k} on the plane of |zeta>, +-1 elsewhere); U_V |0> = |zeta>."""
    rng = np.random.default_rng(4)
    z = rng.uniform(0.1, 1.0, 4)
    z /= np.linalg.norm(z)
    np.testing.assert_allclose(q.state_prep_unitary(z)[:, 0], z, atol=1e-15)
    qq = q.amplitude_estimation_iterate(z)
    np.testing.assert_allclose(qq @ qq.T, np.eye(16), atol=1e-13)
    for k in range(4):
        ev = np.linalg.eigvals(qq[4 * k:4 * k + 4, 4 * k:4 * k + 4])
        ang = np.sort(np.abs(np.angle(ev)))
        want = 2 * np.arcsin(z[k])
        assert np.min(np.abs(ang - want)) < 1e-12


def test_qadc_square_is_exact_on_the_clock_grid():
    """zeta = (sin pi/8, sin 3pi/8): both phases sit on the 4-bit clock grid, so the
    postselected state is exactly (1/sqrt 2) sum_k zeta_k^2 |k> (x) |zeta>."""
    z = np.array([np.sin(np.pi / 8), np.sin(3 * np.pi / 8)])
    _, v = q.qadc_square(z, 4, c=1.0)
    want = np.kron(z ** 2 / np.sqrt(2.0), z)
    np.testing.assert_allclose(v, want, atol=1e-12)


def test_qadc_square_off_grid_converges():
    rng = np.random.default_rng(6)
    z = rng.uniform(0.2, 1.0, 4)
    z /= np.linalg.norm(z)
    _, v = q.qadc_square(z, 8, c=1.0)
    marg = v.reshape(4, 4) @ z             # project the data register on |zeta>
    np.testing.assert_allclose(marg.real, z ** 2 / 2.0, atol=0.02)
