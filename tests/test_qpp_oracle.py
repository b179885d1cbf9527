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


def test_controlled_swap_brute_force():
    """The Fredkin decomposition against the explicit permutation on 3 qubits."""
    rng = np.random.default_rng(9)
    psi = rng.normal(size=8) + 1j * rng.normal(size=8)
    got = psi.copy()
    q._controlled_swap(got, 3, 2, 0, 1)
    want = psi.copy()
    want[[5, 6]] = psi[[6, 5]]                 # c = bit 2 set: |c=1, y=0, x=1> <-> |c=1, y=1, x=0>
    np.testing.assert_allclose(got, want, atol=0)


@pytest.mark.parametrize("n", [2, 4, 8])
def test_swap_test_state_is_the_printed_superposition(n):
    """STEPS 1-3 run gate by gate give, per address s, (1/2 sqrt N)[(|zeta>|s> + |s>|zeta>)|0>
    + (|zeta>|s> - |s>|zeta>)|1>] on ua, a1, a2; the weight of a2 = 0 is (1 + zeta_s^2) / 2
    (= sin^2(pi beta) of STEP 4)."""
    rng = np.random.default_rng(n)
    z = rng.normal(size=n)
    z /= np.linalg.norm(z)
    psi = q.swap_test_prepare(z).reshape(n, 2, n, n)          # [s, a2, a1, ua]
    for s in range(n):
        zs = np.kron(np.eye(n)[s], z).reshape(n, n)            # |zeta>_ua |s>_a1: row a1 = s
        sz = zs.T                                              # |s>_ua |zeta>_a1
        np.testing.assert_allclose(psi[s, 0], (zs + sz) / (2 * np.sqrt(n)), atol=1e-15)
        np.testing.assert_allclose(psi[s, 1], (zs - sz) / (2 * np.sqrt(n)), atol=1e-15)
        w0 = n * float(np.sum(np.abs(psi[s, 0]) ** 2))
        assert w0 == pytest.approx((1 + z[s] ** 2) / 2, abs=1e-14)


def test_swap_test_iterate_eigenphases():
    """Q is orthogonal; each block's start state lies in the eigenspaces e^{+-2 i theta_s}
    with sin^2 theta_s = (1 + zeta_s^2) / 2."""
    rng = np.random.default_rng(12)
    z = rng.uniform(-1.0, 1.0, 4)
    z /= np.linalg.norm(z)
    qq = q.swap_test_iterate(z)
    np.testing.assert_allclose(qq @ qq.T, np.eye(len(qq)), atol=1e-13)
    prep = q.swap_test_prepare(z).reshape(4, -1) * 2.0
    dim = qq.shape[0] // 4
    for s in range(4):
        w, vec = np.linalg.eig(qq[s * dim:(s + 1) * dim, s * dim:(s + 1) * dim])
        coef = np.linalg.solve(vec, prep[s])
        theta = np.arcsin(np.sqrt((1 + z[s] ** 2) / 2))
        on = np.abs(np.abs(np.angle(w)) - 2 * theta) < 1e-9
        assert float(np.sum(np.abs(coef[on]) ** 2)) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("z,c", [((0.0, 1.0), 1.0), ((0.0, 1.0), 0.9), ((0.0, 0.0, -1.0, 0.0), 0.8)])
def test_swap_qadc_exact_on_the_clock_grid(z, c):
    """zeta_s in {0, +-1}: beta = 1/4 or 1/2 sit on the clock grid, so the postselected vector is
    exactly c zeta_s^2 / sqrt(N) times each address's STEPS 1-3 state."""
    z = np.array(z)
    n = len(z)
    _, v = q.qadc_swap_square(z, 4, c=c)
    prep = q.swap_test_prepare(z).reshape(n, -1) * np.sqrt(n)
    want = (c * z[:, None] ** 2 / np.sqrt(n)) * prep
    np.testing.assert_allclose(v, want.reshape(-1), atol=1e-12)
    np.testing.assert_allclose(q.swap_squares(v, z), c * z ** 2 / np.sqrt(n), atol=1e-12)


def test_swap_qadc_off_grid_converges_like_the_amplitude_estimation_form():
    """Random zeta: the address amplitudes approach zeta^2 / 2 as the clock grows, and the
    swap-test and amplitude-estimation conversions agree within their grid errors."""
    rng = np.random.default_rng(6)
    z = rng.uniform(0.2, 1.0, 4)
    z /= np.linalg.norm(z)
    errs = []
    for n_c in (6, 9):
        _, v = q.qadc_swap_square(z, n_c, c=1.0)
        errs.append(np.abs(q.swap_squares(v, z).real - z ** 2 / 2).max())
    assert errs[1] < 0.002 and errs[1] < errs[0]
    _, v_ae = q.qadc_square(z, 9, c=1.0)
    _, v_sw = q.qadc_swap_square(z, 9, c=1.0)
    np.testing.assert_allclose(q.swap_squares(v_sw, z).real, (v_ae.reshape(4, 4) @ z).real, atol=0.004)
