"""GPU parity of the QPP nonlinear transform (App. D: QADC, squaring rotation, QDAC) run as a
UNITARY plan, in its amplitude-estimation and swap-test forms: the state against the oracle's
gate-level circuit, the exact on-grid cases, and off-grid convergence of the address
amplitudes to z_k^2."""
import numpy as np
import pytest

from oracle import qpp_oracle as q

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-5}


@pytest.fixture(scope="module")
def hhl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2307_00391_gb300 as pkg
    pkg.load()
    return pkg


def _np(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def test_library_iterate_and_table_match_the_oracle(hhl):
    from paper_2307_00391_gb300 import qpp
    rng = np.random.default_rng(8)
    z = rng.uniform(0.1, 1.0, 8)
    z /= np.linalg.norm(z)
    np.testing.assert_allclose(qpp.iterate(z), q.amplitude_estimation_iterate(z), atol=1e-14)
    np.testing.assert_allclose(qpp.rotation_table(7, 0.9), q.squaring_angles(7, 0.9), atol=1e-15)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_qadc_square_on_grid_exact(hhl, prec):
    from paper_2307_00391_gb300 import qpp
    z = np.array([np.sin(np.pi / 8), np.sin(3 * np.pi / 8)])
    res = qpp.square_amplitudes(z, 4, precision=prec)
    np.testing.assert_allclose(res["v"], np.kron(z ** 2 / np.sqrt(2.0), z), atol=10 * TOL[prec])


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_qadc_square_parity_and_convergence(hhl, prec):
    from paper_2307_00391_gb300 import qpp
    rng = np.random.default_rng(6)
    z = rng.uniform(0.2, 1.0, 4)
    z /= np.linalg.norm(z)
    n_c = 8
    psi_ref, v_ref = q.qadc_square(z, n_c, c=1.0)
    res = qpp.square_amplitudes(z, n_c, precision=prec)
    half = 1 << (4 + n_c)
    np.testing.assert_allclose(_np(res["state"])[half:], psi_ref[half:], atol=TOL[prec])
    np.testing.assert_allclose(res["v"], v_ref, atol=10 * TOL[prec])
    np.testing.assert_allclose(res["squares"].real, z ** 2 / 2.0, atol=0.02)


def test_library_swap_form_matches_the_oracle(hhl):
    from paper_2307_00391_gb300 import qpp
    rng = np.random.default_rng(10)
    z = rng.uniform(-1.0, 1.0, 4)
    z /= np.linalg.norm(z)
    np.testing.assert_allclose(qpp.swap_register_state(z), q.swap_test_prepare(z).real, atol=1e-15)
    np.testing.assert_allclose(qpp.swap_iterate(z), q.swap_test_iterate(z), atol=1e-14)
    np.testing.assert_allclose(qpp.swap_rotation_table(7, 0.9), q.swap_squaring_angles(7, 0.9), atol=1e-15)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("z,c", [((0.0, 1.0), 1.0), ((0.0, 0.0, -1.0, 0.0), 0.8)])
def test_swap_qadc_on_grid_exact(hhl, prec, z, c):
    from paper_2307_00391_gb300 import qpp
    z = np.array(z)
    res = qpp.square_amplitudes(z, 4, c=c, precision=prec, form="swap")
    np.testing.assert_allclose(res["squares"], c * z ** 2 / np.sqrt(len(z)), atol=10 * TOL[prec])


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_swap_qadc_parity_and_convergence(hhl, prec):
    """The swap-test form (3a + 1 = 7 system qubits, 8 clock bits, 16 qubits in all) against
    the oracle's gate-level circuit, and its address amplitudes against zeta^2 / 2."""
    from paper_2307_00391_gb300 import qpp
    rng = np.random.default_rng(6)
    z = rng.uniform(0.2, 1.0, 4)
    z /= np.linalg.norm(z)
    n_c = 8
    psi_ref, v_ref = q.qadc_swap_square(z, n_c, c=1.0)
    res = qpp.square_amplitudes(z, n_c, precision=prec, form="swap")
    half = 1 << (7 + n_c)
    np.testing.assert_allclose(_np(res["state"])[half:], psi_ref[half:], atol=TOL[prec])
    np.testing.assert_allclose(res["v"], v_ref, atol=10 * TOL[prec])
    np.testing.assert_allclose(res["squares"].real, q.swap_squares(v_ref, z).real, atol=10 * TOL[prec])
    np.testing.assert_allclose(res["squares"].real, z ** 2 / 2.0, atol=0.005)
