"""T0 - Q_PE scans (Sec. VI, Figs. 3b-d): the fit helpers on synthetic fidelity grids with a
known optimum (host logic), and a small scan through the batched engine on the GPU with
sampled instances re-checked by the oracle circuit."""
import math

import numpy as np
import pytest

from oracle import hhl_oracle as o


def _synthetic(a_true, b_true):
    from paper_2307_00391_gb300 import tq_scan
    kappa = 10.0 ** np.linspace(0.5, 3.5, 12)
    scales = 10.0 ** np.linspace(-1.5, 1.5, 61)
    ncs = [4, 5, 6]
    F = np.zeros((len(kappa), len(ncs), len(scales)))
    for p, k in enumerate(kappa):
        t_star = math.exp(a_true) * k ** b_true
        s_star = t_star / tq_scan.t0_power_law_per_unit(k)
        for c, nc in enumerate(ncs):
            floor = 0.3 * 2.0 ** (-nc)
            F[p, c] = 1.0 - floor - 0.1 * (np.log(scales / s_star)) ** 2
    return dict(F=F, scales=scales, n_clocks=ncs, kappa=kappa)


def test_fits_recover_a_known_power_law_and_floor():
    from paper_2307_00391_gb300 import tq_scan
    sw = _synthetic(1.2, -0.5)
    fit = tq_scan.fit_t0_kappa(sw)
    assert fit["b"] == pytest.approx(-0.5, abs=0.03) and fit["a"] == pytest.approx(1.2, abs=0.1)
    assert fit["r2"] > 0.99
    fl = tq_scan.eps_floor_slope(sw)
    assert fl["beta_mean"] == pytest.approx(-math.log(2.0), abs=0.02)   # grid offset of the optimum
    assert list(tq_scan.qpe_min(sw, 0.3 * 2.0 ** -5 + 1e-3)) == [5] * 12   # floor(5) + grid offset < target < floor(4)
    assert tq_scan.kappa_tridiag(2.0, -1.0, 16) == pytest.approx(o.condition_number(
        o.dense_from_tridiag(np.full(16, 2.0), np.full(15, -1.0))), rel=1e-12)


@pytest.mark.gpu
def test_scan_on_the_batched_engine():
    """9 problems x 4 clock counts x 13 T0 values (468 instances): sampled fidelities equal
    the oracle circuit's, the error floor falls with the clock count, and the fitted
    T0*-kappa relation is reported with its fit quality."""
    import torch
    assert torch.cuda.is_available()
    from paper_2307_00391_gb300 import tq_scan
    from synth_inputs import rhs  # noqa: F401  (the scan's problem generator uses it)
    sw = tq_scan.scan(n_problems=9, n_clocks=(4, 5, 6, 7), scales=10.0 ** np.linspace(-1.5, 1.5, 13),
                      seed=3, ns_range=(3, 4))
    F = sw["F"]
    assert F.shape == (9, 4, 13) and np.all((F >= 0) & (F <= 1 + 1e-6))
    rng = np.random.default_rng(1)
    for _ in range(4):
        p, c, s = int(rng.integers(9)), int(rng.integers(4)), int(rng.integers(13))
        pr = sw["problems"][p]
        a = o.dense_from_tridiag(np.full(pr["N"], pr["diag"]), np.full(pr["N"] - 1, pr["off"]))
        nc = sw["n_clocks"][c]
        t0 = sw["scales"][s] * tq_scan.t0_power_law_per_unit(sw["kappa"][p]) * (1 << nc)
        pl = o.plan(a, nc, t0_rule="user", t0=t0)
        v = o.postselect(o.hhl_circuit(pr["b"], pr["n_s"], pl), pr["n_s"], nc)["v"]
        xc = np.linalg.solve(a, pr["b"])
        f_ref = abs(np.vdot(xc / np.linalg.norm(xc), v / np.linalg.norm(v)))
        assert F[p, c, s] == pytest.approx(f_ref, abs=2e-4), (p, c, s)
    fl = tq_scan.eps_floor_slope(sw)
    assert fl["beta_mean"] < 0.0
    fit = tq_scan.fit_t0_kappa(sw)
    assert math.isfinite(fit["a"]) and math.isfinite(fit["b"]) and fit["points"] == 36
