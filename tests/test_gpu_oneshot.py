"""GPU parity of the signed-clock HHL path and of the one-shot time-stepping systems
(App. A, Eqs. FE_OBM / BE_OBM) through their Hermitian dilation: the whole circuit against
the oracle's gate-level circuit, element by element, and the read-out final field against
the oracle's postselected vector (the same circuit) and, loosely, the classical solve.

Tolerances (max absolute amplitude error): 1e-10 for complex128, 1e-5 for complex64.
"""
import math

import numpy as np
import pytest

from oracle import hhl_oracle as o
from oracle import oneshot_oracle as os1

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


@pytest.mark.parametrize("prec,gemm", [("c128", "simt"), ("c64", "simt")])
def test_signed_clock_on_grid_indefinite(hhl, prec, gemm):
    """Indefinite 4 x 4 A with eigenvalues 3, -5, 7, -2 on the clock grid: the GPU state
    equals the oracle's, and the postselected vector is C Ahat^{-1} bhat."""
    rng = np.random.default_rng(11)
    q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    a = q @ np.diag([3.0, -5.0, 7.0, -2.0]) @ q.T
    lub = o.gershgorin_bound(a)
    n_s, n_c = 2, 5
    t0 = 2 * math.pi * lub
    pl = o.plan(a, n_c, t0_rule="user", t0=t0, signed=True)
    b = rng.uniform(0.0, 1.0, 4)
    ref = o.hhl_circuit(b, n_s, pl)
    plan = hhl.HHLPlan(n_s, n_c, dense=a, precision=prec, gemm=gemm, t0_rule="user", t0=t0, signed_clock=True,
                       full_uncompute=True)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    np.testing.assert_allclose(_np(st), ref, atol=TOL[prec])
    meas = plan.measure(st)
    v = meas["xhat"] * math.sqrt(meas["p_success"])
    want = pl["C"] * np.linalg.solve(a / lub, b / np.linalg.norm(b))
    np.testing.assert_allclose(v, want, atol=10 * TOL[prec])


def test_unsigned_clock_refuses_an_indefinite_matrix(hhl):
    a = np.diag([1.0, -2.0, 3.0, 4.0])
    with pytest.raises(RuntimeError, match="positive definite"):
        hhl.HHLPlan(2, 4, dense=a)


@pytest.mark.parametrize("scheme,prec,gemm,n,n_c", [("fe", "c128", "simt", 4, 8), ("fe", "c64", "simt", 4, 8),
                                                   ("be", "c128", "simt", 4, 8), ("be", "c64", "simt", 4, 8),
                                                   ("fe", "c64", "tcgen05", 8, 9), ("be", "c64", "tcgen05", 8, 9),
                                                   ("be", "c128", "simt", 8, 9)])
def test_one_shot_dilated_system_parity(hhl, scheme, prec, gemm, n, n_c):
    """N_g = 4 (8) grid points, m = 5 steps held for p = 2 more: a 32 x 32 (64 x 64) block
    system, its 64 x 64 (128 x 128) dilation with 8 (9) signed clock qubits: 15 (17) qubits;
    the larger case takes the tcgen05 GEMM in complex64."""
    from paper_2307_00391_gb300 import oneshot as lib1
    rng = np.random.default_rng(17)
    m, p = 5, 2
    a = os1.time_operator(n)
    f = np.full(n, 8.0)
    u_in = rng.uniform(0.0, 1.0, n)
    dt = 0.25 / (n + 1) ** 2         # Courant number 0.25
    big, rhs = (os1.fe_system if scheme == "fe" else os1.be_system)(a, f, u_in, dt, m, p)
    hp, rp = os1.dilated_problem(big, rhs)
    n_s = int(math.log2(hp.shape[0]))
    pl = o.plan(hp, n_c, signed=True)
    ref = o.hhl_circuit(rp, n_s, pl)
    res = lib1.solve_one_shot(a, f, u_in, dt, m, p, n_c, scheme=scheme, precision=prec, gemm=gemm)
    assert res["info"]["t0"] == pytest.approx(pl["t0"], rel=1e-12)
    assert res["info"]["lambda_ub"] == pytest.approx(pl["lam_ub"], rel=1e-12)
    # postselect-early mode: the anc = 1 half is the uncomputed one
    half = 1 << (n_s + n_c)
    np.testing.assert_allclose(_np(res["state"])[half:], ref[half:], atol=TOL[prec])
    # read-out: the final field from the oracle's postselected vector, denormalised the same way
    ps = o.postselect(ref, n_s, n_c)
    x_ref = np.linalg.norm(rp) * ps["v"].real / (pl["C"] * pl["lam_ub"])
    k = big.shape[0]
    final_ref = os1.final_slice(os1.solution_part(x_ref, k), n, m, p)
    scale = np.abs(final_ref).max()
    assert np.abs(res["final"] - final_ref).max() <= (1e-8 if prec == "c128" else 2e-3) * scale
    # 8-9 signed clock qubits resolve these dilations (kappa 8-15) well: within 3% of the
    # classical solve of the block system (the oracle's own circuit is within 0.7-2.3%)
    exact = os1.final_slice(np.linalg.solve(big, rhs), n, m, p)
    assert np.abs(res["final"] - exact).max() <= 0.03 * np.abs(exact).max()


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_qsp2_sparse_preparation(hhl, prec):
    """QSP-2 on a signed sparse vector (9 nonzeros of 2^7, plus one position outside the
    register, which is ignored): every clock row holds the oracle's QSP-2 state / 2^(n_c/2),
    the anc = 1 half is zero, and |val| is recorded."""
    import torch
    rng = np.random.default_rng(23)
    n_s, n_c = 7, 4
    N, R = 1 << n_s, 1 << n_c
    idx = np.sort(rng.choice(N, size=9, replace=False))
    val = rng.uniform(0.2, 1.0, 9) * rng.choice([-1.0, 1.0], 9)
    ref_sys = o.qsp2_prepare(idx, val, n_s)
    diag, off = o.laplacian_tridiag(N)
    plan = hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision=prec)
    st = plan.new_state()
    idx_all = np.concatenate([idx, [N + 5]])
    val_all = np.concatenate([val, [3.0]])
    plan.prepare_rhs_qsp2(torch.tensor(idx_all, dtype=torch.int64, device="cuda"),
                          torch.tensor(val_all, dtype=torch.float64, device="cuda"), st)
    got = _np(st).reshape(2, R, N)
    for c in range(R):
        np.testing.assert_allclose(got[0, c], ref_sys / math.sqrt(R), atol=TOL[prec])
    assert np.abs(got[1]).max() == 0.0
    out = torch.empty(4 + 2 * N, dtype=torch.float64, device="cuda")
    plan.measure_async(st, out)   # before the circuit: only the recorded |b| and the norm
    assert out[3].item() == pytest.approx(np.linalg.norm(val), rel=1e-12)
    assert out[2].item() == pytest.approx(1.0, abs=10 * TOL[prec])


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_one_shot_with_qsp2_preparation(hhl, prec):
    """The one-shot FE system prepared by QSP-2 (its right-hand side has 24 nonzeros in 2^6):
    the same circuit output as with amplitude encoding."""
    from paper_2307_00391_gb300 import oneshot as lib1
    rng = np.random.default_rng(29)
    n, m, p, n_c = 4, 5, 2, 8
    a = os1.time_operator(n)
    f = np.full(n, 8.0)
    u_in = rng.uniform(0.0, 1.0, n)
    dt = 0.25 / 25.0
    r1 = lib1.solve_one_shot(a, f, u_in, dt, m, p, n_c, precision=prec, gemm="simt", prep="amplitude")
    r2 = lib1.solve_one_shot(a, f, u_in, dt, m, p, n_c, precision=prec, gemm="simt", prep="qsp2")
    np.testing.assert_allclose(_np(r2["state"]), _np(r1["state"]), atol=TOL[prec])
    np.testing.assert_allclose(r2["final"], r1["final"], rtol=1e-6 if prec == "c128" else 1e-3)


@pytest.mark.parametrize("prec,prep", [("c128", "qsp1"), ("c64", "qsp1"), ("c64", "amplitude")])
def test_iterative_backward_euler_loop(hhl, prec, prep):
    """The hybrid BE loop (16 grid points, 10 clock qubits): every step's read-out equals the
    oracle's HHL read-out on the same right-hand side, and the trajectory tracks the exact
    backward-Euler march to within the HHL error (0.6% per step at this clock size)."""
    from paper_2307_00391_gb300 import iterative
    n, nu, dt, n_c, steps = 16, 1.0, 0.01, 10, 5
    a = os1.time_operator(n, nu)
    f = np.full(n, 2.0)
    u0 = np.zeros(n)
    a1 = os1.be1_operator(a, dt)
    pl = o.plan(a1, n_c)

    def check(j, b, u_next):
        psi = o.hhl_circuit(b, 4, pl)
        v = o.postselect(psi, 4, n_c)["v"]
        ref = o.velocity(v, np.linalg.norm(b), pl["C"], pl["lam_ub"])
        assert np.abs(u_next - ref).max() <= (1e-9 if prec == "c128" else 1e-4) * np.abs(ref).max(), j

    out = iterative.iterative_be(n, nu, f, u0, dt, n_c, steps, tol=0.0, precision=prec, prep=prep, on_step=check)
    assert out["info"]["lambda_ub"] == pytest.approx(pl["lam_ub"], rel=1e-12)
    march = os1.be_march(a, f, u0, dt, steps, 0)
    for j in range(1, steps + 1):
        assert np.abs(out["fields"][j] - march[j]).max() <= 0.01 * j * np.abs(march[j]).max()
    assert len(out["residues"]) == steps and all(r > 0 for r in out["residues"])
