"""The postselected solve (hhl_solve_postselected: QPE by doubling, the clock block, the
uncompute, final Hadamards and postselection folded into one row) against the FP64 oracle's
whole circuit and against the library's full-state path, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import hhl_oracle as o
from tests.oracle_stages import problem, run_stages

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-5}


@pytest.fixture(scope="module")
def hhl():
    import torch
    assert torch.cuda.is_available()
    import paper_2307_00391_gb300 as pkg
    pkg.load()
    return pkg


def _b_dev(b):
    import torch
    return torch.tensor(np.asarray(b, dtype=np.complex128), device="cuda")


def _postselected(hhl, plan, b, n_s, n_c):
    import torch
    N = 1 << n_s
    st = plan.new_state()
    out = torch.empty(4 + 2 * N, dtype=torch.float64, device="cuda")
    eps = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.solve_postselected(_b_dev(b), st, out, eps)
    torch.cuda.synchronize()
    o_h = out.cpu().numpy()
    v = st.view(2, 1 << n_c, N)[1, 0].cpu().numpy().astype(np.complex128)
    return dict(p_success=o_h[0], p_anc1=o_h[1], norm=o_h[2], b_norm=o_h[3], xhat=o_h[4::2] + 1j * o_h[5::2],
                v=v, eps=float(eps.item()))


@pytest.mark.parametrize("prec", ["c128", "c64", "c128-fp64pipe"])
@pytest.mark.parametrize("flow,n_s,n_c,dt,r_max", [("poiseuille", 5, 4, 8.0, 0),     # one bit per pass
                                                   ("couette", 5, 9, 1.0e4, 0),      # 8 bits in one pass
                                                   ("couette", 5, 10, 500.0, 0),     # groups and single bits
                                                   ("poiseuille", 10, 7, 50.0, 8),   # rows of several windows
                                                   ("couette", 1, 3, 1.0, 8)])       # the smallest row
@pytest.mark.parametrize("split", [False, True])
def test_postselected_solve_matches_oracle(hhl, monkeypatch, prec, flow, n_s, n_c, dt, r_max, split):
    """split: the clock block as split register passes (the path of large states, where pass B
    sums the two halves' weights instead of storing the anc = 0 half), forced on small states."""
    if prec == "c128-fp64pipe":
        monkeypatch.setenv("HHL_FP64_PIPE", "1")
        prec = "c128"
    if split:
        if n_c < 8 or (1 << n_s) * 8 < 256:
            pytest.skip("the split passes need 8 or more clock bits and 256-byte rows")
        monkeypatch.setenv("HHL_FFT_SPLIT", "1")
        monkeypatch.setenv("HHL_CLOCK_CLUSTER", "0")
    diag, off, b, walls = problem(flow, n_s)
    nu = 0.05
    pl = o.plan(o.dense_from_tridiag(diag, off), n_c, t0_rule="range_fill")
    lub = pl["lam_ub"]
    ref = run_stages(b, n_s, pl, trotter=dict(diag=diag / lub, off=off / lub, dt=dt, r_max=r_max))
    psi = ref["final_h"]
    post = o.postselect(psi, n_s, n_c)
    plan = hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision=prec, expm="trotter", trotter_dt=dt,
                       trotter_steps_max=r_max, nu=nu, walls=walls)
    got = _postselected(hhl, plan, b, n_s, n_c)
    tol = TOL[prec]
    N = 1 << n_s
    v_ref = psi.reshape(2, 1 << n_c, N)[1, 0]
    dv = np.abs(got["v"] - v_ref).max()
    assert dv <= tol, dv
    # P(anc = 1) before the uncompute equals the whole circuit's (the uncompute is unitary)
    assert got["p_anc1"] == pytest.approx(post["p_anc1"], rel=1e-9 if prec == "c128" else 1e-4)
    assert got["norm"] == pytest.approx(1.0, abs=1e-12 if prec == "c128" else 1e-5)
    assert got["b_norm"] == pytest.approx(np.linalg.norm(b), rel=1e-14)
    assert got["p_success"] == pytest.approx(post["p_success"], rel=1e-9 if prec == "c128" else 1e-4)
    bound = (1.0 + math.sqrt(N)) * dv / (np.linalg.norm(got["v"]) - math.sqrt(N) * dv) + 1e-13
    np.testing.assert_allclose(got["xhat"], post["xhat"], atol=bound)
    u_ref = o.velocity(post["v"], np.linalg.norm(b), pl["C"], pl["lam_ub"])
    eps_ref = o.dissipation(u_ref, walls[0], walls[1], nu)
    assert got["eps"] == pytest.approx(eps_ref, rel=1e-9 if prec == "c128" else 1e-3)


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_postselected_equals_full_state_path(hhl, prec):
    """A 26-qubit case (2^16 system amplitudes, 9 clock qubits): the postselected solve against
    the full-state circuit of the same plan (hhl_apply_circuit + hhl_measure), and the readouts
    that take the postselected row (dissipation, shots) on both."""
    import torch
    from synth_inputs import uniform_draws
    n_s, n_c = 16, 9
    N = 1 << n_s
    diag, off, b, walls = problem("poiseuille", n_s)
    plan = hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision=prec, expm="trotter", trotter_dt=1024.0,
                       trotter_steps_max=8, walls=walls)
    got = _postselected(hhl, plan, b, n_s, n_c)
    st = plan.new_state()
    plan.prepare_rhs(_b_dev(b), st)
    plan.apply_circuit(st)
    m = plan.measure(st)
    v_full = st.view(2, 1 << n_c, N)[1, 0].cpu().numpy().astype(np.complex128)
    # complex64: 1e-5 of the largest entry (the entries are ~1e-4); complex128: 1e-10 absolute
    bound = 1e-5 * np.abs(v_full).max() if prec == "c64" else 1e-10
    assert np.abs(got["v"] - v_full).max() <= bound
    assert got["p_anc1"] == pytest.approx(m["p_anc1"], rel=1e-4 if prec == "c64" else 1e-9)
    assert got["p_success"] == pytest.approx(m["p_success"], rel=1e-4 if prec == "c64" else 1e-9)
    assert abs(np.vdot(got["xhat"], m["xhat"])) >= 1 - 1e-6
    assert got["eps"] == pytest.approx(plan.dissipation(st), rel=1e-3 if prec == "c64" else 1e-9)


def test_postselected_solve_refuses_other_plans(hhl):
    import torch
    diag, off, b, walls = problem("poiseuille", 4)
    out = torch.empty(4 + 32, dtype=torch.float64, device="cuda")
    for kw in (dict(expm="trotter", full_uncompute=True),
               dict(expm="trotter", trotter_dt=1e-3, trotter_steps_max=40)):   # a bit over several passes
        plan = hhl.HHLPlan(4, 5, diag=diag, off=off, precision="c64", **kw)
        st = plan.new_state()
        with pytest.raises(hhl.HHLError) as e:
            plan.solve_postselected(_b_dev(b), st, out)
        assert e.value.status == 8


@pytest.mark.slow
def test_postselected_32_qubits_against_full_state(hhl):
    """The 32-qubit Poiseuille workload (N = 2^18, n_c = 13, complex64): the postselected solve
    against the full-state circuit, element by element on v (relative to its largest entry)."""
    import torch
    from synth_inputs import rhs
    n_s, n_c = 18, 13
    N = 1 << n_s
    diag, off = o.laplacian_tridiag(N)
    b = rhs("poiseuille", N)
    plan = hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision="c64", expm="trotter", trotter_dt=1024.0,
                       trotter_steps_max=8)
    got = _postselected(hhl, plan, b, n_s, n_c)
    torch.cuda.empty_cache()
    st = plan.new_state()
    plan.prepare_rhs(_b_dev(b), st)
    plan.apply_circuit(st)
    m = plan.measure(st)
    v_full = st.view(2, 1 << n_c, N)[1, 0].cpu().numpy().astype(np.complex128)
    del st
    torch.cuda.empty_cache()
    assert np.abs(got["v"] - v_full).max() <= 1e-5 * np.abs(v_full).max()
    assert got["p_anc1"] == pytest.approx(m["p_anc1"], rel=1e-4)
    assert got["norm"] == pytest.approx(1.0, abs=1e-5)
    assert abs(np.vdot(got["xhat"], m["xhat"])) >= 1 - 1e-6


@pytest.mark.parametrize("prec,gemm,flow,n_s,n_c", [("c64", "tcgen05", "couette", 7, 8),      # k = 7 on tcgen05
                                                    ("c64", "tcgen05", "poiseuille", 8, 10),  # k = 7..9 on tcgen05
                                                    ("c64", "simt", "poiseuille", 4, 6),
                                                    ("c128", "simt", "couette", 5, 7),
                                                    ("c128", "simt", "poiseuille", 1, 3)])
def test_postselected_dense_matches_oracle(hhl, prec, gemm, flow, n_s, n_c):
    """The dense form of the postselected solve (the trees as controlled-U GEMMs on 2^k rows:
    tcgen05 where 2^k >= 128, CUDA cores below) against the oracle's whole circuit."""
    diag, off, b, walls = problem(flow, n_s)
    nu = 0.05
    pl = o.plan(o.dense_from_tridiag(diag, off), n_c, t0_rule="range_fill")
    psi = run_stages(b, n_s, pl)["final_h"]
    post = o.postselect(psi, n_s, n_c)
    plan = hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision=prec, gemm=gemm, nu=nu, walls=walls)
    got = _postselected(hhl, plan, b, n_s, n_c)
    N = 1 << n_s
    tol = TOL[prec]
    v_ref = psi.reshape(2, 1 << n_c, N)[1, 0]
    dv = np.abs(got["v"] - v_ref).max()
    assert dv <= tol, dv
    assert got["p_anc1"] == pytest.approx(post["p_anc1"], rel=1e-9 if prec == "c128" else 1e-4)
    assert got["p_success"] == pytest.approx(post["p_success"], rel=1e-9 if prec == "c128" else 1e-4)
    bound = (1.0 + math.sqrt(N)) * dv / (np.linalg.norm(got["v"]) - math.sqrt(N) * dv) + 1e-13
    np.testing.assert_allclose(got["xhat"], post["xhat"], atol=bound)
    u_ref = o.velocity(post["v"], np.linalg.norm(b), pl["C"], pl["lam_ub"])
    assert got["eps"] == pytest.approx(o.dissipation(u_ref, walls[0], walls[1], nu), rel=1e-9 if prec == "c128" else 1e-3)


@pytest.mark.parametrize("gemm", ["tcgen05", "simt"])
def test_postselected_dense_general_matrix(hhl, gemm):
    """A dense symmetric A that is not Toeplitz (U_k from its Jacobi eigenvectors; the small
    tree steps then multiply stored CUDA-core operands) against the oracle's whole circuit."""
    n_s, n_c = 7, 8
    N = 1 << n_s
    rng = np.random.default_rng(29)
    q = np.linalg.qr(rng.standard_normal((N, N)))[0]
    a = q @ np.diag(rng.uniform(1.0, 9.0, N)) @ q.T
    a = 0.5 * (a + a.T)
    b = rng.random(N)
    pl = o.plan(a, n_c, t0_rule="range_fill")
    psi = run_stages(b, n_s, pl)["final_h"]
    post = o.postselect(psi, n_s, n_c)
    plan = hhl.HHLPlan(n_s, n_c, dense=a, precision="c64", gemm=gemm)
    got = _postselected(hhl, plan, b, n_s, n_c)
    dv = np.abs(got["v"] - psi.reshape(2, 1 << n_c, N)[1, 0]).max()
    assert dv <= TOL["c64"], dv
    assert got["p_success"] == pytest.approx(post["p_success"], rel=1e-4)


def test_postselected_dense_refuses_full_uncompute(hhl):
    import torch
    diag, off, b, walls = problem("poiseuille", 4)
    plan = hhl.HHLPlan(4, 5, diag=diag, off=off, precision="c64", full_uncompute=True)
    with pytest.raises(hhl.HHLError) as e:
        plan.solve_postselected(_b_dev(b), plan.new_state(), torch.empty(40, dtype=torch.float64, device="cuda"))
    assert e.value.status == 8
