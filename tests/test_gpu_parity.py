"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (max absolute amplitude error): 1e-10 for complex128, 1e-5 for complex64. Where the
amplitudes of a register are themselves of order 1e-5 (the 32- and 34-qubit states), the same
bound is applied relative to the largest amplitude of the compared row or column. Quantities
derived from the postselected vector v are checked against the bound that the amplitude bound
implies for them: xhat = v / |v| moves by at most (1 + sqrt(N)) max|dv| / |v| per entry.
"""
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
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2307_00391_gb300 as pkg
    pkg.load()
    return pkg


def _np(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def _oracle_plan(diag, off, n_c, rule="range_fill", t0=None, conv="total", C=None):
    a = o.dense_from_tridiag(diag, off)
    return o.plan(a, n_c, t0_rule=rule, t0=t0, t0_convention=conv, c_const=C)


def _gpu_plan(hhl, diag, off, n_s, n_c, prec, **kw):
    return hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision=prec, **kw)


def _b_dev(b):
    import torch
    return torch.tensor(np.asarray(b, dtype=np.complex128), device="cuda")


def _half(psi, n_s, n_c, anc):
    return psi.reshape(2, 1 << n_c, 1 << n_s)[anc]


def xhat_bound(dv_max, v_norm, n):
    """Entry-wise bound on the change of xhat = v / |v| when every entry of v moves by at most
    dv_max: |dx_i| <= |dv_i| / |v'| + |v_i| | |v| - |v'| | / (|v| |v'|) <= (1 + sqrt(n)) dv_max / |v'|
    (|v_i| <= |v|, | |v| - |v'| | <= |dv|_2 <= sqrt(n) dv_max), plus FP64 rounding slack."""
    return (1.0 + math.sqrt(n)) * dv_max / (v_norm - math.sqrt(n) * dv_max) + 1e-13


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("flow,n_s,n_c,rule", [("poiseuille", 4, 6, "power_law"),   # the 11-qubit Poiseuille case
                                               ("couette", 7, 8, "range_fill"),
                                               ("poiseuille", 5, 3, "range_fill"),
                                               ("couette", 3, 12, "range_fill")])   # cluster-split clock
def test_stagewise_parity(hhl, prec, full, flow, n_s, n_c, rule):
    import torch
    diag, off, b, walls = problem(flow, n_s)
    pl = _oracle_plan(diag, off, n_c, rule)
    ref = run_stages(b, n_s, pl)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, t0_rule=rule, full_uncompute=full, gemm="simt")
    assert plan.info["t0"] == pytest.approx(pl["t0"], rel=1e-12)
    st = plan.new_state()
    plan.prepare_rhs(_b_dev(b), st)
    tol = TOL[prec]
    np.testing.assert_allclose(_np(st), ref["prep"], atol=tol)
    plan.apply_stage("qpe_u", st)
    np.testing.assert_allclose(_np(st), ref["qpe_u"], atol=tol)
    plan.apply_stage("clock_block", st)
    got = _np(st)
    np.testing.assert_allclose(_half(got, n_s, n_c, 1), _half(ref["clock_block"], n_s, n_c, 1), atol=tol)
    anc0_ref = ref["clock_block"] if full else ref["rotated"]
    np.testing.assert_allclose(_half(got, n_s, n_c, 0), _half(anc0_ref, n_s, n_c, 0), atol=tol)
    plan.apply_stage("uncompute_u", st)
    got = _np(st)
    np.testing.assert_allclose(_half(got, n_s, n_c, 1), _half(ref["uncompute_u"], n_s, n_c, 1), atol=tol)
    if full:
        np.testing.assert_allclose(got, ref["uncompute_u"], atol=tol)
    plan.apply_stage("final_h", st)
    got = _np(st)
    np.testing.assert_allclose(_half(got, n_s, n_c, 1), _half(ref["final_h"], n_s, n_c, 1), atol=tol)
    if full:
        np.testing.assert_allclose(got, ref["final_h"], atol=tol)
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n_s,n_c,kind", [(2, 3, "worked"), (4, 6, "poiseuille"), (6, 5, "random"),
                                          (10, 4, "couette")])
def test_qsp1_gate_level_preparation(hhl, prec, n_s, n_c, kind):
    """The QSP-1 tree on the GPU against the oracle's gate sequence (App. C), and against the
    direct amplitude encoding of hhl_prepare_rhs for non-negative b."""
    import json
    import os
    import torch
    from synth_inputs import random_rhs
    N = 1 << n_s
    if kind == "worked":
        fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "qsp1_worked_example.json")))
        b = np.sqrt(np.array(fx["leaf_probabilities"], dtype=np.float64))
    elif kind == "random":
        b = random_rhs(N, seed_offset=31)
    else:
        b = problem(kind, n_s)[2]
    diag, off = o.laplacian_tridiag(N)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec)
    st = plan.new_state()
    plan.prepare_rhs_qsp1(torch.tensor(b, dtype=torch.float64, device="cuda"), st)
    got = _np(st)
    sys_ref = o.qsp1_prepare(b / np.linalg.norm(b))
    ref = np.zeros(2 << (n_s + n_c), dtype=np.complex128)
    ref[: 1 << (n_s + n_c)] = np.tile(sys_ref, 1 << n_c) / math.sqrt(1 << n_c)
    np.testing.assert_allclose(got, ref, atol=TOL[prec])
    np.testing.assert_allclose(got, o.prepare_state(b, n_s, n_c), atol=TOL[prec])


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_shots_match_the_oracle_sampler(hhl, prec):
    """Shots of the postselected register from the same uniforms: the oracle's inverse-
    transform sampler on the oracle's final state against the GPU sampler on the GPU state;
    shots whose uniform falls within the two states' probability difference of a bin edge are
    the only ones allowed to differ."""
    import torch
    from synth_inputs import uniform_draws
    n_s, n_c = 6, 7
    diag, off, b, walls = problem("poiseuille", n_s)
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    v_ref = o.postselect(o.hhl_circuit(b, n_s, pl), n_s, n_c)["v"]
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    u = uniform_draws(8000, seed_offset=7)
    counts = torch.empty(1 << n_s, dtype=torch.int64, device="cuda")
    plan.sample(st, torch.tensor(u, device="cuda"), counts)
    got = counts.cpu().numpy()
    ref = o.sample_counts(v_ref, u)
    assert got.sum() == 8000
    p = np.abs(v_ref) ** 2
    cdf = np.cumsum(p) / p.sum()
    margin = 1e-12 if prec == "c128" else 1e-4
    near = np.min(np.abs(u[:, None] - cdf[None, :]), axis=1) < margin
    assert np.abs(got - ref).sum() <= 2 * int(near.sum()), (int(near.sum()), np.abs(got - ref).sum())
    plan.sample(st, torch.empty(0, dtype=torch.float64, device="cuda"), counts)   # zero shots
    assert int(counts.abs().sum().item()) == 0
    # the GPU sampler on a state it did not compute: exact
    psi = np.zeros(2 << (n_s + n_c), dtype=np.complex128)
    vv = np.sqrt(np.arange(1, (1 << n_s) + 1, dtype=np.float64)) * np.exp(1j * np.arange(1 << n_s))
    psi[(1 << (n_s + n_c)):(1 << (n_s + n_c)) + (1 << n_s)] = vv
    st2 = torch.tensor(psi, dtype=st.dtype, device="cuda")
    plan.sample(st2, torch.tensor(u, device="cuda"), counts)
    vv_in = (vv.astype(np.complex64) if prec == "c64" else vv).astype(np.complex128)  # the stored amplitudes
    np.testing.assert_array_equal(counts.cpu().numpy(), o.sample_counts(vv_in, u))


@pytest.mark.parametrize("prec", ["c128", "c64", "c128-fp64pipe"])
@pytest.mark.parametrize("flow", ["poiseuille", "couette"])
def test_measure_and_dissipation_parity(hhl, monkeypatch, prec, flow):
    if prec == "c128-fp64pipe":
        monkeypatch.setenv("HHL_FP64_PIPE", "1")
        prec = "c128"
    n_s, n_c = 6, 7
    diag, off, b, walls = problem(flow, n_s)
    nu = 0.05
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    psi = o.hhl_circuit(b, n_s, pl)
    ref = o.postselect(psi, n_s, n_c)
    u_ref = o.velocity(ref["v"], np.linalg.norm(b), pl["C"], pl["lam_ub"])
    eps_ref = o.dissipation(u_ref, walls[0], walls[1], nu)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, nu=nu, walls=walls)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    m = plan.measure(st)
    tol = TOL[prec]
    assert m["p_success"] == pytest.approx(ref["p_success"], rel=1e-9 if prec == "c128" else 1e-4)
    assert m["p_anc1"] == pytest.approx(ref["p_anc1"], rel=1e-9 if prec == "c128" else 1e-4)
    assert m["b_norm"] == pytest.approx(np.linalg.norm(b), rel=1e-14)
    # norm of the whole buffer: 1 (the early mode keeps the rotated anc = 0 half)
    assert m["norm"] == pytest.approx(1.0, abs=1e-12 if prec == "c128" else 1e-5)
    # the postselected vector v (anc = 1, clock = 0 after the final Hadamards) at the amplitude
    # bound; xhat at the bound that implies
    v_got = _half(_np(st), n_s, n_c, 1)[0]
    v_ref = _half(psi, n_s, n_c, 1)[0]
    dv = np.abs(v_got - v_ref).max()
    assert dv <= tol
    np.testing.assert_allclose(m["xhat"], ref["xhat"], atol=xhat_bound(dv, np.linalg.norm(v_got), 1 << n_s))
    eps, u = plan.dissipation(st, want_u=True)
    np.testing.assert_allclose(u, u_ref, rtol=1e-9 if prec == "c128" else 2e-4,
                               atol=1e-12 * np.abs(u_ref).max())
    assert eps == pytest.approx(eps_ref, rel=1e-9 if prec == "c128" else 1e-3)


def test_complex_rhs_and_user_t0_per_unit(hhl):
    n_s, n_c = 5, 6
    diag, off = o.laplacian_tridiag(32)
    rng = np.random.default_rng(17)
    b = rng.random(32) + 1j * rng.standard_normal(32)
    pl = _oracle_plan(diag, off, n_c, "user", t0=1.7, conv="per_unit", C=0.05)
    ref = o.hhl_circuit(b, n_s, pl)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, "c128", t0_rule="user", t0=1.7, t0_convention="per_unit", C=0.05)
    st = plan.new_state()
    plan.prepare_rhs_host(b.real.copy(), st, b_im=b.imag.copy())
    plan.apply_circuit(st)
    np.testing.assert_allclose(_half(_np(st), n_s, n_c, 1), _half(ref, n_s, n_c, 1), atol=1e-10)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_dense_complex_hermitian(hhl, prec):
    n_s, n_c = 3, 5
    rng = np.random.default_rng(23)
    q = np.linalg.qr(rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)))[0]
    a = q @ np.diag(rng.uniform(1.0, 9.0, 8)) @ q.conj().T
    a = 0.5 * (a + a.conj().T)
    b = rng.random(8)
    pl = o.plan(a, n_c, t0_rule="range_fill")
    ref = o.hhl_circuit(b, n_s, pl)
    plan = hhl.HHLPlan(n_s, n_c, dense=a, precision=prec, full_uncompute=True)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    np.testing.assert_allclose(_np(st), ref, atol=TOL[prec])


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_dense_real_general_tridiagonal(hhl, prec):
    n_s, n_c = 4, 5
    rng = np.random.default_rng(5)
    diag = 4.0 + rng.random(16)
    off = -rng.random(15)
    b = rng.random(16)
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    ref = o.hhl_circuit(b, n_s, pl)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, full_uncompute=True)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    np.testing.assert_allclose(_np(st), ref, atol=TOL[prec])


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("full", [True, False])
@pytest.mark.parametrize("n_c", [1, 2])
def test_smallest_registers(hhl, prec, full, n_c):
    """n_s = 1 with one or two clock qubits: one system qubit (a 2 x 2 A, the narrowest row
    the kernels handle), both uncompute modes and precisions."""
    diag, off = np.array([3.0, 3.0]), np.array([-1.0])
    b = np.array([0.3, 0.8])
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    ref = o.hhl_circuit(b, 1, pl)
    plan = _gpu_plan(hhl, diag, off, 1, n_c, prec, full_uncompute=full)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    tol = 1e-12 if prec == "c128" else 1e-6
    got = _np(st)
    if full:
        np.testing.assert_allclose(got, ref, atol=tol)
    else:
        np.testing.assert_allclose(_half(got, 1, n_c, 1), _half(ref, 1, n_c, 1), atol=tol)
    m = plan.measure(st)
    want = o.postselect(ref, 1, n_c)
    assert m["p_success"] == pytest.approx(want["p_success"], abs=10 * tol)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n,lo,m", [(6, 0, 6), (10, 3, 5), (12, 0, 7), (14, 4, 10), (16, 2, 13), (9, 8, 1)])
def test_qft_register_blocks(hhl, prec, n, lo, m):
    import torch
    from synth_inputs import random_state
    psi = random_state(n, seed_offset=n * 100 + lo)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    for inverse in (False, True):
        st = torch.tensor(psi, dtype=dt, device="cuda")
        hhl.apply_qft(st, n, lo, m, inverse)
        ref = o.qft_register(psi, n, lo, m, inverse)
        np.testing.assert_allclose(_np(st), ref, atol=TOL[prec])


def _bitrev(n):
    idx = np.arange(1 << n)
    out = np.zeros_like(idx)
    for b in range(n):
        out |= ((idx >> b) & 1) << (n - 1 - b)
    return out


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("n,states,plain", [(9, 2, False), (13, 1, False), (16, 2, False), (18, 1, False),
                                            (21, 1, False), (13, 1, True), (16, 2, True)])
def test_qft_whole_register_parity(hhl, monkeypatch, prec, n, states, plain):
    """The Fig. 1c circuit's QFT on the whole register (low bits in one pass, the rest in
    split passes with the 2^n-point twiddles) against the oracle's gate-by-gate QFT (read in
    bit-reversed order), then the inverse QFT back to the input. ``plain``: the low bits by the
    register transform instead of the persistent low-bit kernel (HHL_LOWBITS_PLAIN)."""
    import torch
    if plain:
        monkeypatch.setenv("HHL_LOWBITS_PLAIN", "1")
    from synth_inputs import random_state
    psis = [random_state(n, seed_offset=500 + n * 10 + j) for j in range(states)]
    dt = torch.complex128 if prec == "c128" else torch.complex64
    st = torch.tensor(np.concatenate(psis), dtype=dt, device="cuda")
    hhl.qft_whole(st, n, states, 0)
    got = _np(st).reshape(states, 1 << n)
    rev = _bitrev(n)
    rel = 1e-4 if prec == "c64" else 1e-9  # of the largest amplitude (the state is normalised)
    for j, psi in enumerate(psis):
        ref = o.qft_register(psi, n, 0, n, False)
        np.testing.assert_allclose(got[j][rev], ref, atol=TOL[prec])
        assert np.abs(got[j][rev] - ref).max() <= rel * np.abs(ref).max()
    hhl.qft_whole(st, n, states, 1)
    back = _np(st).reshape(states, 1 << n)
    for j, psi in enumerate(psis):
        np.testing.assert_allclose(back[j], psi, atol=TOL[prec])
        assert np.abs(back[j] - psi).max() <= rel * np.abs(psi).max()


@pytest.mark.parametrize("prec", ["c128", "c64", "c128-fp64pipe"])
@pytest.mark.parametrize("dt,r_max", [(3.0, 0), (0.5, 40), (50.0, 7)])
def test_trotter_parity(hhl, monkeypatch, prec, dt, r_max):
    """Controlled Strang products (several passes, odd and even pass counts) against the
    oracle's gate-by-gate Trotter circuit; complex128 in double-float arithmetic (default) and
    on the FP64 pipe (HHL_FP64_PIPE=1)."""
    if prec == "c128-fp64pipe":
        monkeypatch.setenv("HHL_FP64_PIPE", "1")
        prec = "c128"
    n_s, n_c = 5, 4
    diag, off, b, walls = problem("poiseuille", n_s)
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    lub = pl["lam_ub"]
    tro = dict(diag=diag / lub, off=off / lub, dt=dt, r_max=r_max)
    ref = run_stages(b, n_s, pl, trotter=tro)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, expm="trotter", trotter_dt=dt, trotter_steps_max=r_max,
                     full_uncompute=True)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_stage("qpe_u", st)
    tol = TOL[prec]
    np.testing.assert_allclose(_np(st), ref["qpe_u"], atol=tol)
    for stage in ("clock_block", "uncompute_u", "final_h"):
        plan.apply_stage(stage, st)
    np.testing.assert_allclose(_np(st), ref["final_h"], atol=tol)


@pytest.mark.parametrize("prec,runs", [("c128", None), ("c64", None), ("c64", 3)])
@pytest.mark.parametrize("n_c,dt,r_max", [(9, 1.0e4, 0), (10, 400.0, 0)])
def test_trotter_grouped_clock_bits_parity(hhl, monkeypatch, prec, runs, n_c, dt, r_max):
    """Clock bits sharing one pass (up to 8 single-step bits, 17 layers for a row with all of
    them set; larger steps counts in smaller groups and windows), against the oracle's
    gate-by-gate controlled Strang products, the whole circuit in both uncompute modes
    (runs: a cap on the warps of a pass, so that each walks many rows)."""
    if runs is not None:
        monkeypatch.setenv("HHL_TROTTER_RUNS", str(runs))
    n_s = 5
    diag, off, b, walls = problem("couette", n_s)
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    lub = pl["lam_ub"]
    tro = dict(diag=diag / lub, off=off / lub, dt=dt, r_max=r_max)
    ref = run_stages(b, n_s, pl, trotter=tro)
    tol = TOL[prec]
    for full in (False, True):
        plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, expm="trotter", trotter_dt=dt, trotter_steps_max=r_max,
                         full_uncompute=full)
        st = plan.new_state()
        plan.prepare_rhs_host(b, st)
        plan.apply_stage("qpe_u", st)
        np.testing.assert_allclose(_np(st), ref["qpe_u"], atol=tol)
        for stage in ("clock_block", "uncompute_u", "final_h"):
            plan.apply_stage(stage, st)
        got = _np(st)
        np.testing.assert_allclose(_half(got, n_s, n_c, 1), _half(ref["final_h"], n_s, n_c, 1), atol=tol)
        if full:
            np.testing.assert_allclose(got, ref["final_h"], atol=tol)


@pytest.mark.parametrize("prec,runs", [("c128", None), ("c128", 7), ("c64", 1), ("c64", 5)])
def test_trotter_large_row_spans_many_tiles(hhl, monkeypatch, prec, runs):
    """A 2^13-point system row spans 18 warp windows with halos; checked against the
    oracle's gate-by-gate Strang products on the controlled rows. runs caps the warps of a
    pass, so that each walks a long run of windows across row ends (halos carried from one
    window to the next, side-buffer halos only where two runs meet)."""
    import torch
    if runs is not None:
        monkeypatch.setenv("HHL_TROTTER_RUNS", str(runs))
    n_s, n_c = 13, 2
    n = n_s + n_c + 1
    diag, off = o.laplacian_tridiag(1 << n_s)
    lub = 4.0 * ((1 << n_s) + 1) ** 2      # Gershgorin bound of tridiag(-1, 2, -1)/h^2
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, expm="trotter", trotter_dt=0.25, trotter_steps_max=0,
                     t0_rule="user", t0=8.0)
    from synth_inputs import random_state
    psi = random_state(n, seed_offset=77)
    st = torch.tensor(psi if prec == "c128" else psi.astype(np.complex64), device="cuda")
    plan.apply_stage("qpe_u", st)
    ref = psi.copy()
    anc0 = ref[: 1 << (n - 1)]          # the stage acts on the anc = 0 half only
    t_k = [8.0 * (1 << k) / 4 for k in range(n_c)]
    for k in range(n_c):
        r = o.trotter_steps(t_k[k], 0.25, 0)
        o.apply_trotter_controlled(anc0, n - 1, n_s, n_s + k, diag / lub, off / lub, t_k[k], r)
    np.testing.assert_allclose(_np(st), ref, atol=1e-10 if prec == "c128" else 1e-6)


def test_apply_circuit_equals_stages_and_counts_launches(hhl):
    n_s, n_c = 4, 6
    diag, off, b, walls = problem("poiseuille", n_s)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, "c64")
    s1, s2 = plan.new_state(), plan.new_state()
    plan.prepare_rhs_host(b, s1)
    plan.prepare_rhs_host(b, s2)
    before = hhl.kernel_launch_count()
    plan.apply_circuit(s1)
    launched = hhl.kernel_launch_count() - before
    assert launched >= 2 * n_c + 2
    for stage in ("qpe_u", "clock_block", "uncompute_u", "final_h"):
        plan.apply_stage(stage, s2)
    np.testing.assert_array_equal(_np(s1), _np(s2))


def test_invalid_state_calls_return_status(hhl):
    diag, off, b, walls = problem("poiseuille", 3)
    plan = _gpu_plan(hhl, diag, off, 3, 3, "c64")
    st = plan.new_state()
    plan.prepare_rhs_host(np.zeros(8), st)
    plan.apply_circuit(st)
    with pytest.raises(hhl.HHLError) as e:
        plan.measure(st)
    assert e.value.status == 3
    import ctypes
    assert plan._lib.hhl_apply_stage(plan._h, 9, ctypes.c_void_p(st.data_ptr()), None) == 1


# ----------------------------------------------------------------------------- full size


@pytest.fixture(scope="module")
def couette_1024_oracle():
    """The 23-qubit Couette workload (N = 1024, n_c = 12) through the FP64 oracle (~30 s)."""
    diag, off, b, walls = problem("couette", 10)
    pl = _oracle_plan(diag, off, 12, "range_fill")
    psi = o.hhl_circuit(b, 10, pl)
    return dict(psi=psi, pl=pl, b=b, diag=diag, off=off, walls=walls, post=o.postselect(psi, 10, 12))


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_couette_1024_full_size_parity(hhl, couette_1024_oracle, prec):
    ref = couette_1024_oracle
    plan = _gpu_plan(hhl, ref["diag"], ref["off"], 10, 12, prec, walls=ref["walls"])
    st = plan.new_state()
    plan.prepare_rhs_host(ref["b"], st)
    plan.apply_circuit(st)
    got = _np(st)
    np.testing.assert_allclose(_half(got, 10, 12, 1), _half(ref["psi"], 10, 12, 1), atol=TOL[prec])
    m = plan.measure(st)
    v_got = _half(got, 10, 12, 1)[0]
    dv = np.abs(v_got - _half(ref["psi"], 10, 12, 1)[0]).max()
    np.testing.assert_allclose(m["xhat"], ref["post"]["xhat"], atol=xhat_bound(dv, np.linalg.norm(v_got), 1024))
    assert m["p_success"] == pytest.approx(ref["post"]["p_success"], rel=1e-8 if prec == "c128" else 1e-4)


@pytest.mark.slow
def test_couette_1024_c64_fidelity_against_c128(hhl, couette_1024_oracle):
    """Fidelity of the complex64 postselected solution against the complex128 one."""
    ref = couette_1024_oracle
    xs = {}
    for prec in ("c128", "c64"):
        plan = _gpu_plan(hhl, ref["diag"], ref["off"], 10, 12, prec)
        st = plan.new_state()
        plan.prepare_rhs_host(ref["b"], st)
        plan.apply_circuit(st)
        xs[prec] = plan.measure(st)["xhat"]
    f = abs(np.vdot(xs["c128"], xs["c64"]))
    assert f >= 1 - 1e-6


# ----------------------------------------------------------------------------- tcgen05 GEMM


@pytest.mark.parametrize("n_s,n_c,bn", [(7, 8, None), (8, 9, None), (9, 10, None), (8, 9, "128"), (9, 10, "128")])
def test_tcgen05_gemm_parity(hhl, monkeypatch, n_s, n_c, bn):
    """Split-FP16 tcgen05 controlled-U GEMMs (1 to 4 tiles in each direction) against the
    oracle, stage by stage, complex64 tolerance; ``bn``: 128-column tiles (HHL_TC_BN)."""
    if bn is not None:
        monkeypatch.setenv("HHL_TC_BN", bn)
    diag, off, b, walls = problem("couette", n_s)
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    ref = run_stages(b, n_s, pl)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, "c64", gemm="tcgen05")
    assert plan.info["gemm_impl"] == 2
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_stage("qpe_u", st)
    np.testing.assert_allclose(_np(st), ref["qpe_u"], atol=1e-5)
    for stage in ("clock_block", "uncompute_u", "final_h"):
        plan.apply_stage(stage, st)
    np.testing.assert_allclose(_half(_np(st), n_s, n_c, 1), _half(ref["final_h"], n_s, n_c, 1), atol=1e-5)
    m = plan.measure(st)
    # The tensor-core accumulation is not round-to-nearest: over 2 n_c controlled products
    # the norm shrinks by ~1e-5 (measured), inside the element-wise 1e-5 bound checked above.
    assert m["norm"] == pytest.approx(1.0, abs=1e-4)


def test_tcgen05_matches_simt_gemm(hhl):
    """The tensor-core and CUDA-core GEMM paths agree to FP32 accuracy on a random state."""
    import torch
    from synth_inputs import random_state
    n_s, n_c = 8, 9
    diag, off, b, walls = problem("poiseuille", n_s)
    psi = random_state(n_s + n_c + 1, seed_offset=5)
    outs = []
    for gemm in ("simt", "tcgen05"):
        plan = _gpu_plan(hhl, diag, off, n_s, n_c, "c64", gemm=gemm)
        st = torch.tensor(psi, dtype=torch.complex64, device="cuda")
        plan.apply_stage("qpe_u", st)
        outs.append(_np(st))
    assert np.abs(outs[0] - outs[1]).max() < 5e-6


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_poiseuille_2p18_trotter_full_size_sampled_rows(hhl, prec):
    """The 32-qubit Poiseuille workload (N = 2^18, n_c = 13, Strang-Trotter U_k, the bench's
    step bounds; complex64 as benched, complex128 the 64 GiB maximum). After the controlled
    products, clock row 0 still holds bhat / 2^(n_c/2) and clock row 2^k holds
    U_k bhat / 2^(n_c/2); the oracle computes each sampled U_k bhat with its own gate sequence
    on one system vector."""
    import torch
    from synth_inputs import rhs
    n_s, n_c = 18, 13
    N, R = 1 << n_s, 1 << n_c
    diag, off = o.laplacian_tridiag(N)
    b = rhs("poiseuille", N)
    dt, r_max = 1024.0, 8
    # Bounds on the sampled U_k rows (relative to the row's largest amplitude: the amplitudes
    # are ~2e-5 here, so an absolute 1e-5 would pin nothing) and on transformed columns (per unit
    # of their largest input amplitude); complex128 keeps its absolute 1e-10 as well.
    row_abs, row_rel, col = (None, TOL["c64"], TOL["c64"]) if prec == "c64" else (1e-10, 1e-9, 1e-10)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, expm="trotter", trotter_dt=dt, trotter_steps_max=r_max)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_stage("qpe_u", st)
    torch.cuda.synchronize()
    lub = 4.0 * (N + 1) ** 2
    t0 = o.t0_total("range_fill", n_c)
    assert plan.info["t0"] == pytest.approx(t0, rel=1e-12)
    bhat = b / np.linalg.norm(b) / math.sqrt(R)
    np.testing.assert_allclose(_np(st[:N]), bhat, rtol=1e-6 if prec == "c64" else 1e-13, atol=0)
    for k in (0, 4, 9, 11, 12):
        t_k = t0 * (1 << k) / R
        r = o.trotter_steps(t_k, dt, r_max)
        psi = np.zeros(2 * N, dtype=np.complex128)
        psi[N:] = bhat
        o.apply_trotter_controlled(psi, n_s + 1, n_s, n_s, diag / lub, off / lub, t_k, r)
        got = _np(st[(1 << k) * N:((1 << k) + 1) * N])
        ref = psi[N:]
        if row_abs is not None:
            assert np.abs(got - ref).max() <= row_abs
        assert np.abs(got - ref).max() <= row_rel * np.abs(ref).max(), k
    out = torch.empty(4 + 2 * N, dtype=torch.float64, device="cuda")
    plan.measure_async(st, out)          # p_success is 0 before the inversion: read the norm only
    assert out[2].item() == pytest.approx(1.0, abs=TOL[prec])
    # The clock block and the Hadamard layer at full size (split register passes) on a seeded
    # random state: every system column j is transformed on its own, so the oracle checks
    # sampled columns one by one.
    g = torch.Generator(device="cuda")
    g.manual_seed(20230701)
    view = st.view(2, R, N)
    torch.view_as_real(view[0]).normal_(generator=g)
    cols = [0, 1, 77, N // 2 + 5, N - 1]
    before = [_np(view[0, :, j]) for j in cols]
    plan.apply_stage("clock_block", st)
    theta = o.rotation_angles(n_c, t0)
    for j, x in zip(cols, before):
        psi = np.zeros(2 * R, dtype=np.complex128)
        psi[:R] = x
        o.qft(psi, n_c + 1, 0, n_c, inverse=True)
        o.apply_clock_controlled_ry(psi, 0, n_c, theta)
        rotated0 = psi[:R].copy()
        o.qft(psi, n_c + 1, 0, n_c, inverse=False)
        scale = np.abs(x).max()
        assert np.abs(_np(view[0, :, j]) - rotated0).max() <= col * scale, j
        assert np.abs(_np(view[1, :, j]) - psi[R:]).max() <= col * scale, j
    torch.view_as_real(view[1]).normal_(generator=g)
    before1 = [_np(view[1, :, j]) for j in cols]
    plan.apply_stage("final_h", st)
    for j, x in zip(cols, before1):
        psi = x.copy()
        for q in range(n_c):
            o.apply_1q(psi, n_c, q, o.H_GATE)
        assert np.abs(_np(view[1, :, j]) - psi).max() <= col * np.abs(x).max(), j
    del st
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_poiseuille_34_qubits_maximum_register(hhl):
    """The largest register a plan accepts: n_s = 20, n_c = 13, one ancilla (34 qubits, a
    128 GiB complex64 state). The controlled Strang products on sampled clock rows and the
    clock block on sampled system columns against the oracle, and the norm after the whole
    circuit; one qubit more is refused."""
    import torch
    from synth_inputs import rhs
    n_s, n_c = 20, 13
    N, R = 1 << n_s, 1 << n_c
    diag, off = o.laplacian_tridiag(N)
    b = rhs("poiseuille", N)
    dt, r_max = 1024.0, 8
    with pytest.raises(hhl.HHLError):
        _gpu_plan(hhl, *o.laplacian_tridiag(2 * N), n_s + 1, n_c, "c64", expm="trotter", trotter_dt=dt,
                  trotter_steps_max=r_max)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, "c64", expm="trotter", trotter_dt=dt, trotter_steps_max=r_max)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_stage("qpe_u", st)
    lub = 4.0 * (N + 1) ** 2
    t0 = o.t0_total("range_fill", n_c)
    bhat = b / np.linalg.norm(b) / math.sqrt(R)
    for k in (0, 10, 12):
        t_k = t0 * (1 << k) / R
        psi = np.zeros(2 * N, dtype=np.complex128)
        psi[N:] = bhat
        o.apply_trotter_controlled(psi, n_s + 1, n_s, n_s, diag / lub, off / lub, t_k, o.trotter_steps(t_k, dt, r_max))
        got = _np(st[(1 << k) * N:((1 << k) + 1) * N])
        assert np.abs(got - psi[N:]).max() <= TOL["c64"] * np.abs(psi[N:]).max(), k
    g = torch.Generator(device="cuda")
    g.manual_seed(20230702)
    view = st.view(2, R, N)
    torch.view_as_real(view[0]).normal_(generator=g)
    cols = [0, 12345, N - 1]
    before = [_np(view[0, :, j]) for j in cols]
    plan.apply_stage("clock_block", st)
    theta = o.rotation_angles(n_c, t0)
    for j, x in zip(cols, before):
        psi = np.zeros(2 * R, dtype=np.complex128)
        psi[:R] = x
        o.qft(psi, n_c + 1, 0, n_c, inverse=True)
        o.apply_clock_controlled_ry(psi, 0, n_c, theta)
        o.qft(psi, n_c + 1, 0, n_c, inverse=False)
        assert np.abs(_np(view[1, :, j]) - psi[R:]).max() <= TOL["c64"] * np.abs(x).max(), j
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    out = torch.empty(4 + 2 * N, dtype=torch.float64, device="cuda")
    plan.measure_async(st, out)
    assert out[2].item() == pytest.approx(1.0, abs=TOL["c64"])
    assert 0.0 < out[0].item() <= out[1].item() <= 1.0
    del st, view
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("flow,n_s,n_c", [("couette", 4, 8), ("poiseuille", 5, 9), ("couette", 6, 11),
                                          ("poiseuille", 4, 13)])
def test_cluster_clock_block_parity(hhl, monkeypatch, prec, flow, n_s, n_c):
    """The one-pass clustered clock block and Hadamard layer (the path of large states),
    forced on small states, against the oracle stage by stage; postselect-early mode."""
    import torch
    monkeypatch.setenv("HHL_CLOCK_CLUSTER", "1")
    diag, off, b, walls = problem(flow, n_s)
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    ref = run_stages(b, n_s, pl)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, gemm="simt")
    st = plan.new_state()
    plan.prepare_rhs(_b_dev(b), st)
    plan.apply_stage("qpe_u", st)
    tol = TOL[prec]
    hhl.profile_reset()
    hhl.profile_enable(True)
    try:
        plan.apply_stage("clock_block", st)
        got = _np(st)
        np.testing.assert_allclose(_half(got, n_s, n_c, 1), _half(ref["clock_block"], n_s, n_c, 1), atol=tol)
        np.testing.assert_allclose(_half(got, n_s, n_c, 0), _half(ref["rotated"], n_s, n_c, 0), atol=tol)
        plan.apply_stage("uncompute_u", st)
        plan.apply_stage("final_h", st)
        got = _np(st)
        np.testing.assert_allclose(_half(got, n_s, n_c, 1), _half(ref["final_h"], n_s, n_c, 1), atol=tol)
        torch.cuda.synchronize()
        prof = hhl.profile_read()
    finally:
        hhl.profile_enable(False)
    assert prof["k_clock_cluster"][0] == 1 and prof["k_hadamard_cluster"][0] == 1


@pytest.mark.parametrize("prec,group", [("c128", None), ("c128-fp64pipe", None), ("c64", None), ("c64", "8,64"),
                                        ("c64", "2,1"), ("c64", "16,1"), ("c64", "4,1"), ("c64", "1,1")])
@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("flow,n_s,n_c", [("couette", 5, 8), ("poiseuille", 6, 9), ("couette", 7, 11),
                                          ("poiseuille", 6, 12), ("couette", 5, 13)])
def test_split_register_passes_parity(hhl, monkeypatch, prec, group, full, flow, n_s, n_c):
    """The clock block and the Hadamard layer as split register passes (the path large states
    take), forced on small states, stage by stage against the oracle: streaming passes
    (group None) or L2-staged group passes with G CTAs per cluster and an L2 budget in MiB
    ("G,MiB": a budget of 1 MiB leaves fewer clusters than column blocks, so each cluster
    runs several groups); complex128 in double-float arithmetic (default) and on the FP64 pipe."""
    import torch
    if prec == "c128-fp64pipe":
        monkeypatch.setenv("HHL_FP64_PIPE", "1")
        prec = "c128"
    monkeypatch.setenv("HHL_FFT_SPLIT", "1")
    monkeypatch.setenv("HHL_CLOCK_CLUSTER", "0")
    monkeypatch.setenv("HHL_GROUP", "0" if group is None else "1")
    if group is not None:
        monkeypatch.setenv("HHL_GROUP_SHAPE", group)
    diag, off, b, walls = problem(flow, n_s)
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    ref = run_stages(b, n_s, pl)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, full_uncompute=full, gemm="simt")
    st = plan.new_state()
    plan.prepare_rhs(_b_dev(b), st)
    plan.apply_stage("qpe_u", st)
    tol = TOL[prec]
    hhl.profile_reset()
    hhl.profile_enable(True)
    try:
        plan.apply_stage("clock_block", st)
        got = _np(st)
        np.testing.assert_allclose(_half(got, n_s, n_c, 1), _half(ref["clock_block"], n_s, n_c, 1), atol=tol)
        anc0_ref = ref["clock_block"] if full else ref["rotated"]
        np.testing.assert_allclose(_half(got, n_s, n_c, 0), _half(anc0_ref, n_s, n_c, 0), atol=tol)
        plan.apply_stage("uncompute_u", st)
        plan.apply_stage("final_h", st)
        got = _np(st)
        np.testing.assert_allclose(_half(got, n_s, n_c, 1), _half(ref["final_h"], n_s, n_c, 1), atol=tol)
        if full:
            np.testing.assert_allclose(got, ref["final_h"], atol=tol)
        torch.cuda.synchronize()
        prof = hhl.profile_read()
    finally:
        hhl.profile_enable(False)
    if group is None:
        assert all(prof[f"k_clock_pass_{x}"][0] == 1 for x in "abc") and "k_clock_block" not in prof
        assert prof["k_hadamard_pass"][0] == 2 and "k_register_transform" not in prof
    else:
        assert prof["k_clock_group"][0] == 1 and prof["k_hadamard_group"][0] == 1
        assert not any(k.startswith(("k_clock_pass", "k_hadamard_pass", "k_register_transform")) for k in prof)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("shape", ["1,0", "2,1", "4,2", "2,3"])
@pytest.mark.parametrize("flow,n_s,n_c", [("couette", 5, 8), ("poiseuille", 6, 10)])
def test_clock_block_cluster_shapes(hhl, monkeypatch, prec, shape, flow, n_s, n_c):
    """The one-pass clock block and Hadamard layer of L2-resident states with the block width
    and cluster size forced ("W,cb": W columns per block, 2^cb CTAs per cluster; a shape that
    does not fit falls back to the default), stage by stage against the oracle."""
    import torch
    monkeypatch.setenv("HHL_FFT_SPLIT", "0")
    monkeypatch.setenv("HHL_CLOCK_CLUSTER", "0")
    monkeypatch.setenv("HHL_FFT_SHAPE", shape)
    diag, off, b, walls = problem(flow, n_s)
    pl = _oracle_plan(diag, off, n_c, "range_fill")
    ref = run_stages(b, n_s, pl)
    plan = _gpu_plan(hhl, diag, off, n_s, n_c, prec, gemm="simt")
    st = plan.new_state()
    plan.prepare_rhs(_b_dev(b), st)
    plan.apply_stage("qpe_u", st)
    tol = TOL[prec]
    hhl.profile_reset()
    hhl.profile_enable(True)
    try:
        plan.apply_stage("clock_block", st)
        got = _np(st)
        np.testing.assert_allclose(_half(got, n_s, n_c, 1), _half(ref["clock_block"], n_s, n_c, 1), atol=tol)
        np.testing.assert_allclose(_half(got, n_s, n_c, 0), _half(ref["rotated"], n_s, n_c, 0), atol=tol)
        plan.apply_stage("uncompute_u", st)
        plan.apply_stage("final_h", st)
        np.testing.assert_allclose(_half(_np(st), n_s, n_c, 1), _half(ref["final_h"], n_s, n_c, 1), atol=tol)
        torch.cuda.synchronize()
        prof = hhl.profile_read()
    finally:
        hhl.profile_enable(False)
    assert prof["k_clock_block"][0] == 1 and not any(k.startswith("k_clock_pass") for k in prof)


@pytest.mark.slow
def test_qft_whole_register_32_qubits_on_a_fourier_mode(hhl):
    """The Fig. 1c transform at full size (32 qubits, complex64, the bench's launches): the
    QFT of the Fourier mode psi_x = e^{-2 pi i x k0 / 2^32} / 2^16 is |k0> exactly (closed
    form), read at bit-reversed position; the inverse QFT restores the mode (sampled)."""
    import torch
    n, k0 = 32, 123456789
    L = 1 << n
    st = torch.empty(L, dtype=torch.complex64, device="cuda")
    chunk = 1 << 28
    for c0 in range(0, L, chunk):   # the mode in chunks (FP64 phase, exact mod 2^32)
        x = torch.arange(c0, c0 + chunk, dtype=torch.int64, device="cuda")
        ph = ((x * k0) % L).to(torch.float64) * (-2.0 * math.pi / L)
        st[c0:c0 + chunk] = (torch.polar(torch.ones_like(ph), ph) / 65536.0).to(torch.complex64)
        del x, ph
    probe = torch.tensor([0, 1, 77, L // 3, L - 1], device="cuda")
    before = _np(st[probe])
    hhl.qft_whole(st, n, 1, 0)
    rev = int(format(k0, "032b")[::-1], 2)
    assert abs(_np(st[rev:rev + 1])[0] - 1.0) < 2e-3
    others = torch.randint(0, L, (4096,), device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    others = others[others != rev]
    assert np.abs(_np(st[others])).max() < 2e-3
    hhl.qft_whole(st, n, 1, 1)
    np.testing.assert_allclose(_np(st[probe]), before, atol=2e-7)
    del st
    torch.cuda.empty_cache()
