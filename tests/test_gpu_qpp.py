"""GPU parity of the LCU post-processing of the dissipation rate (App. D, QPP): against the
direct read-out of the same state (hhl_dissipation, Sec. VII), against the oracle's circuit
on the GPU's own velocity field (probability p0), and against the oracle's whole pipeline."""
import numpy as np
import pytest

from oracle import hhl_oracle as o
from oracle import qpp_oracle as q
from tests.oracle_stages import problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hhl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2307_00391_gb300 as pkg
    pkg.load()
    return pkg


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("flow,n_s,n_c", [("poiseuille", 4, 8), ("couette", 5, 9), ("couette", 7, 8)])
def test_qpp_dissipation(hhl, prec, flow, n_s, n_c):
    diag, off, b, walls = problem(flow, n_s)
    nu = 0.1
    plan = hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision=prec, nu=nu, walls=walls)
    st = plan.new_state()
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    eps_direct, u = plan.dissipation(st, want_u=True)
    eps_qpp, p0 = plan.qpp_dissipation(st)
    # the same field, read two ways: equal to FP64 rounding
    assert eps_qpp == pytest.approx(eps_direct, rel=1e-10)
    # the circuit's probability against the oracle's circuit on this field
    w = q.lcu_register(u, walls[0], walls[1])
    assert p0 == pytest.approx(q.lcu_probability(w), rel=1e-10)
    # and against the oracle's whole pipeline (HHL circuit, then its LCU circuit)
    pl = o.plan(o.dense_from_tridiag(diag, off), n_c)
    psi = o.hhl_circuit(b, n_s, pl)
    v = o.postselect(psi, n_s, n_c)["v"]
    u_ref = o.velocity(v, np.linalg.norm(b), pl["C"], pl["lam_ub"])
    eps_ref, _ = q.qpp_dissipation(u_ref, walls[0], walls[1], nu)
    assert eps_qpp == pytest.approx(eps_ref, rel=1e-8 if prec == "c128" else 2e-3)
    # a second call reuses the plan's register
    assert plan.qpp_dissipation(st)[0] == pytest.approx(eps_qpp, rel=1e-14)
