"""The batched engine (one CUDA graph over uneven instances) against the FP64 oracle and
against the single-plan path, instance by instance."""
import math

import numpy as np
import pytest

from oracle import hhl_oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hhl():
    import torch
    assert torch.cuda.is_available()
    import paper_2307_00391_gb300 as pkg
    pkg.load()
    return pkg


def _instances(specs, seed=0):
    """specs: (n_s, n_c, flow, t0_scale, gemm)."""
    from synth_inputs import rhs
    rng = np.random.default_rng(seed)
    probs, bs, choice = [], [], []
    for n_s, n_c, flow, scale, gemm in specs:
        n = 1 << n_s
        diag, off = o.laplacian_tridiag(n)
        probs.append(dict(n_sys_qubits=n_s, n_clock=n_c, diag=diag, off=off, nu=0.05,
                          walls=(0.0, 1.0) if flow == "couette" else (0.0, 0.0), t0_rule="power_law",
                          t0_scale=scale))
        b = rng.random(n) if flow == "random" else rhs("couette" if flow == "couette" else "poiseuille", n)
        bs.append(b)
        choice.append(gemm)
    return probs, bs, choice


SPECS = [(4, 5, "poiseuille", 1.0, 0), (6, 8, "random", 3.0, 128), (7, 8, "couette", 0.5, 256),
         (5, 7, "random", 1.0, 0), (8, 9, "random", 2.0, 256), (6, 9, "poiseuille", 0.2, 0),
         (7, 9, "random", 8.0, 128), (3, 6, "couette", 1.0, 0)]


def _check_v_and_xhat(got, post, n, tol=1e-5):
    """The postselected vector v = xhat sqrt(p_success) at the complex64 amplitude bound, and
    xhat at the bound that implies, (1 + sqrt(n)) max|dv| / |v|."""
    v_got = got["xhat"] * math.sqrt(got["p_success"])
    v_ref = post["xhat"] * math.sqrt(post["p_success"])
    dv = np.abs(v_got - v_ref).max()
    assert dv <= tol, dv
    bound = (1.0 + math.sqrt(n)) * dv / (np.linalg.norm(v_got) - math.sqrt(n) * dv) + 1e-13
    np.testing.assert_allclose(got["xhat"], post["xhat"], atol=bound)


def _oracle_instance(pr, b):
    n_s, n_c = pr["n_sys_qubits"], pr["n_clock"]
    a = o.dense_from_tridiag(pr["diag"], pr["off"])
    t0 = o.t0_total("power_law", n_c, kappa=o.condition_number(a)) * pr["t0_scale"]
    pl = o.plan(a, n_c, t0_rule="user", t0=t0)
    post = o.postselect(o.hhl_circuit(b, n_s, pl), n_s, n_c)
    u = o.velocity(post["v"], np.linalg.norm(b), pl["C"], pl["lam_ub"])
    eps = o.dissipation(u, pr["walls"][0], pr["walls"][1], pr["nu"])
    return post, eps, t0


def test_batch_matches_oracle_per_instance_and_replays(hhl):
    import torch
    probs, bs, choice = _instances(SPECS)
    batch = hhl.HHLBatch(probs, gemm_choice=choice, streams=3)
    assert [inst["gemm"] for inst in batch.instances] == choice
    inf = batch.info
    b_dev = torch.tensor(batch.pack_rhs(bs), device="cuda")
    out = torch.empty(inf["out_doubles"], dtype=torch.float64, device="cuda")
    eps = torch.empty(batch.count, dtype=torch.float64, device="cuda")
    batch.run(b_dev, out, eps)
    torch.cuda.synchronize()
    assert batch.info["graph_launches"] > 0
    res = batch.unpack(out.cpu().numpy())
    eps_h = eps.cpu().numpy()
    for i, (pr, b) in enumerate(zip(probs, bs)):
        post, eps_ref, t0 = _oracle_instance(pr, b)
        assert batch.instances[i]["t0"] == pytest.approx(t0, rel=1e-12)
        assert res[i]["p_success"] == pytest.approx(post["p_success"], rel=2e-4), i
        _check_v_and_xhat(res[i], post, 1 << pr["n_sys_qubits"])
        assert res[i]["norm"] == pytest.approx(1.0, abs=1e-4)
        assert eps_h[i] == pytest.approx(eps_ref, rel=2e-3), i
    # replay with other right-hand sides
    rng = np.random.default_rng(7)
    bs2 = [rng.random(len(b)) + 0.1 for b in bs]
    b_dev.copy_(torch.tensor(batch.pack_rhs(bs2)))
    batch.run(b_dev, out, eps)
    torch.cuda.synchronize()
    res2 = batch.unpack(out.cpu().numpy())
    for i in (0, 2, 4, 6):
        post, _, _ = _oracle_instance(probs[i], bs2[i])
        _check_v_and_xhat(res2[i], post, 1 << probs[i]["n_sys_qubits"])


def test_batch_equals_single_plan_path(hhl):
    """Every instance of the graph gives the single-plan result (same kernels, just-in-time U_k)."""
    import torch
    probs, bs, choice = _instances(SPECS, seed=3)
    batch = hhl.HHLBatch(probs, gemm_choice=choice, streams=4)
    out, eps = batch.run_host(batch.pack_rhs(bs))
    res = batch.unpack(out)
    for i, (pr, b) in enumerate(zip(probs, bs)):
        a = o.dense_from_tridiag(pr["diag"], pr["off"])
        t0 = o.t0_total("power_law", pr["n_clock"], kappa=o.condition_number(a)) * pr["t0_scale"]
        plan = hhl.HHLPlan(pr["n_sys_qubits"], pr["n_clock"], diag=pr["diag"], off=pr["off"], precision="c64",
                           t0_rule="user", t0=t0, gemm="simt", nu=pr["nu"], walls=pr["walls"])
        st = plan.new_state()
        plan.prepare_rhs_host(b, st)
        plan.apply_circuit(st)
        m = plan.measure(st)
        f = abs(np.vdot(m["xhat"], res[i]["xhat"]))
        assert f > 1 - 1e-6, (i, f)   # the two paths build U_k differently (eigenvectors / g_k), both FP64
        assert res[i]["p_success"] == pytest.approx(m["p_success"], rel=1e-3)
        plan.close()


def test_batch_rejects_unsupported_instances(hhl):
    n = 8
    diag = np.arange(1.0, n + 1) + 4.0
    off = -np.ones(n - 1)
    with pytest.raises(hhl.HHLError) as e:
        hhl.HHLBatch([dict(n_sys_qubits=3, n_clock=4, diag=diag, off=off)])
    assert e.value.status == 8


@pytest.mark.slow
def test_full_batch_of_256_in_the_bench_configuration(hhl):
    """The 256 uneven instances exactly as the bench runs them (autotuned GEMM choices, 8
    worker streams, one graph): sampled instances with n_s <= 7 against the FP64 oracle one by
    one, every instance against the invariants (unit norm, 0 < p_success <= p_anc1 <= 1)."""
    import torch
    from paper_2307_00391_gb300 import autotune
    from synth_inputs import batch_instances, walls
    inst = batch_instances(256)
    probs = []
    for it in inst:
        diag, off = hhl.laplacian(1 << it["n_s"])
        probs.append(dict(n_sys_qubits=it["n_s"], n_clock=it["n_c"], diag=diag, off=off, nu=0.1,
                          walls=walls(it["flow"]), t0_rule="power_law", t0_scale=it["t0_mult"]))
    choices = autotune.choices_for([(it["n_s"], it["n_c"]) for it in inst])
    batch = hhl.HHLBatch(probs, gemm_choice=choices, streams=8)
    out, eps = batch.run_host(batch.pack_rhs([it["b"] for it in inst]))
    res = batch.unpack(out)
    for i, r in enumerate(res):
        assert r["norm"] == pytest.approx(1.0, abs=2e-4), i
        assert 0.0 < r["p_success"] <= r["p_anc1"] + 1e-9 <= 1.0 + 1e-6, i
        assert np.isfinite(eps[i])
    small = [i for i, it in enumerate(inst) if it["n_s"] <= 7][:6]
    assert len(small) >= 3
    for i in small:
        it, pr = inst[i], probs[i]
        a = o.dense_from_tridiag(pr["diag"], pr["off"])
        t0 = o.t0_total("power_law", it["n_c"], kappa=o.condition_number(a)) * it["t0_mult"]
        pl = o.plan(a, it["n_c"], t0_rule="user", t0=t0)
        post = o.postselect(o.hhl_circuit(it["b"], it["n_s"], pl), it["n_s"], it["n_c"])
        assert res[i]["p_success"] == pytest.approx(post["p_success"], rel=1e-3), i
        assert abs(np.vdot(post["xhat"], res[i]["xhat"])) > 1 - 1e-6, i
    batch.close()
