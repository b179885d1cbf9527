"""The learned T0 predictor: GPU forward / backward kernels against the FP64 oracle, training,
and the gain of the trained network over the power-law rule, judged by full simulations."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2307_00391_gb300 as p
    p.load()
    return p


def _bf16_weights(params):
    """Round W1, W2, W3 to bfloat16 (as the kernels read them); biases stay FP32."""
    import torch
    from oracle import mlp_oracle as m
    d = m.unpack(params.astype(np.float64))
    for name in ("W1", "W2", "W3"):
        d[name] = torch.tensor(d[name], dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    for name in ("b1", "b2", "b3"):
        d[name] = d[name].astype(np.float32).astype(np.float64)
    return m.pack(d)


def test_mlp_forward_and_gradients_match_oracle(pkg):
    import torch
    from oracle import mlp_oracle as m
    from paper_2307_00391_gb300.t0_model import T0Net
    rng = np.random.default_rng(3)
    params = T0Net.init_params(5) + rng.normal(0, 0.05, T0Net.N_PARAMS).astype(np.float32)
    net = T0Net(params)
    x = rng.standard_normal((100, 6)).astype(np.float32)   # 100 rows: a ragged last CTA
    t = rng.standard_normal((100, 2)).astype(np.float32)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    y = torch.empty((100, 2), device="cuda")
    net.forward_dev(xd, y)
    pref = _bf16_weights(params)
    y_ref, _ = m.forward(pref, x.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), y_ref, atol=2e-5, rtol=2e-5)
    g = torch.empty(T0Net.N_PARAMS, device="cuda")
    loss = torch.empty(1, device="cuda")
    net.gradients_dev(xd, td, g, loss)
    l_ref, g_ref = m.loss_and_grad(pref, x.astype(np.float64), t.astype(np.float64))
    assert loss.item() == pytest.approx(l_ref, rel=1e-5)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g_ref) <= 1e-5 * np.linalg.norm(g_ref)
    np.testing.assert_allclose(gg, g_ref, atol=1e-6 * np.abs(g_ref).max() + 1e-9)
    net.close()


def test_mlp_training_reduces_loss(pkg):
    from paper_2307_00391_gb300.t0_model import T0Net
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, (2048, 6))
    Y = np.stack([np.sin(2 * X[:, 0]) + X[:, 1] ** 2, X[:, 2] * X[:, 3] - 0.5 * X[:, 4]], axis=1)
    net = T0Net(seed=1)
    hist = net.fit(X, Y, steps=800, batch=256, lr=3e-3)
    assert hist[-1] < 0.1 * hist[0], hist
    err = net.predict(X[:256]) - Y[:256]
    assert np.sqrt(np.mean(err ** 2)) < 0.15
    net.close()


def test_learned_t0_beats_power_law_on_held_out_problems(pkg):
    """Sweeps from the batched engine train the network; on held-out problems the predicted
    T0 gives a higher postselected-solution fidelity than the power-law T0 (both judged by a
    full simulation; two of them re-checked by the FP64 oracle)."""
    from oracle import hhl_oracle as o
    from paper_2307_00391_gb300 import t0_model as tm
    problems = tm.sweep_problems(42, seed=11, ns_range=(3, 6))
    ncs = (4, 5, 6)
    sweep = tm.run_sweep(problems, n_clocks=ncs)
    train, held = problems[:34], problems[34:]
    sw_train = dict(F=sweep["F"][:34], scales=sweep["scales"], n_clocks=sweep["n_clocks"])
    X, Y, _ = tm.training_set(train, sw_train)
    net = tm.T0Net(seed=2)
    net.fit(X, Y, steps=1500, batch=128, lr=2e-3)
    # held-out: predicted scale vs the power law (scale 1), both simulated
    rows, specs = [], []
    for p, pr in enumerate(held):
        for nc in ncs:
            rows.append(tm.features(pr["diag"], pr["off"], pr["N"], nc, pr["flow"]))
            specs.append((p, nc))
    pred = net.predict(np.array(rows))
    scales_pred = np.exp(pred[:, 0])
    probs, bs = [], []
    for (p, nc), s in zip(specs, scales_pred):
        pr = held[p]
        for scale in (float(s), 1.0):
            probs.append(dict(n_sys_qubits=pr["n_s"], n_clock=nc, diag=np.full(pr["N"], pr["diag"]),
                              off=np.full(pr["N"] - 1, pr["off"]), t0_rule="power_law", t0_scale=scale))
            bs.append(pr["b"])
    batch = pkg.HHLBatch(probs)
    out, _ = batch.run_host(batch.pack_rhs(bs))
    res = batch.unpack(out)
    f_pred, f_pl = [], []
    for j, (p, nc) in enumerate(specs):
        xc = tm._classical(held[p])
        f_pred.append(abs(np.vdot(xc, res[2 * j]["xhat"])))
        f_pl.append(abs(np.vdot(xc, res[2 * j + 1]["xhat"])))
    f_pred, f_pl = np.array(f_pred), np.array(f_pl)
    assert f_pred.mean() > f_pl.mean() + 0.01, (f_pred.mean(), f_pl.mean())
    # FP64 oracle re-check of the judged fidelity for two small held-out cases
    for j in [k for k, (p, nc) in enumerate(specs) if held[p]["n_s"] <= 4][:2]:
        p, nc = specs[j]
        pr = held[p]
        a = o.dense_from_tridiag(np.full(pr["N"], pr["diag"]), np.full(pr["N"] - 1, pr["off"]))
        t0 = o.t0_total("power_law", nc, kappa=o.condition_number(a)) * float(scales_pred[j])
        pl = o.plan(a, nc, t0_rule="user", t0=t0)
        post = o.postselect(o.hhl_circuit(pr["b"], pr["n_s"], pl), pr["n_s"], nc)
        f_oracle = o.fidelity(post["v"], np.linalg.solve(a, pr["b"]))
        assert f_oracle == pytest.approx(f_pred[j], abs=1e-4)
    net.close()
