"""Learned choice of the Hamiltonian-simulation time T0 and of the clock count.

Sec. VI fits the optimal T0* to kappa from sweeps of (T0, Q_PE) and calls the fit a power
law. Here the batched engine produces such sweeps on the GPU (fidelity of the postselected
solution against the classical solution, for every problem, clock budget and T0 on a grid),
and a small network (``T0Net``: the hhl_mlp_* entry points, trained by the library's own
forward / backward / Adam kernels) learns

    features (log10 kappa, log2 N, the two eigenvalue bounds of Sec. VI over lambda_ub,
              clock budget n_c, right-hand-side kind)
    -> (ln(T0* / T0_power_law), recommended clock count).

The power law stays the fallback: ``choose_t0`` returns the power-law T0 (scale 1) and the
given clock budget when no network is given.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _ffi
from ._ffi import check, load

FLOW_IDS = {"poiseuille": 0, "couette": 1, "random": 2}


class T0Net:
    """The 6 -> 128 -> 128 -> 2 network on the GPU (hhl_mlp_t)."""

    N_PARAMS = 17666

    def __init__(self, params: np.ndarray | None = None, seed: int = 0):
        lib = load()
        self._lib = lib
        h = ctypes.c_void_p()
        check(lib.hhl_mlp_create(ctypes.byref(h)), "hhl_mlp_create")
        self._h = h
        if params is None:
            params = self.init_params(seed)
        self.set_params(params)
        self.x_mean = np.zeros(6, np.float32)
        self.x_std = np.ones(6, np.float32)
        self.y_mean = np.zeros(2, np.float32)
        self.y_std = np.ones(2, np.float32)

    @staticmethod
    def init_params(seed: int = 0) -> np.ndarray:
        """Glorot-uniform weights, zero biases (host, float32)."""
        rng = np.random.default_rng(seed)
        parts = []
        for fan_out, fan_in in ((128, 6), (128, 128), (2, 128)):
            a = math.sqrt(6.0 / (fan_in + fan_out))
            parts.append(rng.uniform(-a, a, fan_out * fan_in))
            parts.append(np.zeros(fan_out))
        return np.concatenate(parts).astype(np.float32)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.hhl_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: np.ndarray) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.N_PARAMS
        check(self._lib.hhl_mlp_set_params(self._h, ctypes.c_void_p(p.ctypes.data), None), "hhl_mlp_set_params")

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.N_PARAMS, dtype=np.float32)
        check(self._lib.hhl_mlp_get_params(self._h, ctypes.c_void_p(p.ctypes.data), None), "hhl_mlp_get_params")
        return p

    # raw device calls (torch float32 tensors)
    def forward_dev(self, x_dev, y_dev, stream=None):
        from . import _stream_handle
        check(self._lib.hhl_mlp_forward(self._h, ctypes.c_void_p(x_dev.data_ptr()), x_dev.shape[0],
                                        ctypes.c_void_p(y_dev.data_ptr()), ctypes.c_void_p(_stream_handle(stream))),
              "hhl_mlp_forward")

    def gradients_dev(self, x_dev, t_dev, grad_dev, loss_dev, stream=None):
        from . import _stream_handle
        check(self._lib.hhl_mlp_gradients(self._h, ctypes.c_void_p(x_dev.data_ptr()), ctypes.c_void_p(t_dev.data_ptr()),
                                          x_dev.shape[0], ctypes.c_void_p(grad_dev.data_ptr()),
                                          ctypes.c_void_p(loss_dev.data_ptr()), ctypes.c_void_p(_stream_handle(stream))),
              "hhl_mlp_gradients")

    def train_step_dev(self, x_dev, t_dev, lr, loss_dev, stream=None):
        from . import _stream_handle
        check(self._lib.hhl_mlp_train_step(self._h, ctypes.c_void_p(x_dev.data_ptr()), ctypes.c_void_p(t_dev.data_ptr()),
                                           x_dev.shape[0], ctypes.c_float(lr), ctypes.c_void_p(loss_dev.data_ptr()),
                                           ctypes.c_void_p(_stream_handle(stream))), "hhl_mlp_train_step")

    # standardised training and prediction
    def fit(self, X: np.ndarray, Y: np.ndarray, steps: int = 1500, batch: int = 256, lr: float = 2e-3,
            seed: int = 0) -> list:
        import torch
        self.x_mean, self.x_std = X.mean(0).astype(np.float32), (X.std(0) + 1e-6).astype(np.float32)
        self.y_mean, self.y_std = Y.mean(0).astype(np.float32), (Y.std(0) + 1e-6).astype(np.float32)
        Xs = torch.tensor((X - self.x_mean) / self.x_std, dtype=torch.float32, device="cuda")
        Ys = torch.tensor((Y - self.y_mean) / self.y_std, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        g = torch.Generator(device="cpu").manual_seed(seed)
        hist = []
        n = Xs.shape[0]
        for it in range(steps):
            idx = torch.randint(0, n, (min(batch, n),), generator=g).cuda()
            xb, yb = Xs[idx].contiguous(), Ys[idx].contiguous()
            self.train_step_dev(xb, yb, lr, loss)
            if it % 100 == 0 or it == steps - 1:
                hist.append(float(loss.item()))
        return hist

    def predict(self, X: np.ndarray) -> np.ndarray:
        import torch
        Xs = torch.tensor((X - self.x_mean) / self.x_std, dtype=torch.float32, device="cuda")
        y = torch.empty((Xs.shape[0], 2), dtype=torch.float32, device="cuda")
        self.forward_dev(Xs, y)
        return y.cpu().numpy() * self.y_std + self.y_mean


def choose_t0(diag: float, off: float, n_points: int, n_clock: int, flow: str, net: "T0Net | None" = None):
    """(T0 scale relative to the power law, recommended clock count) for one problem: from the
    network when given, else the power law itself (scale 1) and the budget."""
    if net is None:
        return 1.0, n_clock
    y = net.predict(features(diag, off, n_points, n_clock, flow)[None, :])[0]
    return float(math.exp(y[0])), int(min(max(round(float(y[1])), 1), n_clock))


def features(diag: float, off: float, n_points: int, n_clock: int, flow: str) -> np.ndarray:
    """Feature row of a Toeplitz tridiagonal A = tridiag(off, diag, off) of size N."""
    N = n_points
    lam = diag + 2.0 * off * np.cos(np.arange(1, N + 1) * np.pi / (N + 1))
    kappa = np.abs(lam).max() / np.abs(lam).min()
    lam_ub = abs(diag) + 2.0 * abs(off)
    b1 = diag
    b2 = abs(off) * math.sqrt(2.0 * (N - 1) / N)
    r = math.sqrt(max(N - 1, 1))
    return np.array([math.log10(kappa), math.log2(N), (b1 - b2 * r) / lam_ub, (b1 + b2 / r) / lam_ub,
                     float(n_clock), float(FLOW_IDS[flow])], dtype=np.float64)


def sweep_problems(count: int, seed: int = 0, ns_range=(3, 7)) -> list:
    """Shifted channel operators A = L_N + beta I (kappa spread by the shift), with a
    right-hand side of each kind."""
    from synth_inputs import rhs
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n_s = int(rng.integers(ns_range[0], ns_range[1] + 1))
        N = 1 << n_s
        h = 1.0 / (N + 1)
        shift = (4.0 / h ** 2) * 10.0 ** rng.uniform(-4.0, -0.5)
        flow = ["poiseuille", "couette", "random"][i % 3]
        b = rng.random(N) if flow == "random" else rhs(flow, N)
        out.append(dict(n_s=n_s, N=N, diag=2.0 / h ** 2 + shift, off=-1.0 / h ** 2, flow=flow, b=b))
    return out


def run_sweep(problems: list, n_clocks=(4, 5, 6, 7), scales=None, streams: int = 8) -> dict:
    """Fidelity |<xhat_Q|xhat_C>| for every (problem, n_c, T0 scale) through the batched engine
    (complex64). Returns dict(F [P, C, S], scales, n_clocks)."""
    import torch

    import paper_2307_00391_gb300 as pkg
    if scales is None:
        scales = 10.0 ** np.linspace(-1.5, 1.5, 25)
    P, C, S = len(problems), len(n_clocks), len(scales)
    F = np.zeros((P, C, S))
    specs = [(p, c, s) for p in range(P) for c in range(C) for s in range(S)]
    chunk = 1536
    for c0 in range(0, len(specs), chunk):
        part = specs[c0:c0 + chunk]
        probs, bs = [], []
        for p, c, s in part:
            pr = problems[p]
            probs.append(dict(n_sys_qubits=pr["n_s"], n_clock=n_clocks[c], diag=np.full(pr["N"], pr["diag"]),
                              off=np.full(pr["N"] - 1, pr["off"]), t0_rule="power_law", t0_scale=float(scales[s])))
            bs.append(pr["b"])
        batch = pkg.HHLBatch(probs, streams=streams)
        out, _ = batch.run_host(batch.pack_rhs(bs))
        res = batch.unpack(out)
        for (p, c, s), r in zip(part, res):
            pr = problems[p]
            xc = _classical(pr)
            F[p, c, s] = abs(np.vdot(xc, r["xhat"]))
        batch.close()
        torch.cuda.synchronize()
    return dict(F=F, scales=np.asarray(scales), n_clocks=list(n_clocks))


def _classical(pr: dict) -> np.ndarray:
    """Normalised A^{-1} b by the Thomas algorithm (Toeplitz tridiagonal)."""
    N, d, o, b = pr["N"], pr["diag"], pr["off"], np.asarray(pr["b"], dtype=np.float64)
    c = np.zeros(N)
    x = np.zeros(N)
    beta = d
    c[0] = o / beta
    x[0] = b[0] / beta
    for i in range(1, N):
        beta = d - o * c[i - 1]
        c[i] = o / beta
        x[i] = (b[i] - o * x[i - 1]) / beta
    for i in range(N - 2, -1, -1):
        x[i] -= c[i] * x[i + 1]
    return x / np.linalg.norm(x)


def training_set(problems: list, sweep: dict, tol: float = 0.01):
    """(X, Y, Fbest): features per (problem, n_c); Y = (ln T0*/T0_pl, recommended n_c), the
    recommendation being the smallest budget whose best fidelity is within tol of this one's."""
    F, scales, ncs = sweep["F"], sweep["scales"], sweep["n_clocks"]
    X, Y, FB = [], [], []
    for p, pr in enumerate(problems):
        best = F[p].max(axis=1)
        for c, nc in enumerate(ncs):
            s_best = scales[int(np.argmax(F[p, c]))]
            rec = next(ncs[c2] for c2 in range(c + 1) if best[c2] >= best[c] - tol)
            X.append(features(pr["diag"], pr["off"], pr["N"], nc, pr["flow"]))
            Y.append([math.log(s_best), float(rec)])
            FB.append(best[c])
    return np.array(X), np.array(Y), np.array(FB)


def experiment(n_problems: int = 270, n_clocks=(4, 5, 6), train_frac: float = 0.9, seed: int = 11,
               steps: int = 3000) -> dict:
    """Sweep (n_problems x n_clocks x 25 T0 values through the batched engine), train on the
    first train_frac of the problems, and compare held-out fidelities at the predicted T0 and
    at the power-law T0 (both simulated)."""
    import time

    import paper_2307_00391_gb300 as pkg
    t0 = time.perf_counter()
    problems = sweep_problems(n_problems, seed=seed, ns_range=(3, 6))
    sweep = run_sweep(problems, n_clocks=n_clocks)
    t_sweep = time.perf_counter() - t0
    n_train = int(train_frac * n_problems)
    X, Y, _ = training_set(problems[:n_train], dict(F=sweep["F"][:n_train], scales=sweep["scales"],
                                                    n_clocks=sweep["n_clocks"]))
    net = T0Net(seed=seed)
    t1 = time.perf_counter()
    hist = net.fit(X, Y, steps=steps, batch=256, lr=2e-3)
    t_train = time.perf_counter() - t1
    held = problems[n_train:]
    rows, specs = [], []
    for p, pr in enumerate(held):
        for nc in n_clocks:
            rows.append(features(pr["diag"], pr["off"], pr["N"], nc, pr["flow"]))
            specs.append((p, nc))
    pred = net.predict(np.array(rows))
    probs, bs = [], []
    for (p, nc), s in zip(specs, np.exp(pred[:, 0])):
        pr = held[p]
        for scale in (float(s), 1.0):
            probs.append(dict(n_sys_qubits=pr["n_s"], n_clock=nc, diag=np.full(pr["N"], pr["diag"]),
                              off=np.full(pr["N"] - 1, pr["off"]), t0_rule="power_law", t0_scale=scale))
            bs.append(pr["b"])
    batch = pkg.HHLBatch(probs)
    out, _ = batch.run_host(batch.pack_rhs(bs))
    res = batch.unpack(out)
    fp, fl = [], []
    for j, (p, nc) in enumerate(specs):
        xc = _classical(held[p])
        fp.append(abs(np.vdot(xc, res[2 * j]["xhat"])))
        fl.append(abs(np.vdot(xc, res[2 * j + 1]["xhat"])))
    fp, fl = np.array(fp), np.array(fl)
    best = np.array([sweep["F"][n_train + p, list(n_clocks).index(nc)].max() for p, nc in specs])
    return dict(instances_swept=int(sweep["F"].size), sweep_seconds=t_sweep, train_rows=int(len(X)),
                train_seconds=t_train, loss_first=hist[0], loss_last=hist[-1], held_out=len(specs),
                fidelity_learned_mean=float(fp.mean()), fidelity_power_law_mean=float(fl.mean()),
                fidelity_grid_best_mean=float(best.mean()),
                learned_better_fraction=float(np.mean(fp > fl)))


if __name__ == "__main__":
    import json
    print(json.dumps(experiment()))
