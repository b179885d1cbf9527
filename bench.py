"""Benchmark of the HHL state-vector hot path on GB300.

python bench.py [--gpus N --steps K --warmup W]
                [--workload poiseuille_2p18|couette_1024|batch_256|poiseuille_16|poiseuille_2p16|qft_iqft_20x16|qft_iqft_30|qft_iqft_32]
                [--impl ours|reference] [--precision c64|c128] [--gemm auto|simt|tcgen05]

A step is one whole HHL solve of the workload: a1 prepare_rhs, a2..a5 apply_circuit (QPE
controlled-U_k, fused inverse QFT + inversion RY + QFT, uncompute, clock Hadamards),
a6 postselection statistics and a7 the dissipation readout, on device-resident inputs.
Prints one JSON line (rank 0). Under torchrun each rank runs an independent replica of
the solve on its own GPU (the single solve does not shard; no collective on the data path).

--impl reference times the FP64 CPU oracle (the plain gate-by-gate simulator) on the
host cores on the same workload; it never touches a GPU.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "statevector gate GB/s (% of HBM peak); batched HHL solves/s at 1e-6 fidelity"
DEFAULT_WORKLOAD = "poiseuille_2p18"
L2_FLUSH_BYTES = 256 << 20

WORKLOADS = {
    "couette_1024": dict(flow="couette", n_s=10, n_c=12, expm="dense", unit="HHL solves/s",
                         desc="Couette flow, N=1024 (10 system qubits), n_c=12 clock + 1 ancilla = 23 qubits, "
                              "dense controlled exp(i A t) as complex GEMMs"),
    "poiseuille_16": dict(flow="poiseuille", n_s=4, n_c=6, expm="dense", unit="HHL solves/s", t0_rule="power_law",
                          desc="Poiseuille flow, N=16, n_c=6, 11 qubits, T0 from the power law"),
    "batch_256": dict(kind="batch", count=256, unit="HHL solves/s", n_s=0, n_c=0, expm="dense",
                      desc="256 uneven Poiseuille/Couette instances: n_s ~ U{6..12}, n_c ~ U{8..12}, "
                           "b ~ U[0,1)^N, T0 = power law x 10^U(-1,1); complex64, one CUDA graph"),
    "poiseuille_2p16": dict(flow="poiseuille", n_s=16, n_c=11, expm="trotter", unit="GB/s",
                            trotter_dt=1024.0, trotter_steps_max=8,
                            desc="Poiseuille flow, N=2^16, n_c=11, 28 qubits, Strang-Trotter exp(i A t) "
                                 "(a 2 GiB case of the 32-qubit kernels, for profiling)"),
    # the paper's Fig. 1c gate benchmark: QFT then inverse QFT on whole registers of random states
    "qft_iqft_20x16": dict(kind="qft", n=20, states=16, unit="GB/s", n_s=0, n_c=0, expm="none",
                           desc="QFT then inverse QFT on all 20 qubits of 16 random states (Fig. 1c circuit)"),
    "qft_iqft_30": dict(kind="qft", n=30, states=1, unit="GB/s", n_s=0, n_c=0, expm="none",
                        desc="QFT then inverse QFT on all 30 qubits of one random state (Fig. 1c circuit)"),
    "qft_iqft_32": dict(kind="qft", n=32, states=1, unit="GB/s", n_s=0, n_c=0, expm="none",
                        desc="QFT then inverse QFT on all 32 qubits of one random state (Fig. 1c circuit)"),
    "poiseuille_2p18": dict(flow="poiseuille", n_s=18, n_c=13, expm="trotter", unit="GB/s",
                            trotter_dt=1024.0, trotter_steps_max=8,
                            desc="Poiseuille flow, N=2^18, n_c=13, 32 qubits, Strang-Trotter exp(i A t)"),
}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel as a
# fraction of its algorithmic bytes, from Nsight Compute captures summarised under profiles/
# (on the 28-qubit case where the 32-qubit workload is too large to capture with counters:
# the traffic of a launch grows with the rows it processes, so the fraction carries over),
# with the SHA-256 prefix of the kernel's source file at capture time: reported only while the
# source is unchanged (otherwise null, the counters no longer describe the kernel).
KERNEL_TRAFFIC = {
    ("poiseuille_2p18", "c64", "k_trotter_pass"): (0.9625, "hhl_trotter.cu", "6096110439013a16"),
    # DRAM bytes per launch of the full-size product (mean of three launches of one capture; the
    # operands A and B once each, hi and lo; the rows it writes stay in L2)
    ("couette_1024", "c64", "k_ctrl_gemm_tc"): (33.635e6, "hhl_gemm_tc.cu", "1ff6a778caf96620", "bytes"),
}


def _traffic(workload: str, precision: str, kernel: str, algorithmic: float):
    ent = KERNEL_TRAFFIC.get((workload, precision, kernel))
    if ent is None:
        return None
    import hashlib
    path = os.path.join(ROOT, "paper_2307_00391_gb300", "csrc", ent[1])
    try:
        digest = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if digest != ent[2]:
        return None
    return ent[0] if len(ent) > 3 and ent[3] == "bytes" else ent[0] * algorithmic


def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The largest of the ranks' values (timings: the job takes as long as its slowest rank)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The sum of the ranks' values (counts of units done on each rank)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def replica_rate(units_per_rank: float, world: int, slowest_s: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' units over the slowest time."""
    return world * units_per_rank / slowest_s


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _fp32_simt_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("", "[N/A]"))}


# ------------------------------------------------------------------------------ oracle arm


def _oracle_setup(wl: dict):
    from oracle import hhl_oracle as o
    from synth_inputs import rhs
    n = 1 << wl["n_s"]
    diag, off = o.laplacian_tridiag(n)
    pl = o.plan(o.dense_from_tridiag(diag, off), wl["n_c"], t0_rule=wl.get("t0_rule", "range_fill"))
    t_k = [pl["t0"] * (1 << k) / (1 << wl["n_c"]) for k in range(wl["n_c"])]
    ev = [o.evolution_dense(pl["a_hat"], t) for t in t_k]
    return o, pl, ev, rhs(wl["flow"], n)


def _oracle_solve(o, pl, ev, b, wl):
    psi = o.hhl_circuit(b, wl["n_s"], pl, evolutions=ev)
    post = o.postselect(psi, wl["n_s"], wl["n_c"])
    u = o.velocity(post["v"], float((b @ b) ** 0.5), pl["C"], pl["lam_ub"])
    return o.dissipation(u, 0.0, 1.0 if wl["flow"] == "couette" else 0.0, 0.1)


def _oracle_batch_sample(budget_s: float) -> dict:
    """Oracle solves of batch instances with n_s <= 9 (spread over the batch in instance
    order), plan excluded; the batch time is extrapolated by the controlled-product flops."""
    from oracle import hhl_oracle as o
    from synth_inputs import batch_instances, walls
    inst = batch_instances(WORKLOADS["batch_256"]["count"])
    flops = [2.0 * it["n_c"] * 8.0 * (1 << (it["n_c"] - 1)) * (1 << it["n_s"]) ** 2 for it in inst]
    pick = [i for i, it in enumerate(inst) if it["n_s"] <= 9]
    t_sum, f_sum, done = 0.0, 0.0, []
    t_start = time.perf_counter()
    for i in pick:
        it = inst[i]
        n = 1 << it["n_s"]
        diag, off = o.laplacian_tridiag(n)
        a = o.dense_from_tridiag(diag, off)
        t0 = o.t0_total("power_law", it["n_c"], kappa=o.condition_number(a)) * it["t0_mult"]
        pl = o.plan(a, it["n_c"], t0_rule="user", t0=t0)
        ev = [o.evolution_dense(pl["a_hat"], t0 * (1 << k) / (1 << it["n_c"])) for k in range(it["n_c"])]
        w = walls(it["flow"])
        tt = time.perf_counter()
        post = o.postselect(o.hhl_circuit(it["b"], it["n_s"], pl, evolutions=ev), it["n_s"], it["n_c"])
        o.dissipation(o.velocity(post["v"], float(np.linalg.norm(it["b"])), pl["C"], pl["lam_ub"]), w[0], w[1], 0.1)
        t_sum += time.perf_counter() - tt
        f_sum += flops[i]
        done.append(i)
        if time.perf_counter() - t_start > budget_s:
            break
    est = sum(flops) / (f_sum / t_sum)
    return {"value": len(inst) / est, "unit": "HHL solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "extrapolated": True,
            "sample": f"{len(done)} oracle solves of batch instances with n_s <= 9 ({t_sum:.1f} s, plan excluded); "
                      f"batch time extrapolated by controlled-product flops"}


def _trotter_steps(wl: dict) -> list:
    """r_k = clamp(ceil(t_k / dt), 1, r_max) with the range-fill T0 (the planner's rule)."""
    n_c = wl["n_c"]
    t0 = 2.0 * math.pi * ((1 << n_c) - 1)
    out = []
    for k in range(n_c):
        r = max(1, math.ceil(t0 * (1 << k) / (1 << n_c) / wl["trotter_dt"]))
        if wl.get("trotter_steps_max", 0) > 0:
            r = min(r, wl["trotter_steps_max"])
        out.append(r)
    return out


def algorithmic_bytes_per_solve(wl: dict, prec_bytes: int = 8) -> float:
    """Minimum HBM bytes of one Trotter-mode solve (postselect-early): prepare (write both
    halves), the controlled products (every row a pass changes, read and written once; clock
    bits grouped while a row's layer list stays within 17 layers, as the planner does), the
    clock block (read anc = 0, write both halves), the Hadamard layer (anc = 1 read and
    written) and the measurement (both halves read)."""
    n_s, n_c = wl["n_s"], wl["n_c"]
    N, R = 1 << n_s, 1 << n_c
    half = R * N * prec_bytes
    r = _trotter_steps(wl)
    rows = []
    for order in (list(range(n_c)), list(range(n_c - 1, -1, -1))):
        group, layers = [], 1
        for k in order:
            lk = 2 * r[k]
            if lk + 1 > 17:
                if group:
                    rows.append(R / 2 if len(group) == 1 else R * (1 - 2.0 ** -len(group)))
                group, layers = [], 1
                rows.extend([R / 2] * (1 + max(0, -(-(lk + 1 - 17) // 16))))
                continue
            if layers + lk > 17:
                rows.append(R / 2 if len(group) == 1 else R * (1 - 2.0 ** -len(group)))
                group, layers = [], 1
            group.append(k)
            layers += lk
        if group:
            rows.append(R / 2 if len(group) == 1 else R * (1 - 2.0 ** -len(group)))
    trotter = sum(2.0 * x * N * prec_bytes for x in rows)
    return 2.0 * half + trotter + 3.0 * half + 2.0 * half + 2.0 * half


def _trotter_groups(wl: dict) -> tuple[list, list]:
    """The planner's passes as (kb, bits) groups: forward (QPE) from bit 0 up, adjoint
    (uncompute) from the top bit down; consecutive single-step bits share a pass while the
    all-bits-set layer list stays within 17 layers."""
    n_c = wl["n_c"]
    r = _trotter_steps(wl)
    out = []
    for order in (list(range(n_c)), list(range(n_c - 1, -1, -1))):
        groups, group, layers = [], [], 1
        for k in order:
            lk = 2 * r[k]
            if layers + lk > 17 and group:
                groups.append((min(group), len(group)))
                group, layers = [], 1
            group.append(k)
            layers += lk
        if group:
            groups.append((min(group), len(group)))
        out.append(groups)
    return out[0], out[1]


def postselected_bytes(wl: dict, prec_bytes: int) -> dict:
    """Minimum HBM bytes per kernel of one postselected solve (hhl_solve_postselected): the
    expansion passes write every clock row but row 0 once and read each source row once; the
    clock block reads the anc = 0 half and writes both halves; the sums read both halves; the
    reduction passes read the rows they fold and write the rows they keep."""
    n_s, n_c = wl["n_s"], wl["n_c"]
    N, R = 1 << n_s, 1 << n_c
    row = N * prec_bytes
    half = R * row
    fwd, adj = _trotter_groups(wl)
    expand = sum(((1 << kb) * ((1 << g) - 1) + (1 << kb)) * row for kb, g in fwd)
    reduce = sum(((1 << kb) * (1 << g) + (1 << kb)) * row for kb, g in adj)
    return {"k_trotter_expand": (expand, len(fwd)), "k_trotter_reduce": (reduce, len(adj)),
            "k_clock": (3.0 * half, 3), "k_measure_sums": (2.0 * half, 1), "k_prep_row": (row, 1)}


def _oracle_trotter_sample(wl: dict, budget_s: float) -> dict:
    """The oracle on units of the 32-qubit solve, timed one by one and extrapolated: the
    controlled Strang product U_k on one system row (for each k; the solve applies it to
    2^(n_c-1) rows in QPE and again in the uncompute), the clock block on one system column
    (inverse QFT, controlled RY, QFT over n_c + 1 qubits; 2^n_s columns) and the Hadamard
    layer on one column (2^n_s columns). Preparation and measurement (single numpy passes
    over the state) are not timed. Value: algorithmic bytes per solve / estimated time."""
    from oracle import hhl_oracle as o
    n_s, n_c = wl["n_s"], wl["n_c"]
    N, R = 1 << n_s, 1 << n_c
    diag, off = o.laplacian_tridiag(N)
    lub = 4.0 * (N + 1) ** 2
    t0 = o.t0_total("range_fill", n_c)
    theta = o.rotation_angles(n_c, t0)
    r = _trotter_steps(wl)
    rng = np.random.default_rng(230700391)
    t_start = time.perf_counter()
    # one column of the clock block and of the Hadamard layer
    col = rng.standard_normal(2 * R) + 1j * rng.standard_normal(2 * R)
    col[R:] = 0.0
    tt = time.perf_counter()
    o.qft(col, n_c + 1, 0, n_c, inverse=True)
    o.apply_clock_controlled_ry(col, 0, n_c, theta)
    o.qft(col, n_c + 1, 0, n_c, inverse=False)
    t_clock = time.perf_counter() - tt
    hcol = col[R:].copy()
    tt = time.perf_counter()
    for q in range(n_c):
        o.apply_1q(hcol, n_c, q, o.H_GATE)
    t_h = time.perf_counter() - tt
    # system rows through each U_k, repeatedly while the budget lasts (mean per k)
    t_sum, t_cnt = {}, {}
    psi = np.zeros(2 * N, dtype=np.complex128)
    rounds = 0
    while True:
        for k in range(n_c - 1, -1, -1):
            psi[N:] = rng.standard_normal(N)
            t_k = t0 * (1 << k) / R
            tt = time.perf_counter()
            o.apply_trotter_controlled(psi, n_s + 1, n_s, n_s, diag / lub, off / lub, t_k, r[k])
            t_sum[k] = t_sum.get(k, 0.0) + time.perf_counter() - tt
            t_cnt[k] = t_cnt.get(k, 0) + 1
            if time.perf_counter() - t_start > budget_s:
                break
        rounds += 1
        if time.perf_counter() - t_start > 0.5 * budget_s or rounds >= 8:
            break
    t_row = {k: t_sum[k] / t_cnt[k] for k in t_sum}
    for k in range(n_c):  # bits not reached: their layer count times the measured per-layer time
        if k not in t_row:
            per_layer = sum(t_row.values()) / sum(2 * r[j] + 1 for j in t_row)
            t_row[k] = per_layer * (2 * r[k] + 1)
    est = 2 * (R // 2) * sum(t_row.values()) + N * (t_clock + t_h)
    value = algorithmic_bytes_per_solve(wl) / est / 1e9
    return {"value": value, "unit": wl["unit"], "cores": os.cpu_count(), "kind": "oracle",
            "extrapolated": True,
            "sample": f"oracle units of one solve ({sum(t_cnt.values())} controlled Strang products on one "
                      f"2^{n_s}-amplitude row each, over {len(t_row)} clock bits; one clock-block column, one Hadamard column; "
                      f"{time.perf_counter() - t_start:.1f} s), extrapolated to the whole solve "
                      f"({est:.0f} s per solve); algorithmic bytes per solve / estimated time"}


def _oracle_qft_sample(wl: dict, budget_s: float) -> dict:
    """The oracle's gate-by-gate QFT then inverse QFT on 20-qubit random states (whole
    circuits, repeated while the budget lasts), extrapolated to the workload by gate count x
    state size (n (n+1) / 2 gates of 2^n amplitudes per transform)."""
    from oracle import hhl_oracle as o
    from synth_inputs import random_state
    n0 = min(wl["n"], 20)
    times = []
    t_start = time.perf_counter()
    while True:
        psi = random_state(n0, seed_offset=900 + len(times))
        tt = time.perf_counter()
        o.qft_then_iqft(psi, n0)
        times.append(time.perf_counter() - tt)
        if time.perf_counter() - t_start > budget_s * 0.5 or len(times) >= 8:
            break
    t0 = sum(times) / len(times)
    n = wl["n"]
    est = t0 * (n * (n + 1) * 2.0 ** n) / (n0 * (n0 + 1) * 2.0 ** n0) * wl["states"]
    value = 4.0 * wl["states"] * (2 ** n) * 8 / est / 1e9
    return {"value": value, "unit": wl["unit"], "cores": os.cpu_count(), "kind": "oracle",
            "extrapolated": not (n == n0 and wl["states"] == 1),
            "sample": f"{len(times)} oracle QFT-IQFT circuits on {n0}-qubit random states "
                      f"({sum(times):.1f} s)" + ("" if n == n0 and wl["states"] == 1 else
                                                 f", extrapolated to {wl['states']} x {n} qubits by gates x amplitudes")}


def cpu_baseline_sample(workload: str, budget_s: float = 30.0) -> dict:
    """The oracle as it stands, timed on the host cores on whole solves of the workload
    (the plan's matrix exponentials excluded, as on the GPU side); stops after the first
    solve that takes the total past ``budget_s``."""
    wl = WORKLOADS[workload]
    if wl.get("kind") == "batch":
        return _oracle_batch_sample(budget_s)
    if wl.get("kind") == "qft":
        return _oracle_qft_sample(wl, budget_s)
    if wl["expm"] != "dense":
        return _oracle_trotter_sample(wl, budget_s)
    o, pl, ev, b = _oracle_setup(wl)
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        _oracle_solve(o, pl, ev, b, wl)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s or len(times) >= 50:
            break
    return {"value": len(times) / sum(times), "unit": wl["unit"], "cores": os.cpu_count(), "kind": "oracle",
            "extrapolated": False,
            "sample": f"{len(times)} whole oracle solve(s) of {workload} (plan excluded), "
                      f"{sum(times):.1f} s, numpy BLAS threads = {os.environ.get('OPENBLAS_NUM_THREADS', 'default')}"}


def _cpu_baseline_subprocess(workload: str) -> dict:
    env = dict(os.environ, OPENBLAS_NUM_THREADS=str(os.cpu_count()), OMP_NUM_THREADS=str(os.cpu_count()),
               CUDA_VISIBLE_DEVICES="")
    code = ("import json, bench; print('CPUBASE' + json.dumps(bench.cpu_baseline_sample(%r)))" % workload)
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=240)
        for line in out.stdout.splitlines():
            if line.startswith("CPUBASE"):
                return json.loads(line[7:])
        return {"value": None, "kind": "oracle", "sample": "failed: " + out.stderr[-300:]}
    except Exception as e:
        return {"value": None, "kind": "oracle", "sample": f"failed: {e}"}


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    if wl.get("kind") == "batch":
        cb = _oracle_batch_sample(120.0)
        print(json.dumps({
            "metric": METRIC, "value": cb["value"], "unit": wl["unit"], "n_gpus": world, "steps": 1,
            "warmup": 0, "ms_per_step": 1e3 * wl["count"] / cb["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": args.workload, "desc": wl["desc"]},
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": wl["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    if wl.get("kind") == "qft":
        warm = min(args.warmup, 3)
        for _ in range(warm):            # untimed short samples (imports, first-touch)
            _oracle_qft_sample(wl, 0.5)
        samples = [_oracle_qft_sample(wl, 20.0) for _ in range(max(1, min(args.steps, 3)))]
        value = sum(x["value"] for x in samples) / len(samples)
        step_bytes = 4.0 * wl["states"] * (2 ** wl["n"]) * 8
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": wl["unit"], "n_gpus": world, "steps": len(samples),
            "warmup": warm, "ms_per_step": 1e3 * step_bytes / (value * 1e9), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"]}, "impl": "reference",
            "cpu_baseline": dict(samples[-1], value=value),
            "e2e": {"value": value, "unit": wl["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    if wl["expm"] != "dense":
        # each step: one bounded oracle sample of the solve (see _oracle_trotter_sample); the
        # warm-up steps are short untimed samples
        warm = min(args.warmup, 3)
        for _ in range(warm):
            _oracle_trotter_sample(wl, 0.5)
        samples = [_oracle_trotter_sample(wl, 20.0) for _ in range(max(1, min(args.steps, 3)))]
        value = sum(x["value"] for x in samples) / len(samples)
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": wl["unit"], "n_gpus": world, "steps": len(samples),
            "warmup": warm, "ms_per_step": 1e3 * algorithmic_bytes_per_solve(wl) / (value * 1e9),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"]}, "impl": "reference",
            "cpu_baseline": dict(samples[-1], value=value),
            "e2e": {"value": value, "unit": wl["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    o, pl, ev, b = _oracle_setup(wl)
    for _ in range(min(args.warmup, 1)):
        _oracle_solve(o, pl, ev, b, wl)
    times = []
    deadline = time.perf_counter() + 150.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _oracle_solve(o, pl, ev, b, wl)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > deadline:
            break
    value = len(times) / sum(times)
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": wl["unit"], "n_gpus": world, "steps": len(times),
        "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"]}, "impl": "reference",
        "cpu_baseline": {"value": value, "unit": wl["unit"], "cores": os.cpu_count(), "kind": "oracle",
                         "extrapolated": False, "sample": f"{len(times)} whole oracle solves (plan excluded)"},
        "e2e": {"value": value, "unit": wl["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------------------ GPU arm


def _algorithmic(plan_info: dict, wl: dict, prec_bytes: int) -> dict:
    """Algorithmic work per launch of each kernel (flops for the GEMMs, bytes otherwise)."""
    n_s, n_c = wl["n_s"], wl["n_c"]
    N, R = 1 << n_s, 1 << n_c
    half = R * N * prec_bytes
    m_sub = R // 2
    passes = plan_info.get("trotter_passes", 0)
    tb_launch = plan_info.get("trotter_bytes", 0.0) / passes if passes else 0.0
    return {
        "k_ctrl_gemm_simt<f32>": ("flop", 8.0 * m_sub * N * N),
        "k_ctrl_gemm_simt<f64>": ("flop", 8.0 * m_sub * N * N),
        "k_ctrl_gemm_tc": ("flop", 8.0 * m_sub * N * N),
        "k_rows_scatter": ("byte", 2.0 * m_sub * N * prec_bytes),
        "k_clock_block": ("byte", 3.0 * half),
        "k_register_transform": ("byte", 2.0 * half),
        # split register passes: the stage's single-pass minimum spread over its launches
        # (clock block: read anc = 0, write both halves, 3 passes; Hadamard layer: 2 passes)
        "k_clock_pass_a": ("byte", 3.0 * half / 3),
        "k_clock_pass_b": ("byte", 3.0 * half / 3),
        "k_clock_pass_c": ("byte", 3.0 * half / 3),
        "k_hadamard_pass": ("byte", 2.0 * half / 2),
        # the same stages as single L2-staged group launches
        "k_clock_group": ("byte", 3.0 * half),
        "k_hadamard_group": ("byte", 2.0 * half),
        "k_prep_fill": ("byte", 2.0 * half),
        "k_measure_sums": ("byte", 2.0 * half),
        # grouped Trotter passes change different row counts: the plan's total over its passes
        # (the complex128 passes in double-float arithmetic are bound by FP32 issue, not HBM)
        "k_trotter_pass": ("byte", tb_launch),
        "k_trotter_pass_df": ("byte", tb_launch),
        # the halos saved at the boundaries between warps' runs are an overhead of the
        # in-place passes, not algorithmic traffic
        "k_trotter_bounds": ("byte", 0.0),
        **_tree_algorithmic(wl, prec_bytes),
    }


def _tree_algorithmic(wl: dict, prec_bytes: int) -> dict:
    if wl.get("expm") != "trotter":
        return {}
    pb = postselected_bytes(wl, prec_bytes)
    out = {}
    for base in ("k_trotter_expand", "k_trotter_reduce"):
        total, launches = pb[base]
        for suffix in ("", "_df"):
            out[base + suffix] = ("byte", total / launches)
    return out


def _breakdown(prof: dict, steps: int) -> dict:
    total = sum(ms for _, ms in prof.values()) or 1.0
    return {name: {"launches_per_step": n / steps, "ms_per_step": ms / steps, "share": ms / total}
            for name, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1])}


def _roofline(prof: dict, alg: dict, peaks: dict, workload: str, precision: str, timing: str):
    """The dominant kernel's achieved algorithmic rate (per-launch CUDA events on its stream)
    against its measured peak."""
    if not prof:
        return None
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    if dom not in alg:
        return {"kernel": dom, "bound": None, "note": "no algorithmic work model for this kernel"}
    kind, per = alg[dom]
    n, ms = prof[dom]
    avg_s = ms / n / 1e3
    if kind == "flop":
        achieved = per / avg_s / 1e12
        if dom.startswith("k_ctrl_gemm_tc"):
            peak = peaks.get("bf16_tflops", 1900.0)
            bound, note = "tensor", ("FP16 dense = measured bf16 burst (same nominal rate); the split-FP16 "
                                     "scheme issues 3 MMAs per algorithmic product")
        elif dom.endswith("<f64>"):
            peak = 1.25
            bound, note = "alu", "FP64 nominal 1.25 TFLOP/s"
        else:
            peak = _fp32_simt_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
            bound, note = "alu", "FP32 CUDA cores: 152 SMs x 128 lanes x 2 flop x max SM clock"
        unit = "TFLOP/s"
    else:
        achieved = per / avg_s / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        bound, note, unit = "hbm", "measured HBM copy (MEASURED_PEAKS.json)", "GB/s"
    return {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": _traffic(workload, precision, dom, per), "peak_source": note,
            "algorithmic_per_launch": per, "avg_launch_ms": avg_s * 1e3, "timing": timing}


def solve_block(pkg, workload: str, precision: str, gemm: str, steps: int, warmup: int, world: int,
                local_rank: int, e2e_steps: int = 10, postselected: bool = False) -> dict:
    """One workload of whole solves (prepare_rhs, apply_circuit, measure, dissipation; or with
    `postselected` the one call hhl_solve_postselected) on device-resident inputs, L2 flushed
    between steps: a plain timed loop (CUDA events around each step, no per-launch events), then
    a second timed loop with per-launch events (the per-kernel breakdown and the dominant
    kernel's roofline), then the same solve end to end through the public API with host b and
    host results."""
    import numpy as np
    import torch
    from synth_inputs import rhs, walls

    wl = WORKLOADS[workload]
    n_s, n_c = wl["n_s"], wl["n_c"]
    N = 1 << n_s
    diag, off = pkg.laplacian(N)
    b = rhs(wl["flow"], N)
    plan = pkg.HHLPlan(n_s, n_c, diag=diag, off=off, precision=precision, expm=wl["expm"],
                       t0_rule=wl.get("t0_rule", "range_fill"), gemm=gemm, nu=0.1, walls=walls(wl["flow"]),
                       trotter_dt=wl.get("trotter_dt", 1.0), trotter_steps_max=wl.get("trotter_steps_max", 0))
    info = plan.info
    stream = torch.cuda.Stream()
    st = plan.new_state()
    b_dev = torch.tensor(b.astype(np.complex128), device="cuda")
    meas = torch.empty(4 + 2 * N, dtype=torch.float64, device="cuda")
    eps = torch.empty(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def step():
        if postselected:
            plan.solve_postselected(b_dev, st, meas, eps, stream=stream)
            return
        plan.prepare_rhs(b_dev, st, stream=stream)
        plan.apply_circuit(st, stream=stream)
        plan.measure_async(st, meas, stream=stream)
        plan.dissipation_async(st, eps, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    stream.synchronize()
    plan.status(stream)

    def timed_loop(profile: bool):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if profile:
            pkg.profile_reset()
            pkg.profile_enable(True)
        launches0 = pkg.kernel_launch_count()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local_rank) as clk:
            with torch.cuda.stream(stream):
                for i in range(steps):
                    flush.zero_()
                    evs[i][0].record(stream)
                    step()
                    evs[i][1].record(stream)
            torch.cuda.synchronize()
        launches = pkg.kernel_launch_count() - launches0
        prof = None
        if profile:
            pkg.profile_enable(False)
            prof = pkg.profile_read()
        plan.status(stream)
        total = max_over_ranks(sum(a.elapsed_time(c) for a, c in evs) / 1e3, world)
        return total, launches, prof, clk.summary()

    total_s, launches, _, clocks = timed_loop(False)
    prof_total_s, _, prof, _ = timed_loop(True)

    b_pin = torch.tensor(b, dtype=torch.float64).pin_memory()
    bz_pin = torch.tensor(b.astype(np.complex128)).pin_memory()
    meas_pin = torch.empty(4 + 2 * N, dtype=torch.float64).pin_memory()
    eps_pin = torch.empty(1, dtype=torch.float64).pin_memory()
    e2e_times = []
    for _ in range(max(3, e2e_steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if postselected:   # host b in, host results out, through the same public call
            with torch.cuda.stream(stream):
                b_dev.copy_(bz_pin, non_blocking=True)
                plan.solve_postselected(b_dev, st, meas, eps, stream=stream)
                meas_pin.copy_(meas, non_blocking=True)
                eps_pin.copy_(eps, non_blocking=True)
            stream.synchronize()
            m = {"p_success": float(meas_pin[0])}
            e = float(eps_pin[0])
        else:
            plan.prepare_rhs_host(b_pin, st, stream=stream)
            plan.apply_circuit(st, stream=stream)
            m = plan.measure(st, stream=stream)
            e = plan.dissipation(st, stream=stream)
        e2e_times.append(time.perf_counter() - t0)
    e2e_times = e2e_times[1:]
    e2e_total = max_over_ranks(sum(e2e_times), world)

    prec_bytes = 8 if precision == "c64" else 16
    alg = _algorithmic(info, wl, prec_bytes)
    if postselected:  # its clock block reads the anc = 0 half and writes the anc = 1 half only
        half = (1 << (wl["n_s"] + wl["n_c"])) * prec_bytes
        for x in "abc":
            alg[f"k_clock_pass_{x}"] = ("byte", 2.0 * half / 3)
        if wl["expm"] == "dense":  # tensor-core tree steps: 2^k rows for k >= 7, both trees
            n_c, N = wl["n_c"], 1 << wl["n_s"]
            tc_steps = max(1, n_c - 7)
            alg["k_ctrl_gemm_tc"] = ("flop", 2.0 * 8.0 * sum(1 << k for k in range(7, n_c)) * N * N / (2 * tc_steps))
            # the steps below 128 rows: on-the-fly Toeplitz products on the CUDA cores
            small = [k for k in range(n_c) if k < 7]
            alg["k_toeplitz_rows"] = ("flop", 2.0 * 8.0 * sum(1 << k for k in small) * N * N / (2 * len(small)))
    hbm_bytes_step, hbm_ms_step = 0.0, 0.0
    for name, (n, ms) in prof.items():
        kind, per = alg.get(name, (None, 0.0))
        if kind == "byte":
            hbm_bytes_step += per * n / steps
            hbm_ms_step += ms / steps
    if wl["unit"] == "GB/s":
        value = replica_rate(hbm_bytes_step * steps, world, total_s) / 1e9
        e2e_value = replica_rate(hbm_bytes_step * len(e2e_times), world, e2e_total) / 1e9
    else:
        value = replica_rate(steps, world, total_s)
        e2e_value = replica_rate(len(e2e_times), world, e2e_total)
    out = {
        "workload": workload, "desc": wl["desc"] + ("; postselected solve (hhl_solve_postselected)" if postselected else ""),
        "precision": precision, "value": value, "unit": wl["unit"],
        "solves_per_s": replica_rate(steps, world, total_s),
        "ms_per_step": 1e3 * total_s / steps, "steps": steps, "warmup": warmup,
        "roofline": _roofline(prof, alg, _peaks(), workload + ("_postselected" if postselected else ""), precision,
                              "per-launch CUDA events on the launching stream, second timed loop of the same steps"),
        "gate_gbs": {"bytes_per_step": hbm_bytes_step, "ms_per_step": hbm_ms_step,
                     "achieved_gbs": hbm_bytes_step / (hbm_ms_step / 1e3) / 1e9 if hbm_ms_step else None},
        "profiled_ms_per_step": 1e3 * prof_total_s / steps,
        "breakdown": _breakdown(prof, steps),
        "plan": {"plan_seconds": info["plan_seconds"], "t0": info["t0"], "kappa": info["kappa"],
                 "gemm_flops_per_solve": info["gemm_flops"], "trotter_passes": info["trotter_passes"],
                 "gemm_impl": ["auto", "simt", "tcgen05"][info["gemm_impl"]] if wl["expm"] == "dense" else None},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": wl["unit"], "h2d_bytes_per_step": N * (16 if postselected else 8),
                "d2h_bytes_per_step": (4 + 2 * N) * 8 + 8 + (0 if postselected else 8)},
        "gpu_launches": launches,
        "result": {"p_success": m["p_success"], "eps": e},
    }
    del st, flush
    plan.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank: int, world: int, local_rank: int) -> None:
    import torch

    import paper_2307_00391_gb300 as pkg
    from paper_2307_00391_gb300 import build as _b

    torch.cuda.set_device(local_rank)
    if rank == 0:
        _b.build()
    if world > 1:
        torch.distributed.barrier()
    pkg.load()
    wl = WORKLOADS[args.workload]
    main = solve_block(pkg, args.workload, args.precision, args.gemm, args.steps, args.warmup, world, local_rank,
                       postselected=args.postselected)
    sub = {}
    if args.workload == DEFAULT_WORKLOAD and args.sub == "all" and not args.postselected:
        # the rest of the metric, each timed with CUDA events and with its own roofline: the same
        # 32-qubit solve at the paper's FP64 precision, the dense tensor-core solve of the 23-qubit
        # Couette system, and the batched solves/s at 1e-6 fidelity
        sub["poiseuille_2p18_postselected"] = solve_block(pkg, "poiseuille_2p18", "c64", "auto", args.steps,
                                                          args.warmup, world, local_rank, postselected=True)
        sub["poiseuille_2p18_c128"] = solve_block(pkg, "poiseuille_2p18", "c128", "auto", min(args.steps, 5),
                                                  min(args.warmup, 3), world, local_rank, e2e_steps=3)
        sub["couette_1024"] = solve_block(pkg, "couette_1024", "c64", "auto", args.steps, args.warmup, world,
                                          local_rank)
        sub["couette_1024_postselected"] = solve_block(pkg, "couette_1024", "c64", "auto", args.steps, args.warmup,
                                                       world, local_rank, postselected=True)
        sub["batch_256"] = batch_block(pkg, args, world, local_rank)
    if rank != 0:
        return
    cpu = _cpu_baseline_subprocess(args.workload) if (world == 1 and not args.no_cpu_baseline) else None
    out = {
        "metric": METRIC, "value": main["value"], "unit": wl["unit"], "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "c64" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "precision": args.precision,
                   "expm": wl["expm"], "gemm_impl": main["plan"]["gemm_impl"],
                   "uncompute": "postselect-early",
                   "readout": "postselected solve" if args.postselected else "full final state",
                   "l2": "flushed between timed steps (256 MiB write outside the events)",
                   "parallelism": f"replicas x{world}"},
        "roofline": main["roofline"],
        "gate_gbs": dict(main["gate_gbs"], peak_gbs=_peaks().get("hbm_gbs")),
        "profiled_ms_per_step": main["profiled_ms_per_step"],
        "breakdown": main["breakdown"],
        "plan": main["plan"],
        "clocks": main["clocks"],
        "e2e": main["e2e"],
        "gpu_launches": main["gpu_launches"],
        "cpu_baseline": cpu,
        "result": main["result"],
    }
    if sub:
        out["sub"] = sub
    print(json.dumps(out))


def run_qft(args, rank: int, world: int, local_rank: int) -> None:
    """The Fig. 1c gate benchmark: QFT then inverse QFT on whole registers of random states
    (seeded, on the device). value = algorithmic bytes / time, where each of the two
    transforms must read and write every amplitude once."""
    import torch

    import paper_2307_00391_gb300 as pkg
    from paper_2307_00391_gb300 import build as _b

    torch.cuda.set_device(local_rank)
    if rank == 0:
        _b.build()
    if world > 1:
        torch.distributed.barrier()
    pkg.load()
    wl = WORKLOADS[args.workload]
    n, states = wl["n"], wl["states"]
    dt = torch.complex64 if args.precision == "c64" else torch.complex128
    amp_bytes = 8 if args.precision == "c64" else 16
    st = torch.empty(states << n, dtype=dt, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(230700391 + rank)
    torch.view_as_real(st).normal_(generator=gen)
    view = st.view(states, 1 << n)
    view /= torch.linalg.vector_norm(view, dim=1, keepdim=True)
    x0 = view[:, :4].clone()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()

    def step():
        pkg.qft_whole(st, n, states, 0, stream=stream)
        pkg.qft_whole(st, n, states, 1, stream=stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    pkg.profile_reset()
    pkg.profile_enable(True)
    launches0 = pkg.kernel_launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    launches = pkg.kernel_launch_count() - launches0
    pkg.profile_enable(False)
    prof = pkg.profile_read()
    total_s = sum(a.elapsed_time(c) for a, c in evs) / 1e3
    total_s = max_over_ranks(total_s, world)
    step_bytes = 4.0 * states * (1 << n) * amp_bytes
    # QFT-IQFT is the identity: the state after all steps is the input up to rounding
    drift = float((view[:, :4] - x0).abs().max().item())
    # end to end: the states from pinned host memory, both transforms, the states back
    host = torch.empty(states << n, dtype=dt, pin_memory=True)
    host.copy_(st)
    e2e_t = []
    for _ in range(max(3, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            st.copy_(host, non_blocking=True)
            step()
            host.copy_(st, non_blocking=True)
        stream.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    passes = sum(c for c, _ in prof.values())
    per_launch = step_bytes * args.steps / passes if passes else 0.0
    breakdown = {k: {"launches_per_step": c / args.steps, "ms_per_step": ms / args.steps}
                 for k, (c, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    peaks = _peaks()
    roofline = None
    if dom is not None:
        c, ms = prof[dom]
        achieved = per_launch / (ms / c / 1e3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None, "peak_source": "measured HBM copy (MEASURED_PEAKS.json)",
                    "algorithmic_per_launch": per_launch, "avg_launch_ms": ms / c,
                    "note": "the two transforms' minimum bytes spread evenly over their passes"}
    cpu = _cpu_baseline_subprocess(args.workload) if (world == 1 and not args.no_cpu_baseline) else None
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": replica_rate(step_bytes * args.steps, world, total_s) / 1e9, "unit": wl["unit"],
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "c64" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "precision": args.precision,
                       "l2": "inputs larger than L2" if states * (1 << n) * amp_bytes > (256 << 20) else "L2-resident",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "breakdown": breakdown, "clocks": clk.summary(),
            "e2e": {"value": replica_rate(step_bytes * len(e2e_t), world, max_over_ranks(sum(e2e_t), world)) / 1e9,
                    "unit": wl["unit"],
                    "h2d_bytes_per_step": states * (1 << n) * amp_bytes,
                    "d2h_bytes_per_step": states * (1 << n) * amp_bytes},
            "gpu_launches": launches, "cpu_baseline": cpu,
            "result": {"max_drift_after_all_steps": drift}}))


def batch_block(pkg, args, world: int, local_rank: int) -> dict:
    """The batched engine: one step = one replay of the graph over all 256 instances (complex64,
    autotuned GEMM choices); each replay's device status is checked right after its timed
    events. Then the per-kernel breakdown from an eager launch of the same work, the end-to-end
    rate with host buffers, and every instance again through the complex128 single-instance
    plan path (CUDA-core FP64 GEMMs) on the same GPU: that loop is timed with CUDA events (the
    FP64 single-instance solves/s) and is the reference of the fidelity count
    F = |<xhat_c128 | xhat_c64>| >= 1 - 1e-6 over all instances.
    With N ranks every rank runs a batch of 256 instances of its own (independent problems drawn
    with the rank as seed offset; rank 0's batch is the one-GPU batch); the whole-job rate is all
    ranks' instances over the slowest rank's time and the fidelity counts are summed."""
    import numpy as np
    import torch

    from paper_2307_00391_gb300 import autotune
    from synth_inputs import batch_instances, walls

    wl = WORKLOADS["batch_256"]
    rank = torch.distributed.get_rank() if world > 1 else 0
    inst = batch_instances(wl["count"], seed_offset=rank)
    probs = []
    for it in inst:
        diag, off = pkg.laplacian(1 << it["n_s"])
        probs.append(dict(n_sys_qubits=it["n_s"], n_clock=it["n_c"], diag=diag, off=off, nu=0.1,
                          walls=walls(it["flow"]), t0_rule="power_law", t0_scale=it["t0_mult"]))
    choices = autotune.choices_for([(it["n_s"], it["n_c"]) for it in inst])
    t_plan = time.perf_counter()
    batch = pkg.HHLBatch(probs, gemm_choice=choices, streams=args.streams)
    t_plan = time.perf_counter() - t_plan
    binf = batch.info
    stream = torch.cuda.Stream()
    b_dev = torch.tensor(batch.pack_rhs([it["b"] for it in inst]), device="cuda")
    out = torch.empty(binf["out_doubles"], dtype=torch.float64, device="cuda")
    eps = torch.empty(batch.count, dtype=torch.float64, device="cuda")
    for _ in range(max(args.warmup, 1)):
        batch.run(b_dev, out, eps, stream=stream)         # checked runs
    launches_per_run = batch.info["graph_launches"]
    steps = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(steps):
            evs[i][0].record(stream)
            batch.run(b_dev, out, eps, stream=stream, check_status=False)
            evs[i][1].record(stream)
            batch.status(stream)                             # outside the events
        torch.cuda.synchronize()
    total_s = max_over_ranks(sum(a.elapsed_time(c) for a, c in evs) / 1e3, world)
    res = batch.unpack(out.cpu().numpy())
    # per-kernel times from the same work launched eagerly after the timed region
    pkg.profile_reset()
    pkg.profile_enable(True)
    batch.run_eager(stream=stream)
    stream.synchronize()
    pkg.profile_enable(False)
    prof = pkg.profile_read()
    batch.status(stream)
    b_pin = torch.tensor(batch.pack_rhs([it["b"] for it in inst])).pin_memory()
    e2e = []
    for _ in range(max(2, min(steps, 5))):
        t0 = time.perf_counter()
        batch.run_host(b_pin, stream=stream)
        e2e.append(time.perf_counter() - t0)
    e2e = e2e[1:]
    # GEMM flops of the two trees per instance (2^k rows at step k, both trees); on tcgen05 the
    # steps with 2^k >= 128 of the instances with tiles
    flops = [2.0 * 8.0 * ((1 << it["n_c"]) - 1) * (1 << it["n_s"]) ** 2 for it in inst]
    tc_flops = sum(2.0 * 8.0 * sum(1 << k for k in range(7, it["n_c"])) * (1 << it["n_s"]) ** 2
                   for it, bi in zip(inst, batch.instances) if bi["gemm"])
    # the steps below 128 rows: on-the-fly Toeplitz products on the CUDA cores, every instance
    toep_flops = sum(2.0 * 8.0 * sum(1 << k for k in range(min(7, it["n_c"]))) * (1 << it["n_s"]) ** 2
                     for it in inst)
    batch.close()
    del out, eps, b_dev
    torch.cuda.empty_cache()
    # complex128 single-instance loop over every instance (plans created outside the timing)
    fids, fp64_s, fp64_plan_s = [], 0.0, 0.0
    for i, it in enumerate(inst):
        diag, off = pkg.laplacian(1 << it["n_s"])
        tp = time.perf_counter()
        plan = pkg.HHLPlan(it["n_s"], it["n_c"], diag=diag, off=off, precision="c128", gemm="simt",
                           t0_rule="user", t0=batch.instances[i]["t0"], nu=0.1, walls=walls(it["flow"]))
        st = plan.new_state()
        meas = torch.empty(4 + 2 * (1 << it["n_s"]), dtype=torch.float64, device="cuda")
        ed = torch.empty(1, dtype=torch.float64, device="cuda")
        bd = torch.tensor(it["b"].astype(np.complex128), device="cuda")
        torch.cuda.synchronize()
        fp64_plan_s += time.perf_counter() - tp
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.prepare_rhs(bd, st)
        plan.apply_circuit(st)
        plan.measure_async(st, meas)
        plan.dissipation_async(st, ed)
        e1.record()
        torch.cuda.synchronize()
        fp64_s += e0.elapsed_time(e1) / 1e3
        m = meas.cpu().numpy()
        x128 = m[4::2] + 1j * m[5::2]
        fids.append(float(abs(np.vdot(x128, res[i]["xhat"]))))
        del st, meas, ed, bd
        plan.close()
    torch.cuda.empty_cache()
    peaks = _peaks()
    # roofline of the dominant kernel (by its summed time in the eager launch)
    roofline = None
    models = {"k_ctrl_gemm_tc": (tc_flops, "tensor", peaks.get("bf16_tflops", 1900.0),
                                 "FP16 dense = measured bf16 burst (same nominal rate); 3 MMAs per algorithmic product"),
              "k_toeplitz_rows": (toep_flops, "alu", _fp32_simt_peak_tflops(peaks.get("sm_max_mhz", 2070.0)),
                                  "FP32 CUDA cores: 152 SMs x 128 lanes x 2 flop x max SM clock")}
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    if dom in models:
        fl, bound, peak, src = models[dom]
        n, ms = prof[dom]
        achieved = fl / (ms / 1e3) / 1e12
        roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None, "peak_source": src,
                    "algorithmic_per_launch": fl / n, "avg_launch_ms": ms / n,
                    "timing": "eager launch of the batch right after the timed region (per-launch events; "
                              "up to 8 worker streams share the GPU, so a launch's time includes its neighbours')"}
    elif dom is not None:
        roofline = {"kernel": dom, "bound": None, "note": "no algorithmic work model for this kernel"}
    ok = [f for f in fids if f >= 1 - 1e-6]
    n_inst = sum_over_ranks(float(len(fids)), world)  # every rank's batch
    n_ok = sum_over_ranks(float(len(ok)), world)
    f_min = -max_over_ranks(-min(fids), world)
    fp64_slowest = max_over_ranks(fp64_s, world)
    return {
        "workload": "batch_256", "desc": wl["desc"], "precision": "c64", "value": replica_rate(wl["count"] * steps, world, total_s),
        "unit": wl["unit"], "ms_per_step": 1e3 * total_s / steps, "steps": steps, "warmup": max(args.warmup, 1),
        "config": {"instances": wl["count"], "streams": binf["streams"],
                   "gemm_choices": "tuning.json" if choices else "size rule",
                   "l2": "inputs larger than L2 (all states %.1f GB)" % (binf["state_bytes"] / 1e9)},
        "roofline": roofline,
        "fidelity": {"instances": int(n_inst), "at_1e-6": int(n_ok), "min": f_min,
                     "solves_per_s_at_1e-6": n_ok * steps / total_s,
                     "reference": "complex128 single-instance plan path (CUDA-core FP64 GEMM), same GPU"},
        "fp64_single_instance": {"solves_per_s": n_inst / fp64_slowest, "seconds": fp64_slowest, "plan_seconds": fp64_plan_s,
                                 "timing": "CUDA events around each instance's prepare, circuit, measure and "
                                           "dissipation (plans outside), every instance"},
        "breakdown": {name: {"launches": n, "ms": ms} for name, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        "plan": {"plan_seconds": t_plan, "gemm_flops_per_run": binf["gemm_flops"],
                 "state_bytes": binf["state_bytes"], "workspace_bytes": binf["workspace_bytes"]},
        "clocks": clk.summary(),
        "e2e": {"value": replica_rate(wl["count"] * len(e2e), world, max_over_ranks(sum(e2e), world)),
                "unit": wl["unit"], "h2d_bytes_per_step": binf["b_doubles"] * 8,
                "d2h_bytes_per_step": (binf["out_doubles"] + wl["count"]) * 8},
        "gpu_launches": launches_per_run * steps,
    }


def run_batch(args, rank: int, world: int, local_rank: int) -> None:
    """--workload batch_256 on its own: the batch block as the JSON line."""
    import torch

    import paper_2307_00391_gb300 as pkg
    from paper_2307_00391_gb300 import build as _b

    torch.cuda.set_device(local_rank)
    if rank == 0:
        _b.build()
    if world > 1:
        torch.distributed.barrier()
    pkg.load()
    blk = batch_block(pkg, args, world, local_rank)
    if rank != 0:
        return
    wl = WORKLOADS["batch_256"]
    cpu = None if (world > 1 or args.no_cpu_baseline) else _cpu_baseline_subprocess(args.workload)
    print(json.dumps({
        "metric": METRIC, "value": blk["value"], "unit": wl["unit"], "n_gpus": world, "steps": blk["steps"],
        "warmup": blk["warmup"], "ms_per_step": blk["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(blk["config"], workload=args.workload, desc=wl["desc"], precision="c64",
                       parallelism=f"replicas x{world}"),
        "roofline": blk["roofline"], "fidelity": blk["fidelity"], "fp64_single_instance": blk["fp64_single_instance"],
        "breakdown": blk["breakdown"], "plan": blk["plan"], "clocks": blk["clocks"], "e2e": blk["e2e"],
        "gpu_launches": blk["gpu_launches"], "cpu_baseline": cpu}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--sub", default="all", choices=["all", "none"],
                    help="default workload only: add the complex128, Couette and batch sub-objects")
    ap.add_argument("--precision", default="c64", choices=["c64", "c128"])
    ap.add_argument("--gemm", default="auto", choices=["auto", "simt", "tcgen05"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--postselected", action="store_true",
                    help="Strang-Trotter workloads: time the postselected solve (hhl_solve_postselected)")
    ap.add_argument("--streams", type=int, default=8, help="worker streams of the batched engine")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if WORKLOADS[args.workload].get("kind") == "batch":
            run_batch(args, rank, world, local_rank)
        elif WORKLOADS[args.workload].get("kind") == "qft":
            run_qft(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
