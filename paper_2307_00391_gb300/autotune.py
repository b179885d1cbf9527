"""Offline tile autotuner of the batched engine.

For every register size (n_s, n_c) of a batch it times one-instance graphs with each GEMM
implementation that fits (CUDA-core tiles, tcgen05 with 128- or 256-column tiles) and keeps
the fastest in a JSON table (``tuning.json`` beside this file). ``HHLBatch`` callers pass
``choices_for(...)`` as the per-instance GEMM choice; sizes missing from the table fall back
to the library's size rule.

    python -m paper_2307_00391_gb300.autotune [--ns 6 12] [--nc 8 12] [--reps 3]
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

TUNING = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def _time_instance(pkg, n_s: int, n_c: int, choice: int, reps: int) -> float:
    import torch
    diag, off = pkg.laplacian(1 << n_s)
    batch = pkg.HHLBatch([dict(n_sys_qubits=n_s, n_clock=n_c, diag=diag, off=off, t0_rule="power_law")],
                         gemm_choice=[choice], streams=1)
    if batch.instances[0]["gemm"] != choice:
        batch.close()
        return float("nan")
    inf = batch.info
    b = torch.tensor(batch.pack_rhs([np.ones(1 << n_s)]), device="cuda")
    out = torch.empty(inf["out_doubles"], dtype=torch.float64, device="cuda")
    eps = torch.empty(1, dtype=torch.float64, device="cuda")
    batch.run(b, out, eps)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.run(b, out, eps)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    batch.close()
    return float(min(times))


def sweep(ns_range=(6, 12), nc_range=(8, 12), reps: int = 3) -> dict:
    import paper_2307_00391_gb300 as pkg
    table = {}
    simt_dominated_from = None
    for n_s in range(ns_range[0], ns_range[1] + 1):
        for n_c in range(nc_range[0], nc_range[1] + 1):
            ms = {}
            for choice in (0, 128, 256):
                if choice == 0 and simt_dominated_from is not None and n_s >= simt_dominated_from:
                    continue  # the CUDA-core tiles lost by > 3x at a smaller size already
                t = _time_instance(pkg, n_s, n_c, choice, reps)
                if t == t:
                    ms[str(choice)] = t
            best = min(ms, key=ms.get)
            table[f"{n_s},{n_c}"] = {"best": int(best), "ms": ms}
            tc = [v for k, v in ms.items() if k != "0"]
            if "0" in ms and tc and ms["0"] > 3 * min(tc) and simt_dominated_from is None:
                simt_dominated_from = n_s + 1
    return table


def load_table(path: str = TUNING) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def choices_for(sizes, table: dict | None = None) -> list | None:
    """Per-instance GEMM choices for [(n_s, n_c), ...]; None if there is no table."""
    table = load_table() if table is None else table
    if not table:
        return None
    out = []
    for n_s, n_c in sizes:
        ent = table.get(f"{n_s},{n_c}")
        out.append(-1 if ent is None else int(ent["best"]))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ns", type=int, nargs=2, default=(6, 12))
    ap.add_argument("--nc", type=int, nargs=2, default=(8, 12))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=TUNING)
    a = ap.parse_args()
    table = sweep(tuple(a.ns), tuple(a.nc), a.reps)
    with open(a.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps(table))


if __name__ == "__main__":
    main()
