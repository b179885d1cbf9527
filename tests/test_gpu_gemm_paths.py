"""The launch shapes of the tcgen05 controlled-U GEMM, through the C ABI.

A product of few tiles runs as a stream-K grid whose split tiles a second pass adds up in the
order of the CTAs; a product of many tiles runs one CTA per tile, in clusters of four that
share the B operand by TMA multicast (HHL_TC_CLUSTER=1 turns the sharing off); tree steps
below HHL_TOEP_ROWS rows (128 by default) are on-the-fly Toeplitz products on the CUDA cores.
These tests check that the results do not depend on the run (the split sums are added in a
fixed order), that the clustered tiles equal the unclustered ones bit for bit (the same MMAs
on the same operands), and that moving the Toeplitz threshold keeps the oracle agreement.
The environment switches are read once per process, so the switched runs are child
processes.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import hhl_oracle as o
from tests.oracle_stages import problem, run_stages

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# A child process: one solve of the Couette problem with the given shape, the anc = 1 half
# (full) or the postselected row (postselected) saved to `out`.
_CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
import paper_2307_00391_gb300 as hhl
from tests.oracle_stages import problem
cfg = json.loads({cfg!r})
n_s, n_c = cfg["n_s"], cfg["n_c"]
diag, off, b, walls = problem("couette", n_s)
plan = hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision="c64", gemm="tcgen05", t0_rule="range_fill")
st = plan.new_state()
N = 1 << n_s
if cfg["mode"] == "full":
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    got = st.view(2, 1 << n_c, N)[1].cpu().numpy()
else:
    out = torch.empty(4 + 2 * N, dtype=torch.float64, device="cuda")
    plan.solve_postselected(torch.tensor(np.asarray(b, dtype=np.complex128), device="cuda"), st, out)
    torch.cuda.synchronize()
    got = st.view(2, 1 << n_c, N)[1, 0].cpu().numpy()
np.save(cfg["out"], got)
"""


@pytest.fixture(scope="module")
def hhl():
    import torch
    assert torch.cuda.is_available()
    import paper_2307_00391_gb300 as pkg
    pkg.load()
    return pkg


def _child(tmp_path, env_extra, **cfg):
    out = str(tmp_path / f"out_{len(os.listdir(tmp_path))}.npy")
    cfg["out"] = out
    env = dict(os.environ, **env_extra)
    code = _CHILD.format(root=ROOT, cfg=json.dumps(cfg))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


def _solve(hhl, n_s, n_c, mode):
    import torch
    diag, off, b, walls = problem("couette", n_s)
    plan = hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision="c64", gemm="tcgen05", t0_rule="range_fill")
    assert plan.info["gemm_impl"] == 2
    st = plan.new_state()
    N = 1 << n_s
    if mode == "full":
        plan.prepare_rhs_host(b, st)
        plan.apply_circuit(st)
        return st.view(2, 1 << n_c, N)[1].cpu().numpy()
    out = torch.empty(4 + 2 * N, dtype=torch.float64, device="cuda")
    plan.solve_postselected(torch.tensor(np.asarray(b, dtype=np.complex128), device="cuda"), st, out)
    torch.cuda.synchronize()
    return st.view(2, 1 << n_c, N)[1, 0].cpu().numpy()


@pytest.mark.parametrize("n_s,n_c,mode", [(8, 11, "postselected"),   # tree steps of 2-16 tiles: stream-K
                                          (10, 12, "full")])          # 128 tiles: clusters of four
def test_tc_gemm_results_do_not_depend_on_the_run(hhl, n_s, n_c, mode):
    a = _solve(hhl, n_s, n_c, mode)
    b = _solve(hhl, n_s, n_c, mode)
    assert np.array_equal(a, b)


def test_clustered_tiles_equal_unclustered_tiles(hhl, tmp_path):
    """The 23-qubit Couette solve (QPE and uncompute products of 2048 rows, 128 tiles): one CTA
    per tile with B shared in clusters of four, against the same launch without clusters."""
    with_clusters = _solve(hhl, 10, 12, "full")
    without = _child(tmp_path, {"HHL_TC_CLUSTER": "1"}, n_s=10, n_c=12, mode="full")
    assert np.array_equal(with_clusters, without)


@pytest.mark.parametrize("rows", ["256", "512"])
def test_toeplitz_threshold_keeps_oracle_parity(hhl, tmp_path, rows):
    """Tree steps as Toeplitz products up to 255 or 511 rows (row groups of 16 over several
    blocks) instead of tensor-core products from 128 rows, the postselected row against the
    oracle's whole circuit (complex64)."""
    n_s, n_c = 8, 10
    diag, off, b, walls = problem("couette", n_s)
    pl = o.plan(o.dense_from_tridiag(diag, off), n_c, t0_rule="range_fill")
    v_ref = run_stages(b, n_s, pl)["final_h"].reshape(2, 1 << n_c, 1 << n_s)[1, 0]
    got = _child(tmp_path, {"HHL_TOEP_ROWS": rows}, n_s=n_s, n_c=n_c, mode="postselected")
    assert np.abs(got - v_ref).max() <= 1e-5


def test_toeplitz_cluster_split_matches_oracle_and_repeats(hhl):
    """N = 1024: the tree steps of 4-64 rows take the Toeplitz product with the sum over m
    split across clusters of 4 CTAs (partial tiles added through distributed shared memory in
    rank order); the postselected row against the oracle's whole circuit, and bit for bit
    across two runs."""
    n_s, n_c = 10, 8
    diag, off, b, walls = problem("couette", n_s)
    pl = o.plan(o.dense_from_tridiag(diag, off), n_c, t0_rule="range_fill")
    v_ref = run_stages(b, n_s, pl)["final_h"].reshape(2, 1 << n_c, 1 << n_s)[1, 0]
    a = _solve(hhl, n_s, n_c, "postselected")
    assert np.abs(a - v_ref).max() <= 1e-5
    assert np.array_equal(a, _solve(hhl, n_s, n_c, "postselected"))
