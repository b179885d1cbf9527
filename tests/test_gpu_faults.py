"""Failure detection on the GPU without faulting it: the tcgen05 GEMM's bounded mbarrier waits
run out on purpose (HHL_FAULT=tc_wait makes the producer issue no operand copy and bounds every
wait by about a millisecond, so nothing is in flight when the MMA lane gives up). The call
reports HHL_ERR_TIMEOUT through the status calls, the CUDA context stays usable, and the next
circuit on the same plan or batch is clean again (the flag is cleared when a circuit starts)."""
import numpy as np
import pytest

from oracle import hhl_oracle as o
from tests.oracle_stages import problem

pytestmark = pytest.mark.gpu

TIMEOUT = 6


@pytest.fixture(scope="module")
def hhl():
    import torch
    assert torch.cuda.is_available()
    import paper_2307_00391_gb300 as pkg
    pkg.load()
    return pkg


def test_plan_gemm_wait_runs_out_then_recovers(hhl, monkeypatch):
    import torch
    n_s, n_c = 7, 8                       # 128 rows per controlled product: one 128 x 256 tile row
    diag, off, b, walls = problem("couette", n_s)
    plan = hhl.HHLPlan(n_s, n_c, diag=diag, off=off, precision="c64", gemm="tcgen05", walls=walls)
    assert plan.info["gemm_impl"] == 2
    st = plan.new_state()
    monkeypatch.setenv("HHL_FAULT", "tc_wait")
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)                # launches return; the waits run out on the device
    with pytest.raises(hhl.HHLError) as e:
        plan.status()
    assert e.value.status == TIMEOUT
    with pytest.raises(hhl.HHLError) as e:
        plan.measure(st)
    assert e.value.status == TIMEOUT
    # the context is intact: ordinary work runs
    assert float(torch.ones(4, device="cuda").sum().item()) == 4.0
    monkeypatch.delenv("HHL_FAULT")
    plan.prepare_rhs_host(b, st)
    plan.apply_circuit(st)
    plan.status()                         # the old timeout is not reported again
    m = plan.measure(st)
    pl = o.plan(o.dense_from_tridiag(diag, off), n_c, t0_rule="range_fill")
    ref = o.postselect(o.hhl_circuit(b, n_s, pl), n_s, n_c)
    assert m["p_success"] == pytest.approx(ref["p_success"], rel=1e-4)


def test_batch_gemm_wait_runs_out_then_recovers(hhl, monkeypatch):
    import torch
    from tests.test_gpu_batch import _instances
    probs, bs, choice = _instances([(7, 8, "couette", 1.0, 256), (4, 5, "poiseuille", 1.0, 0)])
    batch = hhl.HHLBatch(probs, gemm_choice=choice, streams=2)
    b_dev = torch.tensor(batch.pack_rhs(bs), device="cuda")
    out = torch.empty(batch.info["out_doubles"], dtype=torch.float64, device="cuda")
    eps = torch.empty(batch.count, dtype=torch.float64, device="cuda")
    # the graph is captured by the first run, with the injected fault in its GEMM launches
    monkeypatch.setenv("HHL_FAULT", "tc_wait")
    batch.run(b_dev, out, eps, check_status=False)
    with pytest.raises(hhl.HHLError) as e:
        batch.status()
    assert e.value.status == TIMEOUT
    with pytest.raises(hhl.HHLError) as e:
        batch.run(b_dev, out, eps)        # checked run: raises
    assert e.value.status == TIMEOUT
    monkeypatch.delenv("HHL_FAULT")
    # the same work launched eagerly (no fault now): the flag is cleared first, the run is clean
    batch.run_eager()
    batch.status()
    res = batch.unpack(out.cpu().numpy())   # the eager run leaves its results in the batch buffers
    del res
    batch.close()
