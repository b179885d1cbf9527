"""The multi-process path of bench.py on CPU: two gloo ranks, each an independent replica;
the job time is the slowest rank's and the rate counts every rank's work (no GPU). The batch
block gives every rank a batch of its own (the rank as seed offset) and sums the ranks'
fidelity counts."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        own = [1.5, 2.5][rank]                        # this rank's timed seconds
        slowest = bench.max_over_ranks(own, world, device="cpu")
        rate = bench.replica_rate(10.0, world, slowest)  # 10 units per rank
        ok = bench.sum_over_ranks([250.0, 256.0][rank], world, device="cpu")   # instances at F >= 1 - 1e-6
        f_min = -bench.max_over_ranks(-[0.9999991, 0.9999999][rank], world, device="cpu")
        from synth_inputs import batch_instances
        first_b = batch_instances(4, seed_offset=rank)[0]["b"]
        out.put((rank, slowest, rate, ok, f_min, first_b))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_report_the_slowest_time_and_the_summed_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=10) for _ in range(2)), key=lambda r: r[0])
    for _, slowest, rate, ok, f_min, _b in res:
        assert slowest == pytest.approx(2.5)
        assert rate == pytest.approx(2 * 10.0 / 2.5)
        assert ok == 506.0
        assert f_min == pytest.approx(0.9999991)
    # every rank's batch is its own; rank 0's is the one-GPU batch
    from synth_inputs import batch_instances
    b0, b1 = res[0][5], res[1][5]
    assert not (len(b0) == len(b1) and (b0 == b1).all())
    assert (b0 == batch_instances(4)[0]["b"]).all()


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.replica_rate(4.0, 1, 2.0) == 2.0
    assert bench.sum_over_ranks(7.0, 1) == 7.0
