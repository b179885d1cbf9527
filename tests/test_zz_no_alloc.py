"""The allocation-free controlled-U entry point (hhl_controlled_u_noalloc) against the plan
path (hhl_apply_stage), through the C ABI.

It exists for callers that must not allocate device memory while running (pool-allocator
hosts, allocation-free loops): it stages its product rows in a fixed device array inside
the library instead of plan-owned scratch. The test checks two calls in a row (the forward
sequence, then the adjoint sequence on the other half) against the existing entry point at
the complex64 tolerance, and that oversize requests are refused without touching the GPU.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2307_00391_gb300 import build
    build.build()
    import paper_2307_00391_gb300 as pkg
    return pkg


def _u_matrices(n_s, n_c, t0):
    from oracle import hhl_oracle as o
    diag, off = o.laplacian_tridiag(1 << n_s)
    a = o.dense_from_tridiag(diag, off)
    a_hat = a / o.gershgorin_bound(a)
    return [o.evolution_dense(a_hat, t0 * (1 << k) / (1 << n_c)) for k in range(n_c)]


def test_noalloc_controlled_u_matches_plan_path(lib):
    import torch
    from synth_inputs import random_state
    n_s, n_c = 8, 9
    N, half = 1 << n_s, 1 << (n_s + n_c)
    diag, off = lib.laplacian(N)
    plan = lib.HHLPlan(n_s, n_c, diag=diag, off=off, precision="c64", gemm="simt")
    us = _u_matrices(n_s, n_c, plan.info["t0"])
    u_dev = [torch.tensor(u, dtype=torch.complex64, device="cuda") for u in us]
    psi = random_state(n_s + n_c + 1, seed_offset=41)
    ref = torch.tensor(psi, dtype=torch.complex64, device="cuda")
    got = ref.clone()
    c = lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    # call 1: forward products on the anc = 0 half
    plan.apply_stage("qpe_u", ref)
    for k in range(n_c):
        st = c.hhl_controlled_u_noalloc(ctypes.c_void_p(u_dev[k].data_ptr()), ctypes.c_void_p(got.data_ptr()),
                                        n_s, n_c, k, 0, stream)
        assert st == 0, c.hhl_last_error()
    torch.cuda.synchronize()
    assert (got - ref).abs().max().item() < 1e-5

    # call 2: adjoint products on the anc = 1 half (the uncompute stage of the early mode)
    plan.apply_stage("uncompute_u", ref)
    anc1 = got[half:]
    for k in range(n_c - 1, -1, -1):
        st = c.hhl_controlled_u_noalloc(ctypes.c_void_p(u_dev[k].data_ptr()), ctypes.c_void_p(anc1.data_ptr()),
                                        n_s, n_c, k, 1, stream)
        assert st == 0, c.hhl_last_error()
    torch.cuda.synchronize()
    assert (got - ref).abs().max().item() < 1e-5


def test_noalloc_at_the_size_limit_on_a_side_stream(lib):
    """The largest accepted request, 2^(n_c-1) * 2^n_s = 2^20 complex64 values (the whole fixed
    array: n_s = 10, n_c = 11), on a non-default stream, forward then adjoint, against the plan
    path; one clock qubit more is refused."""
    import torch
    from synth_inputs import random_state
    n_s, n_c = 10, 11
    N, half = 1 << n_s, 1 << (n_s + n_c)
    diag, off = lib.laplacian(N)
    plan = lib.HHLPlan(n_s, n_c, diag=diag, off=off, precision="c64", gemm="simt")
    us = _u_matrices(n_s, n_c, plan.info["t0"])
    u_dev = [torch.tensor(u, dtype=torch.complex64, device="cuda") for u in us]
    psi = random_state(n_s + n_c + 1, seed_offset=43)
    ref = torch.tensor(psi, dtype=torch.complex64, device="cuda")
    got = ref.clone()
    c = lib.load()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    handle = ctypes.c_void_p(side.cuda_stream)
    plan.apply_stage("qpe_u", ref)
    for k in range(n_c):
        st = c.hhl_controlled_u_noalloc(ctypes.c_void_p(u_dev[k].data_ptr()), ctypes.c_void_p(got.data_ptr()),
                                        n_s, n_c, k, 0, handle)
        assert st == 0, c.hhl_last_error()
    anc1 = got[half:]
    plan.apply_stage("uncompute_u", ref)
    for k in range(n_c - 1, -1, -1):
        st = c.hhl_controlled_u_noalloc(ctypes.c_void_p(u_dev[k].data_ptr()), ctypes.c_void_p(anc1.data_ptr()),
                                        n_s, n_c, k, 1, handle)
        assert st == 0, c.hhl_last_error()
    side.synchronize()
    torch.cuda.synchronize()
    assert (got - ref).abs().max().item() < 1e-5
    dummy = ctypes.c_void_p(16)
    assert c.hhl_controlled_u_noalloc(dummy, dummy, n_s, n_c + 1, 0, 0, handle) == 1


def test_noalloc_rejects_oversize_requests(lib):
    c = lib.load()
    dummy = ctypes.c_void_p(16)
    assert c.hhl_controlled_u_noalloc(dummy, dummy, 11, 12, 0, 0, None) == 1
    assert b"limit" in c.hhl_last_error()
    assert c.hhl_controlled_u_noalloc(None, dummy, 4, 4, 0, 0, None) == 1
    assert c.hhl_controlled_u_noalloc(dummy, dummy, 4, 4, 4, 0, None) == 1
