"""The oracle's HHL circuit cut at the library's stage boundaries (test utility).

Uses only oracle primitives, in the order of oracle.hhl_oracle.hhl_circuit; the CPU test
test_stage_cuts_reproduce_whole_circuit checks that the last cut equals hhl_circuit."""
import numpy as np

from oracle import hhl_oracle as o


def problem(flow, n_s):
    from synth_inputs import rhs, walls
    n = 1 << n_s
    diag, off = o.laplacian_tridiag(n)
    return diag, off, rhs(flow, n), walls(flow)


def run_stages(b, n_s, pl, trotter=None):
    """Return dict of complex128 states after: prep, qpe_u, rotated (inverse QFT + RY),
    clock_block (+ QFT), uncompute_u, final_h."""
    n_c = pl["n_clock"]
    n = n_s + n_c + 1
    t_k = [pl["t0"] * (1 << k) / (1 << n_c) for k in range(n_c)]
    ev = None if trotter else [o.evolution_dense(pl["a_hat"], t) for t in t_k]

    def cu(psi, k, adjoint):
        if trotter is None:
            u = ev[k].conj().T if adjoint else ev[k]
            o.apply_register_unitary(psi, n, 0, n_s, u, control=n_s + k)
        else:
            r = o.trotter_steps(t_k[k], trotter["dt"], trotter["r_max"])
            o.apply_trotter_controlled(psi, n, n_s, n_s + k, trotter["diag"], trotter["off"],
                                       -t_k[k] if adjoint else t_k[k], r)

    out = {}
    psi = o.prepare_state(b, n_s, n_c)
    out["prep"] = psi.copy()
    for k in range(n_c):
        cu(psi, k, False)
    out["qpe_u"] = psi.copy()
    o.qft(psi, n, n_s, n_c, inverse=True)
    o.apply_clock_controlled_ry(psi, n_s, n_c, pl["theta"])
    out["rotated"] = psi.copy()
    o.qft(psi, n, n_s, n_c, inverse=False)
    out["clock_block"] = psi.copy()
    for k in range(n_c - 1, -1, -1):
        cu(psi, k, True)
    out["uncompute_u"] = psi.copy()
    for q in range(n_s, n_s + n_c):
        o.apply_1q(psi, n, q, o.H_GATE)
    out["final_h"] = psi.copy()
    return out
