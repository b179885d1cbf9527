"""Host-side checks of the C ABI that need no GPU: the library loads, exports every entry
point include/hhl.h declares, and rejects invalid requests with status codes before any
CUDA call is made."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_00391_gb300 import build
    build.build()
    from paper_2307_00391_gb300 import _ffi
    return _ffi.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hhl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hhl_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2307_00391_gb300 import _ffi
    syms = declared_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(lib, s), s
    bound = {name for name, _, _ in _ffi.SIGNATURES}
    assert set(syms) == bound, set(syms) ^ bound


def test_version_status_strings_and_defaults(lib):
    from paper_2307_00391_gb300 import _ffi
    assert lib.hhl_api_version() == 1
    for code in range(9):
        assert lib.hhl_status_string(code)
    p = _ffi.Params()
    lib.hhl_params_default(ctypes.byref(p))
    assert (p.n_clock, p.t0_rule, p.precision, p.expm_mode, p.full_uncompute) == (6, 2, 32, 0, 0)


def _plan(lib, prob, par):
    h = ctypes.c_void_p()
    st = lib.hhl_plan_create(ctypes.byref(prob), ctypes.byref(par), ctypes.byref(h))
    return st, lib.hhl_last_error().decode()


def _tridiag(n_s, diag=None, off=None):
    from paper_2307_00391_gb300 import _ffi
    n = 1 << n_s
    d = np.full(n, 2.0) if diag is None else diag
    o = np.full(n - 1, -1.0) if off is None else off
    prob = _ffi.Problem()
    prob.kind = _ffi.MATRIX_TRIDIAG
    prob.n_sys_qubits = n_s
    prob.diag = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    prob.off = o.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return prob, (d, o)


def test_invalid_arguments_are_rejected_on_the_host(lib):
    from paper_2307_00391_gb300 import _ffi
    par = _ffi.Params()
    lib.hhl_params_default(ctypes.byref(par))
    prob, keep = _tridiag(4)
    h = ctypes.c_void_p()
    assert lib.hhl_plan_create(None, ctypes.byref(par), ctypes.byref(h)) == 1
    for field, value in (("n_clock", 0), ("n_clock", 14), ("precision", 16), ("expm_mode", 7),
                         ("t0_rule", 9), ("gemm_impl", 5)):
        bad = _ffi.Params.from_buffer_copy(par)
        setattr(bad, field, value)
        st, msg = _plan(lib, prob, bad)
        assert st == 1, (field, st, msg)
        assert msg
    user = _ffi.Params.from_buffer_copy(par)
    user.t0_rule = _ffi.T0_USER
    user.t0 = -1.0
    assert _plan(lib, prob, user)[0] == 1
    big, keep2 = _tridiag(13)
    assert _plan(lib, big, par)[0] == 1          # dense mode limited to 12 system qubits
    nan_prob, keep3 = _tridiag(3, diag=np.array([2.0, np.nan, 2, 2, 2, 2, 2, 2]))
    assert _plan(lib, nan_prob, par)[0] == 7
    tc = _ffi.Params.from_buffer_copy(par)
    tc.gemm_impl = _ffi.GEMM_TCGEN05
    tc.precision = _ffi.PREC_C128
    assert _plan(lib, prob, tc)[0] == 8


def test_matrix_property_errors(lib):
    from paper_2307_00391_gb300 import _ffi
    par = _ffi.Params()
    lib.hhl_params_default(ctypes.byref(par))
    # singular: [[1, 1], [1, 1]] as a tridiagonal 2 x 2
    sing, k1 = _tridiag(1, diag=np.array([1.0, 1.0]), off=np.array([1.0]))
    assert _plan(lib, sing, par)[0] == 3
    zero, k2 = _tridiag(2, diag=np.zeros(4), off=np.zeros(3))
    assert _plan(lib, zero, par)[0] == 3
    # indefinite: diag (1, -1)
    indef, k3 = _tridiag(1, diag=np.array([1.0, -1.0]), off=np.array([0.0]))
    assert _plan(lib, indef, par)[0] == 8
    # dense, not Hermitian
    a = np.array([[2.0, 1.0], [0.5, 2.0]])
    prob = _ffi.Problem()
    prob.kind = _ffi.MATRIX_DENSE
    prob.n_sys_qubits = 1
    prob.dense_re = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert _plan(lib, prob, par)[0] == 2
    # Trotter mode needs a Toeplitz tridiagonal
    tro = _ffi.Params.from_buffer_copy(par)
    tro.expm_mode = _ffi.EXPM_TROTTER
    nt, k4 = _tridiag(3, diag=np.arange(1.0, 9.0) + 4, off=np.full(7, -1.0))
    assert _plan(lib, nt, tro)[0] == 8


def test_null_handles_and_qft_arguments(lib):
    assert lib.hhl_apply_circuit(None, None, None) == 1
    assert lib.hhl_measure(None, None, None, None, None) == 1
    assert lib.hhl_dissipation(None, None, None, None, None) == 1
    assert lib.hhl_prepare_rhs(None, None, None, None) == 1
    assert lib.hhl_apply_qft(None, 10, 0, 4, 0, 32, None) == 1
    buf = ctypes.c_void_p(1)
    assert lib.hhl_apply_qft(buf, 10, 8, 4, 0, 32, None) == 1   # lo + m > n
    assert lib.hhl_apply_qft(buf, 40, 0, 4, 0, 32, None) == 1
    assert lib.hhl_apply_qft(buf, 20, 0, 14, 0, 32, None) == 1
    assert lib.hhl_apply_qft(buf, 20, 0, 4, 0, 33, None) == 1
    assert lib.hhl_state_bytes(None) == 0
    assert lib.hhl_sample(None, None, None, 0, None, None) == 1


def test_empty_and_negative_counts_are_rejected(lib):
    """An empty batch and a negative shot count are argument errors, found before any device
    work."""
    from paper_2307_00391_gb300 import _ffi
    par = _ffi.Params()
    lib.hhl_params_default(ctypes.byref(par))
    prob, keep = _tridiag(3)
    out = ctypes.c_void_p()
    assert lib.hhl_batch_create(ctypes.byref(prob), ctypes.byref(par), 0, None, 0, ctypes.byref(out)) == 1
    assert lib.hhl_batch_create(ctypes.byref(prob), ctypes.byref(par), -3, None, 0, ctypes.byref(out)) == 1
    assert not out.value
    fake = ctypes.c_void_p(1)
    assert lib.hhl_sample(fake, fake, None, -1, fake, None) == 1
    assert lib.hhl_sample(fake, fake, None, 5, fake, None) == 1      # shots without uniforms


def test_host_fault_injection_plan():
    """HHL_FAULT=plan makes hhl_plan_create fail after validation, on the host."""
    code = (
        "import ctypes, numpy as np\n"
        "from paper_2307_00391_gb300 import _ffi\n"
        "lib = _ffi.load()\n"
        "p = _ffi.Params(); lib.hhl_params_default(ctypes.byref(p))\n"
        "d = np.full(4, 2.0); o = np.full(3, -1.0)\n"
        "pr = _ffi.Problem(); pr.kind = 0; pr.n_sys_qubits = 2\n"
        "pr.diag = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))\n"
        "pr.off = o.ctypes.data_as(ctypes.POINTER(ctypes.c_double))\n"
        "h = ctypes.c_void_p()\n"
        "print(lib.hhl_plan_create(ctypes.byref(pr), ctypes.byref(p), ctypes.byref(h)), lib.hhl_last_error().decode())\n")
    env = dict(os.environ, HHL_FAULT="plan", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("1 injected planner failure"), out.stdout


def test_contract_names_reject_invalid_requests_on_the_host(lib):
    """The hot-path contract's names (hhl_plan, hhl_batch_plan) are the library's calls: the
    same host validation before any CUDA call."""
    from paper_2307_00391_gb300 import _ffi
    par = _ffi.Params()
    lib.hhl_params_default(ctypes.byref(par))
    prob, keep = _tridiag(4)
    h = ctypes.c_void_p()
    assert lib.hhl_plan(None, ctypes.byref(par), ctypes.byref(h)) == 1
    bad = _ffi.Params.from_buffer_copy(par)
    bad.n_clock = 0
    assert lib.hhl_plan(ctypes.byref(prob), ctypes.byref(bad), ctypes.byref(h)) == 1
    assert lib.hhl_batch_plan(None, ctypes.byref(par), 1, ctypes.byref(h)) == 1
    assert lib.hhl_batch_plan(ctypes.byref(prob), ctypes.byref(par), 0, ctypes.byref(h)) == 1


@pytest.mark.parametrize("form", ["ae", "swap"])
def test_qpp_host_builders_against_the_oracle(lib, form):
    """The library's host builders of the QPP transform (iterate, rotation table, start state,
    projection) against the oracle's independent constructions (App. D)."""
    from oracle import qpp_oracle as q
    from paper_2307_00391_gb300 import qpp
    rng = np.random.default_rng(11)
    for a in ((1, 2, 3) if form == "ae" else (1, 2)):
        z = rng.standard_normal(1 << a)
        z /= np.linalg.norm(z)
        if form == "ae":
            np.testing.assert_allclose(qpp.iterate(z), q.amplitude_estimation_iterate(z), atol=1e-14)
        else:
            np.testing.assert_allclose(qpp.swap_iterate(z), q.swap_test_iterate(z), atol=1e-14)
            np.testing.assert_allclose(qpp.swap_register_state(z), q.swap_test_prepare(z).real, atol=1e-15)
    if form == "ae":
        np.testing.assert_allclose(qpp.rotation_table(7, 0.9), q.squaring_angles(7, 0.9), atol=1e-15)
    else:
        np.testing.assert_allclose(qpp.swap_rotation_table(7, 0.9), q.swap_squaring_angles(7, 0.9), atol=1e-15)
    # the projection: a postselected vector built from known address amplitudes w_s times each
    # block's start state returns w_s (the start states are orthonormal per block)
    a = 2
    z = rng.standard_normal(1 << a)
    z /= np.linalg.norm(z)
    n = 1 << a
    f = 0 if form == "ae" else 1
    dim = n * n if form == "ae" else 2 * n ** 3
    b = np.zeros(dim)
    assert lib.hhl_qpp_start_state(ctypes.c_void_p(z.ctypes.data), a, f, ctypes.c_void_p(b.ctypes.data)) == 0
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v = (b.reshape(n, -1) * np.sqrt(n) * w[:, None]).reshape(-1).astype(np.complex128)
    out = np.zeros(2 * n)
    assert lib.hhl_qpp_project(ctypes.c_void_p(v.ctypes.data), ctypes.c_void_p(b.ctypes.data), a, f,
                               ctypes.c_void_p(out.ctypes.data)) == 0
    np.testing.assert_allclose(out[0::2] + 1j * out[1::2], w, atol=1e-14)
    # invalid requests
    assert lib.hhl_qpp_iterate(None, a, f, ctypes.c_void_p(b.ctypes.data)) == 1
    assert lib.hhl_qpp_rotation_table(0, 1.0, f, ctypes.c_void_p(out.ctypes.data)) == 1
    assert lib.hhl_qpp_rotation_table(4, 1.5, f, ctypes.c_void_p(out.ctypes.data)) == 1
