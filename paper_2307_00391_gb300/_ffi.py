"""ctypes declarations of the C ABI in include/hhl.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_uint64, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libhhl.so")

# enums (hhl.h)
HHL_OK = 0
STATUS_NAMES = {0: "HHL_OK", 1: "HHL_ERR_INVALID_ARG", 2: "HHL_ERR_NOT_HERMITIAN", 3: "HHL_ERR_SINGULAR",
                4: "HHL_ERR_OOM", 5: "HHL_ERR_CUDA", 6: "HHL_ERR_TIMEOUT", 7: "HHL_ERR_NUMERIC",
                8: "HHL_ERR_UNSUPPORTED"}
MATRIX_TRIDIAG, MATRIX_DENSE, MATRIX_UNITARY = 0, 1, 2
T0_USER, T0_POWER_LAW, T0_RANGE_FILL = 0, 1, 2
T0_TOTAL, T0_PER_UNIT = 0, 1
EXPM_DENSE, EXPM_TROTTER = 0, 1
PREC_C64, PREC_C128 = 32, 64
GEMM_AUTO, GEMM_SIMT, GEMM_TCGEN05 = 0, 1, 2
STAGE_QPE_U, STAGE_CLOCK_BLOCK, STAGE_UNCOMPUTE_U, STAGE_FINAL_H = 0, 1, 2, 3

_DP = POINTER(c_double)


class Problem(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("n_sys_qubits", c_int32), ("diag", _DP), ("off", _DP),
                ("dense_re", _DP), ("dense_im", _DP), ("nu", c_double), ("wall_lo", c_double),
                ("wall_hi", c_double)]


class Params(ctypes.Structure):
    _fields_ = [("n_clock", c_int32), ("t0_rule", c_int32), ("t0_convention", c_int32),
                ("precision", c_int32), ("t0", c_double), ("C", c_double), ("expm_mode", c_int32),
                ("full_uncompute", c_int32), ("trotter_dt", c_double), ("trotter_steps_max", c_int32),
                ("gemm_impl", c_int32), ("t0_scale", c_double), ("theta_table", _DP), ("signed_clock", c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_sys_qubits", c_int32), ("n_clock", c_int32), ("n_qubits", c_int32),
                ("precision", c_int32), ("expm_mode", c_int32), ("gemm_impl", c_int32),
                ("lambda_ub", c_double), ("lambda_min", c_double), ("lambda_max", c_double),
                ("kappa", c_double), ("t0", c_double), ("C", c_double), ("state_bytes", c_uint64),
                ("table_bytes", c_uint64), ("workspace_bytes", c_uint64), ("gemm_flops", c_double),
                ("trotter_passes", c_int64), ("plan_seconds", c_double), ("trotter_bytes", c_double)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("count", c_int32), ("streams", c_int32), ("state_bytes", c_uint64), ("workspace_bytes", c_uint64),
                ("gemm_flops", c_double), ("graph_launches", c_uint64), ("b_doubles", c_int64),
                ("out_doubles", c_int64)]


class Measurement(ctypes.Structure):
    _fields_ = [("p_success", c_double), ("p_anc1", c_double), ("norm", c_double), ("b_norm", c_double)]


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("hhl_api_version", c_int32, []),
    ("hhl_status_string", c_char_p, [c_int32]),
    ("hhl_last_error", c_char_p, []),
    ("hhl_params_default", None, [POINTER(Params)]),
    ("hhl_plan_create", c_int32, [POINTER(Problem), POINTER(Params), POINTER(c_void_p)]),
    ("hhl_plan", c_int32, [POINTER(Problem), POINTER(Params), POINTER(c_void_p)]),
    ("hhl_plan_destroy", None, [c_void_p]),
    ("hhl_plan_get_info", c_int32, [c_void_p, POINTER(PlanInfo)]),
    ("hhl_state_bytes", c_uint64, [c_void_p]),
    ("hhl_prepare_rhs", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("hhl_prepare_rhs_host", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("hhl_apply_circuit", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("hhl_apply_stage", c_int32, [c_void_p, c_int32, c_void_p, c_void_p]),
    ("hhl_measure_async", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("hhl_solve_postselected", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("hhl_measure", c_int32, [c_void_p, c_void_p, POINTER(Measurement), c_void_p, c_void_p]),
    ("hhl_dissipation_async", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("hhl_dissipation", c_int32, [c_void_p, c_void_p, _DP, c_void_p, c_void_p]),
    ("hhl_batch_create", c_int32, [POINTER(Problem), POINTER(Params), c_int32, c_void_p, c_int32, POINTER(c_void_p)]),
    ("hhl_batch_plan", c_int32, [POINTER(Problem), POINTER(Params), c_int32, POINTER(c_void_p)]),
    ("hhl_batch_destroy", None, [c_void_p]),
    ("hhl_batch_get_info", c_int32, [c_void_p, POINTER(BatchInfo)]),
    ("hhl_batch_instance", c_int32, [c_void_p, c_int32, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32),
                                     POINTER(c_int64), POINTER(c_int64), POINTER(c_double)]),
    ("hhl_batch_run", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("hhl_batch_run_eager", c_int32, [c_void_p, c_void_p]),
    ("hhl_batch_run_host", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("hhl_batch_status", c_int32, [c_void_p, c_void_p]),
    ("hhl_plan_status", c_int32, [c_void_p, c_void_p]),
    ("hhl_mlp_create", c_int32, [POINTER(c_void_p)]),
    ("hhl_mlp_destroy", None, [c_void_p]),
    ("hhl_mlp_set_params", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("hhl_mlp_get_params", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("hhl_mlp_forward", c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    ("hhl_t0_predict", c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    ("hhl_mlp_gradients", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    ("hhl_mlp_train_step", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_float, c_void_p, c_void_p]),
    ("hhl_apply_qft", c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p]),
    ("hhl_qft_whole", c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p]),
    ("hhl_sample", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    ("hhl_prepare_rhs_qsp1", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("hhl_prepare_rhs_qsp2", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    ("hhl_qpp_dissipation", c_int32, [c_void_p, c_void_p, POINTER(c_double), POINTER(c_double), c_void_p]),
    ("hhl_qpp_iterate", c_int32, [c_void_p, c_int32, c_int32, c_void_p]),
    ("hhl_qpp_rotation_table", c_int32, [c_int32, c_double, c_int32, c_void_p]),
    ("hhl_qpp_start_state", c_int32, [c_void_p, c_int32, c_int32, c_void_p]),
    ("hhl_qpp_project", c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p]),
    ("hhl_kernel_launch_count", c_uint64, []),
    ("hhl_controlled_u_noalloc", c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p]),
    ("hhl_profile_enable", None, [c_int32]),
    ("hhl_profile_reset", None, []),
    ("hhl_profile_count", c_int32, []),
    ("hhl_profile_get", c_int32, [c_int32, c_char_p, c_int32, POINTER(c_uint64), POINTER(c_double)]),
]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhhl.so (built by paper_2307_00391_gb300.build) and declare its signatures.
    Raises if the library is missing: there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhhl.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HHLError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {detail}")


def check(status: int, where: str) -> None:
    if status != HHL_OK:
        detail = load().hhl_last_error().decode(errors="replace")
        raise HHLError(status, where, detail)
