"""GB300 (sm_103a) state-vector engine for the HHL circuit of QFlowS.

Python binding of the C ABI (include/hhl.h): every call marshals arguments into
libhhl.so; torch supplies device memory and streams only. The names follow the C
entry points: ``prepare_rhs``, ``apply_circuit``, ``measure``, ``dissipation``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _ffi
from ._ffi import HHLError, check, load

__all__ = ["HHLPlan", "HHLBatch", "HHLError", "load", "apply_qft", "kernel_launch_count", "laplacian",
           "profile_enable", "profile_reset", "profile_read"]

_PREC = {"c64": _ffi.PREC_C64, "c128": _ffi.PREC_C128}
_RULE = {"user": _ffi.T0_USER, "power_law": _ffi.T0_POWER_LAW, "range_fill": _ffi.T0_RANGE_FILL}
_CONV = {"total": _ffi.T0_TOTAL, "per_unit": _ffi.T0_PER_UNIT}
_EXPM = {"dense": _ffi.EXPM_DENSE, "trotter": _ffi.EXPM_TROTTER}
_GEMM = {"auto": _ffi.GEMM_AUTO, "simt": _ffi.GEMM_SIMT, "tcgen05": _ffi.GEMM_TCGEN05}
STAGES = {"qpe_u": _ffi.STAGE_QPE_U, "clock_block": _ffi.STAGE_CLOCK_BLOCK,
          "uncompute_u": _ffi.STAGE_UNCOMPUTE_U, "final_h": _ffi.STAGE_FINAL_H}


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def laplacian(n_points: int) -> tuple[np.ndarray, np.ndarray]:
    """Input arrays (diag, off) describing tridiag(-1, 2, -1)/h^2, h = 1/(N+1)."""
    h = 1.0 / (n_points + 1)
    return np.full(n_points, 2.0 / (h * h)), np.full(n_points - 1, -1.0 / (h * h))


def kernel_launch_count() -> int:
    return int(load().hhl_kernel_launch_count())


def profile_enable(on: bool = True) -> None:
    """Bracket every kernel launch with CUDA events (see hhl_profile_enable)."""
    load().hhl_profile_enable(int(on))


def profile_reset() -> None:
    load().hhl_profile_reset()


def profile_read() -> dict:
    """{kernel name: (launches, total ms)} accumulated since the last reset."""
    lib = load()
    out = {}
    for i in range(lib.hhl_profile_count()):
        name = ctypes.create_string_buffer(128)
        n = ctypes.c_uint64()
        ms = ctypes.c_double()
        check(lib.hhl_profile_get(i, name, 128, ctypes.byref(n), ctypes.byref(ms)), "hhl_profile_get")
        out[name.value.decode()] = (int(n.value), float(ms.value))
    return out


class HHLPlan:
    """An hhl_plan_t: A, T0, C, theta_y and the U_k (or Trotter) tables on the device."""

    def __init__(self, n_sys_qubits: int, n_clock: int, diag=None, off=None, dense=None,
                 precision: str = "c64", t0_rule: str = "range_fill", t0: float = 0.0,
                 t0_convention: str = "total", C: float = 0.0, expm: str = "dense",
                 full_uncompute: bool = False, trotter_dt: float = 1.0, trotter_steps_max: int = 0,
                 gemm: str = "auto", nu: float = 0.1, walls=(0.0, 0.0), signed_clock: bool = False,
                 unitary=None, theta_table=None):
        """``unitary`` (with ``theta_table``, 2^n_clock angles): phase estimation of that unitary
        itself (U_k = Q^(2^k)) with the given ancilla rotation per clock value, in place of
        exp(i Ahat t_k) and the eigenvalue inversion."""
        lib = load()
        self._lib = lib
        self._keep = []
        prob = _ffi.Problem()
        prob.n_sys_qubits = n_sys_qubits
        if unitary is not None:
            dense = unitary
        if dense is not None:
            dense = np.asarray(dense)
            re = np.ascontiguousarray(dense.real, dtype=np.float64)
            im = np.ascontiguousarray(dense.imag, dtype=np.float64) if np.iscomplexobj(dense) else None
            self._keep += [re, im]
            prob.kind = _ffi.MATRIX_UNITARY if unitary is not None else _ffi.MATRIX_DENSE
            prob.dense_re = _dptr(re)
            prob.dense_im = _dptr(im)
        else:
            d = np.ascontiguousarray(diag, dtype=np.float64)
            o = np.ascontiguousarray(off, dtype=np.float64)
            self._keep += [d, o]
            prob.kind = _ffi.MATRIX_TRIDIAG
            prob.diag = _dptr(d)
            prob.off = _dptr(o)
        prob.nu = nu
        prob.wall_lo, prob.wall_hi = walls
        par = _ffi.Params()
        lib.hhl_params_default(ctypes.byref(par))
        par.n_clock = n_clock
        par.t0_rule = _RULE[t0_rule]
        par.t0_convention = _CONV[t0_convention]
        par.precision = _PREC[precision]
        par.t0 = t0
        par.C = C
        par.expm_mode = _EXPM[expm]
        par.full_uncompute = int(full_uncompute)
        par.trotter_dt = trotter_dt
        par.trotter_steps_max = trotter_steps_max
        par.gemm_impl = _GEMM[gemm]
        par.signed_clock = int(signed_clock)
        if theta_table is not None:
            th = np.ascontiguousarray(theta_table, dtype=np.float64)
            self._keep.append(th)
            par.theta_table = _dptr(th)
        h = ctypes.c_void_p()
        check(lib.hhl_plan_create(ctypes.byref(prob), ctypes.byref(par), ctypes.byref(h)), "hhl_plan_create")
        self._h = h
        self.precision = precision
        self.n_s, self.n_c = n_sys_qubits, n_clock
        self.N = 1 << n_sys_qubits
        self.full_uncompute = bool(full_uncompute)
        self._keep.clear()

    # -- lifetime ---------------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.hhl_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- info -------------------------------------------------------------------------
    @property
    def info(self) -> dict:
        inf = _ffi.PlanInfo()
        check(self._lib.hhl_plan_get_info(self._h, ctypes.byref(inf)), "hhl_plan_get_info")
        return {name: getattr(inf, name) for name, _ in _ffi.PlanInfo._fields_}

    @property
    def state_bytes(self) -> int:
        return int(self._lib.hhl_state_bytes(self._h))

    def new_state(self, device="cuda"):
        """A caller-owned state buffer (torch, complex64 or complex128)."""
        import torch
        dt = torch.complex64 if self.precision == "c64" else torch.complex128
        amps = self.state_bytes // (8 if self.precision == "c64" else 16)
        return torch.empty(amps, dtype=dt, device=device)

    # -- the path -----------------------------------------------------------------------
    def prepare_rhs(self, b_dev, state, stream=None) -> None:
        """a1 with b already on the device (torch complex128 tensor of length N)."""
        check(self._lib.hhl_prepare_rhs(self._h, ctypes.c_void_p(b_dev.data_ptr()), ctypes.c_void_p(state.data_ptr()),
                                        ctypes.c_void_p(_stream_handle(stream))), "hhl_prepare_rhs")

    def prepare_rhs_host(self, b_re: np.ndarray, state, b_im: np.ndarray | None = None, stream=None) -> None:
        """a1 with b in host memory (numpy float64, or a pinned torch CPU tensor)."""
        def host_ptr(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(a.data_ptr())
            return ctypes.c_void_p(a.ctypes.data)
        re = b_re if hasattr(b_re, "data_ptr") else np.ascontiguousarray(b_re, dtype=np.float64)
        im = None if b_im is None else (b_im if hasattr(b_im, "data_ptr") else np.ascontiguousarray(b_im, dtype=np.float64))
        check(self._lib.hhl_prepare_rhs_host(self._h, host_ptr(re), host_ptr(im), ctypes.c_void_p(state.data_ptr()),
                                             ctypes.c_void_p(_stream_handle(stream))), "hhl_prepare_rhs_host")

    def apply_circuit(self, state, stream=None) -> None:
        check(self._lib.hhl_apply_circuit(self._h, ctypes.c_void_p(state.data_ptr()),
                                          ctypes.c_void_p(_stream_handle(stream))), "hhl_apply_circuit")

    def apply_stage(self, stage: str, state, stream=None) -> None:
        check(self._lib.hhl_apply_stage(self._h, STAGES[stage], ctypes.c_void_p(state.data_ptr()),
                                        ctypes.c_void_p(_stream_handle(stream))), "hhl_apply_stage")

    def measure(self, state, stream=None, want_x: bool = True) -> dict:
        m = _ffi.Measurement()
        x = np.zeros(2 * self.N, dtype=np.float64) if want_x else None
        check(self._lib.hhl_measure(self._h, ctypes.c_void_p(state.data_ptr()), ctypes.byref(m),
                                    None if x is None else ctypes.c_void_p(x.ctypes.data),
                                    ctypes.c_void_p(_stream_handle(stream))), "hhl_measure")
        out = dict(p_success=m.p_success, p_anc1=m.p_anc1, norm=m.norm, b_norm=m.b_norm)
        if x is not None:
            out["xhat"] = x[0::2] + 1j * x[1::2]
        return out

    def status(self, stream=None) -> None:
        """Raise HHLError if the last circuit's tensor-core GEMMs reported a timeout or an
        out-of-range operand (synchronises the stream)."""
        check(self._lib.hhl_plan_status(self._h, ctypes.c_void_p(_stream_handle(stream))), "hhl_plan_status")

    def solve_postselected(self, b_dev, state, out_dev, eps_dev=None, stream=None) -> None:
        """One whole solve for the read-out only (hhl_solve_postselected): b_dev (torch
        complex128, N) on the device; out_dev (torch float64, 4 + 2N) receives p_success,
        p_anc1, norm, |b| and xhat; eps_dev (torch float64, 1) the dissipation rate. Afterwards
        only the clock = 0 row of the anc = 1 half of ``state`` is defined (it holds v)."""
        check(self._lib.hhl_solve_postselected(self._h, ctypes.c_void_p(b_dev.data_ptr()),
                                               ctypes.c_void_p(state.data_ptr()), ctypes.c_void_p(out_dev.data_ptr()),
                                               None if eps_dev is None else ctypes.c_void_p(eps_dev.data_ptr()),
                                               ctypes.c_void_p(_stream_handle(stream))), "hhl_solve_postselected")

    def measure_async(self, state, out_dev, stream=None) -> None:
        check(self._lib.hhl_measure_async(self._h, ctypes.c_void_p(state.data_ptr()), ctypes.c_void_p(out_dev.data_ptr()),
                                          ctypes.c_void_p(_stream_handle(stream))), "hhl_measure_async")

    def dissipation(self, state, stream=None, want_u: bool = False):
        eps = ctypes.c_double()
        u = np.zeros(self.N, dtype=np.float64) if want_u else None
        check(self._lib.hhl_dissipation(self._h, ctypes.c_void_p(state.data_ptr()), ctypes.byref(eps),
                                        None if u is None else ctypes.c_void_p(u.ctypes.data),
                                        ctypes.c_void_p(_stream_handle(stream))), "hhl_dissipation")
        return (eps.value, u) if want_u else eps.value

    def prepare_rhs_qsp1(self, b_dev, state, stream=None) -> None:
        """Gate-level RHS preparation (QSP-1 tree + clock Hadamards); b_dev: torch float64 (N)."""
        check(self._lib.hhl_prepare_rhs_qsp1(self._h, ctypes.c_void_p(b_dev.data_ptr()),
                                             ctypes.c_void_p(state.data_ptr()),
                                             ctypes.c_void_p(_stream_handle(stream))), "hhl_prepare_rhs_qsp1")

    def prepare_rhs_qsp2(self, idx_dev, val_dev, state, stream=None) -> None:
        """Sparse gate-level RHS preparation (QSP-2 decision-tree paths + clock Hadamards);
        idx_dev: torch int64 strictly increasing positions, val_dev: torch float64 values."""
        check(self._lib.hhl_prepare_rhs_qsp2(self._h, ctypes.c_void_p(idx_dev.data_ptr()),
                                             ctypes.c_void_p(val_dev.data_ptr()), int(idx_dev.numel()),
                                             ctypes.c_void_p(state.data_ptr()),
                                             ctypes.c_void_p(_stream_handle(stream))), "hhl_prepare_rhs_qsp2")

    def qpp_dissipation(self, state, stream=None) -> tuple[float, float]:
        """(eps, p0): the dissipation rate from the LCU post-processing circuit's ancilla-0
        probability p0 (synchronises the stream)."""
        eps, p0 = ctypes.c_double(), ctypes.c_double()
        check(self._lib.hhl_qpp_dissipation(self._h, ctypes.c_void_p(state.data_ptr()), ctypes.byref(eps),
                                            ctypes.byref(p0), ctypes.c_void_p(_stream_handle(stream))),
              "hhl_qpp_dissipation")
        return eps.value, p0.value

    def sample(self, state, uniforms_dev, counts_dev, stream=None) -> None:
        """Shots of the postselected system register: counts_dev (torch int64, N) from the
        uniforms in uniforms_dev (torch float64, one per shot)."""
        check(self._lib.hhl_sample(self._h, ctypes.c_void_p(state.data_ptr()),
                                   ctypes.c_void_p(uniforms_dev.data_ptr()), int(uniforms_dev.numel()),
                                   ctypes.c_void_p(counts_dev.data_ptr()),
                                   ctypes.c_void_p(_stream_handle(stream))), "hhl_sample")

    def dissipation_async(self, state, eps_dev, stream=None) -> None:
        check(self._lib.hhl_dissipation_async(self._h, ctypes.c_void_p(state.data_ptr()),
                                              ctypes.c_void_p(eps_dev.data_ptr()),
                                              ctypes.c_void_p(_stream_handle(stream))), "hhl_dissipation_async")


def apply_qft(state, n_qubits: int, lo: int, m: int, inverse: bool, stream=None) -> None:
    """Fused QFT / inverse QFT block on bits [lo, lo+m) of a torch complex state."""
    import torch
    prec = _ffi.PREC_C64 if state.dtype == torch.complex64 else _ffi.PREC_C128
    check(load().hhl_apply_qft(ctypes.c_void_p(state.data_ptr()), n_qubits, lo, m, int(inverse), prec,
                               ctypes.c_void_p(_stream_handle(stream))), "hhl_apply_qft")


def qft_whole(state, n_qubits: int, n_states: int, direction: int, stream=None) -> None:
    """Whole-register QFT (direction 0, result in bit-reversed order) or inverse QFT
    (direction 1, input in bit-reversed order) of n_states consecutive n-qubit states."""
    import torch
    prec = _ffi.PREC_C64 if state.dtype == torch.complex64 else _ffi.PREC_C128
    check(load().hhl_qft_whole(ctypes.c_void_p(state.data_ptr()), n_qubits, n_states, direction, prec,
                               ctypes.c_void_p(_stream_handle(stream))), "hhl_qft_whole")


class HHLBatch:
    """An hhl_batch_t: many uneven instances (Toeplitz tridiagonal A, complex64) run as one
    CUDA graph. ``problems``: dicts with n_sys_qubits, n_clock, diag, off and optionally nu,
    walls, t0_rule, t0, t0_convention, t0_scale, C. ``gemm_choice``: per instance 0 (CUDA
    cores), 128 or 256 (tcgen05 tile width), or None for the library's size rule."""

    def __init__(self, problems: list, gemm_choice=None, streams: int = 8):
        lib = load()
        self._lib = lib
        n = len(problems)
        probs = (_ffi.Problem * n)()
        pars = (_ffi.Params * n)()
        keep = []
        for i, pr in enumerate(problems):
            d = np.ascontiguousarray(pr["diag"], dtype=np.float64)
            o = np.ascontiguousarray(pr["off"], dtype=np.float64)
            keep += [d, o]
            probs[i].kind = _ffi.MATRIX_TRIDIAG
            probs[i].n_sys_qubits = pr["n_sys_qubits"]
            probs[i].diag = _dptr(d)
            probs[i].off = _dptr(o)
            probs[i].nu = pr.get("nu", 0.1)
            probs[i].wall_lo, probs[i].wall_hi = pr.get("walls", (0.0, 0.0))
            lib.hhl_params_default(ctypes.byref(pars[i]))
            pars[i].n_clock = pr["n_clock"]
            pars[i].t0_rule = _RULE[pr.get("t0_rule", "power_law")]
            pars[i].t0 = pr.get("t0", 0.0)
            pars[i].t0_convention = _CONV[pr.get("t0_convention", "total")]
            pars[i].t0_scale = pr.get("t0_scale", 1.0)
            pars[i].C = pr.get("C", 0.0)
            pars[i].precision = _ffi.PREC_C64
        choice = None
        if gemm_choice is not None:
            choice = (ctypes.c_int32 * n)(*[int(c) for c in gemm_choice])
        h = ctypes.c_void_p()
        check(lib.hhl_batch_create(probs, pars, n, choice, streams, ctypes.byref(h)), "hhl_batch_create")
        self._h = h
        self.count = n
        self.instances = []
        for i in range(n):
            ns, nc, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
            bo, oo, t0 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
            check(lib.hhl_batch_instance(h, i, ctypes.byref(ns), ctypes.byref(nc), ctypes.byref(g), ctypes.byref(bo),
                                         ctypes.byref(oo), ctypes.byref(t0)), "hhl_batch_instance")
            self.instances.append(dict(n_s=ns.value, n_c=nc.value, gemm=g.value, b_offset=bo.value,
                                       out_offset=oo.value, t0=t0.value, N=1 << ns.value))
        del keep

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.hhl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        inf = _ffi.BatchInfo()
        check(self._lib.hhl_batch_get_info(self._h, ctypes.byref(inf)), "hhl_batch_get_info")
        return {name: getattr(inf, name) for name, _ in _ffi.BatchInfo._fields_}

    def pack_rhs(self, bs: list) -> np.ndarray:
        """Packed complex128 (as interleaved float64) right-hand sides in instance order."""
        out = np.zeros(self.info["b_doubles"], dtype=np.float64)
        for inst, b in zip(self.instances, bs):
            z = np.asarray(b, dtype=np.complex128)
            o = inst["b_offset"]
            out[o:o + 2 * inst["N"]:2] = z.real
            out[o + 1:o + 2 * inst["N"]:2] = z.imag
        return out

    def unpack(self, out: np.ndarray) -> list:
        """Per instance dict(p_success, p_anc1, norm, b_norm, xhat) from a packed result array."""
        res = []
        for inst in self.instances:
            o, n = inst["out_offset"], inst["N"]
            blk = out[o:o + 4 + 2 * n]
            res.append(dict(p_success=blk[0], p_anc1=blk[1], norm=blk[2], b_norm=blk[3],
                            xhat=blk[4::2] + 1j * blk[5::2]))
        return res

    def run(self, b_dev, out_dev, eps_dev, stream=None, check_status: bool = True) -> None:
        """Device arrays (torch float64): packed b, packed results, dissipation per instance.
        With check_status (default) the call waits for the run and raises on a device-side
        GEMM error; without it the run stays asynchronous and status() must be called before
        the results are used."""
        check(self._lib.hhl_batch_run(self._h, ctypes.c_void_p(b_dev.data_ptr()), ctypes.c_void_p(out_dev.data_ptr()),
                                      ctypes.c_void_p(eps_dev.data_ptr()), ctypes.c_void_p(_stream_handle(stream))),
              "hhl_batch_run")
        if check_status:
            self.status(stream)

    def status(self, stream=None) -> None:
        """Raise HHLError if the last run's tensor-core GEMMs reported a timeout or an
        out-of-range operand (synchronises the stream)."""
        check(self._lib.hhl_batch_status(self._h, ctypes.c_void_p(_stream_handle(stream))), "hhl_batch_status")

    def run_eager(self, stream=None) -> None:
        """The same work launch by launch (for per-kernel timing), on the inputs of the last run."""
        check(self._lib.hhl_batch_run_eager(self._h, ctypes.c_void_p(_stream_handle(stream))), "hhl_batch_run_eager")

    def run_host(self, b_packed, stream=None):
        """Host arrays: packed b in (numpy or pinned torch float64); returns (packed results, eps)."""
        inf = self.info
        out = np.zeros(inf["out_doubles"], dtype=np.float64)
        eps = np.zeros(self.count, dtype=np.float64)
        bp = b_packed.data_ptr() if hasattr(b_packed, "data_ptr") else np.ascontiguousarray(b_packed).ctypes.data
        check(self._lib.hhl_batch_run_host(self._h, ctypes.c_void_p(bp), ctypes.c_void_p(out.ctypes.data),
                                           ctypes.c_void_p(eps.ctypes.data), ctypes.c_void_p(_stream_handle(stream))),
              "hhl_batch_run_host")
        return out, eps
