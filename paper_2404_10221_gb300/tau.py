"""Thin ctypes binding of libtau_rsfde.so (include/tau_rsfde.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Device vectors are torch CUDA tensors (FP64, contiguous); the stream is torch's
current stream unless given.  There is no CPU fallback: loading fails loudly if
the library has not been built.
"""

from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtau_rsfde.so")

TAU_OK = 0
TAU_EINVAL = -1
TAU_ECUDA = -2
TAU_ENOMEM = -3
TAU_ETIMEOUT = -4
TAU_ESTATE = -5
TAU_EUNSUPPORTED = -6
TAU_ENOTCONV = -7
TAU_X0_ZERO = 0
TAU_X0_PREV = 1
TAU_FP64 = 0
TAU_MIXED = 1
TAU_DF64 = 2
TAU_OPGM = 0
TAU_TPGM = 1
TAU_SPGM = 2
TAU_TC_AUTO = 0
TAU_TC_OFF = 1
TAU_TC_ON = 2
TAU_TUNE_AUTO = 0
TAU_TUNE_ON = 1
TAU_TUNE_OFF = 2
TAU_TUNE_RECORDED = 3
TAU_ROUTE_AUTO = 0
TAU_ROUTE_FFT = 1
TAU_ROUTE_DENSE = 2
TAU_ROUTE_CHIRP = 3
TAU_ROUTE_LONG = 4


class tau_problem_desc(C.Structure):
    _fields_ = [
        ("d", C.c_int),
        ("n", C.c_int64 * 3),
        ("L", C.c_double * 3),
        ("R", C.c_double * 3),
        ("alpha", C.c_double * 3),
        ("kappa", C.c_double * 3),
        ("T", C.c_double),
        ("M", C.c_int64),
        ("tol", C.c_double),
        ("max_iter", C.c_int),
        ("x0_mode", C.c_int),
        ("precision", C.c_int),
        ("route", C.c_int * 3),
        ("e_min", C.c_double),
        ("e_max", C.c_double),
        ("refine_tol", C.c_double),
        ("inner_max_iter", C.c_int),
        ("max_sweeps", C.c_int),
        ("inner_tol", C.c_double),
        ("method", C.c_int),
        ("tc", C.c_int),
        ("autotune", C.c_int),
    ]


class tau_field(C.Structure):
    _fields_ = [
        ("rank", C.c_int),
        ("n_times", C.c_int64),
        ("time_coef", C.POINTER(C.c_double)),
        ("space", C.POINTER(C.c_double) * 3),
    ]


class tau_field_device(C.Structure):
    _fields_ = [
        ("e", C.c_void_p),
        ("e_step", C.c_int64),
        ("f", C.c_void_p),
        ("f_step", C.c_int64),
        ("psi", C.c_void_p),
    ]


class tau_stats(C.Structure):
    _fields_ = [
        ("steps_done", C.c_int64),
        ("total_iters", C.c_int64),
        ("last_iters", C.c_int),
        ("max_iters_step", C.c_int),
        ("last_relres", C.c_double),
        ("ebar", C.c_double),
        ("e_hat", C.c_double),
        ("e_check", C.c_double),
        ("route", C.c_int * 3),
        ("graph", C.c_int),
        ("device_bytes", C.c_int64),
        ("kernels_prologue", C.c_int64),
        ("kernels_per_iter", C.c_int64),
        ("kernels_epilogue", C.c_int64),
        ("kernels_total", C.c_int64),
        ("total_sweeps", C.c_int64),
        ("lines_per_cta", C.c_int * 3),
        ("lines_per_cta_f32", C.c_int * 3),
        ("tc_dims", C.c_int),
        ("route_source", C.c_int * 3),
        ("route_ms", C.c_double * 3),
        ("route_alt_ms", C.c_double * 3),
        ("resid_precision", C.c_int),
    ]


class tau_batch_info(C.Structure):
    _fields_ = [
        ("groups", C.c_int),
        ("grouped_problems", C.c_int),
        ("branches", C.c_int),
        ("launches_prologue_epilogue", C.c_int64),
        ("launches_per_sweep", C.c_int64),
        ("launches_per_inner_iter", C.c_int64),
    ]


TAU_REQ_QUEUED, TAU_REQ_RUNNING, TAU_REQ_DONE, TAU_REQ_FAILED = 0, 1, 2, 3


class tau_request_info(C.Structure):
    _fields_ = [
        ("id", C.c_int64),
        ("state", C.c_int),
        ("status", C.c_int),
        ("t_submit", C.c_double),
        ("t_admit", C.c_double),
        ("t_finish", C.c_double),
        ("unknowns", C.c_int64),
        ("steps", C.c_int64),
        ("gmres_iters", C.c_int64),
        ("device_bytes", C.c_int64),
    ]


class tau_server_stats(C.Structure):
    _fields_ = [
        ("completed", C.c_int64),
        ("failed", C.c_int64),
        ("queued", C.c_int64),
        ("active", C.c_int64),
        ("device_bytes_in_use", C.c_int64),
        ("latency_p50_s", C.c_double),
        ("latency_p99_s", C.c_double),
        ("latency_mean_s", C.c_double),
        ("unknowns_steps", C.c_double),
        ("span_s", C.c_double),
        ("throughput", C.c_double),
        ("group_launches", C.c_int64),
        ("group_rebuilds", C.c_int64),
        ("group_request_steps", C.c_int64),
    ]


class TauError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tau status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load the CUDA library (raises if it is missing: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        D = C.POINTER(C.c_double)
        sigs = {
            "tau_create": [C.POINTER(tau_problem_desc), P, C.POINTER(P)],
            "tau_set_fields": [P, C.POINTER(tau_field), C.POINTER(tau_field), C.POINTER(tau_field)],
            "tau_set_fields_device": [P, C.POINTER(tau_field_device)],
            "tau_setup": [P],
            "tau_step": [P, C.c_int64],
            "tau_solve": [P],
            "tau_sync": [P],
            "tau_get_solution": [P, P, C.c_int, C.POINTER(C.c_int64)],
            "tau_set_solution": [P, P, C.c_int, C.c_int64],
            "tau_get_stats": [P, C.POINTER(tau_stats)],
            "tau_get_iters": [P, C.POINTER(C.c_int), C.c_int64],
            "tau_destroy": [P],
            "tau_apply_A": [P, C.c_int64, P, P],
            "tau_apply_Minv": [P, P, P],
            "tau_apply_MinvA": [P, C.c_int64, P, P],
            "tau_rhs": [P, C.c_int64, P, P],
            "tau_dst": [P, P, P],
            "tau_toeplitz_mode": [P, C.c_int, P, P],
            "tau_get_ebar": [P, D, D, D],
            "tau_measure_fp64_peak": [P, D],
            "tau_selftest_bounded_wait": [P, C.POINTER(C.c_int)],
            "tau_inject_wait_timeout": [P],
            "tau_choose_precision": [C.POINTER(tau_problem_desc), C.POINTER(C.c_int)],
            "tau_apply_A_noalloc": [C.POINTER(tau_problem_desc), P, P, P, P],
            "tau_apply_A_f32": [P, C.c_int64, P, P],
            "tau_batch_create": [C.POINTER(P), C.c_int, P, C.POINTER(P)],
            "tau_batch_step": [P, C.c_int64],
            "tau_batch_sync": [P],
            "tau_batch_destroy": [P],
            "tau_batch_get_info": [P, C.POINTER(tau_batch_info)],
            "tau_server_create": [C.c_int64, C.c_int, C.c_int, C.POINTER(P)],
            "tau_server_submit": [P, C.POINTER(tau_problem_desc), C.POINTER(tau_field), C.POINTER(tau_field),
                                  C.POINTER(tau_field), C.POINTER(C.c_int64)],
            "tau_server_poll": [P, C.c_int64, C.POINTER(tau_request_info)],
            "tau_server_wait": [P, C.c_int64, C.c_double, C.POINTER(tau_request_info)],
            "tau_server_result": [P, C.c_int64, P, C.c_int64],
            "tau_server_release": [P, C.c_int64],
            "tau_server_summary": [P, C.POINTER(tau_server_stats)],
            "tau_server_destroy": [P],
            "tau_apply_Minv_f32": [P, P, P],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.tau_last_error.argtypes = []
        L.tau_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status: int, allow=()):
    if status != TAU_OK and status not in allow:
        msg = lib().tau_last_error().decode(errors="replace")
        raise TauError(status, msg)
    return status


def _ptr(t, dtype: str = "float64") -> int:
    """Device pointer of a contiguous CUDA tensor of the given dtype (float64 by default)."""
    import torch
    dt = getattr(torch, dtype)
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
        raise TypeError(f"expected a contiguous {dtype} CUDA tensor")
    return t.data_ptr()


def _stream(stream=None) -> int:
    if stream is not None:
        return int(stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


def make_desc(prob, precision: int = TAU_FP64, route: Sequence[int] = (0, 0, 0),
              e_bounds: Optional[tuple] = None, refine_tol: float = 0.0, inner_max_iter: int = 0,
              max_sweeps: int = 0, inner_tol: float = 0.0, method: int = TAU_OPGM,
              tc: int = 0, autotune: int = TAU_TUNE_AUTO) -> tau_problem_desc:
    """tau_problem_desc from a workloads.Problem."""
    d = tau_problem_desc()
    d.d = prob.d
    for i in range(3):
        d.n[i] = int(prob.n[i]) if i < prob.d else 1
        d.L[i] = float(prob.L[i]) if i < len(prob.L) else 0.0
        d.R[i] = float(prob.R[i]) if i < len(prob.R) else 1.0
        d.alpha[i] = float(prob.alpha[i]) if i < prob.d else 1.5
        d.kappa[i] = float(prob.kappa[i]) if i < prob.d else 0.0
        d.route[i] = int(route[i])
    d.T = float(prob.T)
    d.M = int(prob.M)
    d.tol = float(prob.tol)
    d.max_iter = int(prob.max_iter)
    d.x0_mode = int(prob.x0_mode)
    d.precision = precision
    d.method = int(method)
    d.tc = int(tc)
    d.autotune = int(autotune)
    if e_bounds is None:
        d.e_min = d.e_max = math.nan
    else:
        d.e_min, d.e_max = float(e_bounds[0]), float(e_bounds[1])
    d.refine_tol = float(refine_tol)
    d.inner_max_iter = int(inner_max_iter)
    d.max_sweeps = int(max_sweeps)
    d.inner_tol = float(inner_tol)
    return d


class _FieldHolder:
    """Keeps the numpy tables alive while tau_set_fields copies them."""

    def __init__(self, tc: np.ndarray, sp: Sequence[np.ndarray]):
        self.tc = np.ascontiguousarray(tc, dtype=np.float64)
        self.sp = [np.ascontiguousarray(s, dtype=np.float64) for s in sp]
        self.f = tau_field()
        self.f.rank = self.tc.shape[1]
        self.f.n_times = self.tc.shape[0]
        self.f.time_coef = self.tc.ctypes.data_as(C.POINTER(C.c_double))
        for i, s in enumerate(self.sp):
            self.f.space[i] = s.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------------------
# functions with the C ABI's names
# ---------------------------------------------------------------------------
def tau_create(desc: tau_problem_desc, stream=None) -> int:
    h = C.c_void_p()
    _check(lib().tau_create(C.byref(desc), C.c_void_p(_stream(stream)), C.byref(h)))
    return h.value


def tau_set_fields(h: int, tables: dict):
    e = _FieldHolder(tables["e_tc"], tables["e_sp"])
    f = _FieldHolder(tables["f_tc"], tables["f_sp"])
    p = _FieldHolder(tables["psi_tc"], tables["psi_sp"])
    _check(lib().tau_set_fields(C.c_void_p(h), C.byref(e.f), C.byref(f.f), C.byref(p.f)))


def tau_set_fields_device(h: int, e, f=None, psi=None, e_step: Optional[int] = None,
                          f_step: Optional[int] = None):
    """Fields as caller-owned CUDA float64 tensors: e of M x n_tot (or n_tot: not time dependent),
    f of M x prod(n_i + 2) on the padded grid (or one slab, or None: f = 0), psi of n_tot (or None).
    The tensors must stay alive and unchanged until the problem is destroyed."""
    fd = tau_field_device()
    fd.e = _ptr(e)
    fd.e_step = int(e_step) if e_step is not None else (e.shape[-1] if e.dim() == 2 else 0)
    fd.f = _ptr(f) if f is not None else None
    fd.f_step = int(f_step) if f_step is not None else (f.shape[-1] if f is not None and f.dim() == 2 else 0)
    fd.psi = _ptr(psi) if psi is not None else None
    _check(lib().tau_set_fields_device(C.c_void_p(h), C.byref(fd)))


def tau_setup(h: int):
    _check(lib().tau_setup(C.c_void_p(h)))


def tau_step(h: int, count: int = 1):
    _check(lib().tau_step(C.c_void_p(h), C.c_int64(count)))


def tau_solve(h: int, allow_notconv: bool = False):
    return _check(lib().tau_solve(C.c_void_p(h)), (TAU_ENOTCONV,) if allow_notconv else ())


def tau_sync(h: int, allow_notconv: bool = False):
    return _check(lib().tau_sync(C.c_void_p(h)), (TAU_ENOTCONV,) if allow_notconv else ())


def tau_get_solution(h: int, out, is_device: bool):
    m = C.c_int64()
    ptr = _ptr(out) if is_device else out.ctypes.data
    _check(lib().tau_get_solution(C.c_void_p(h), C.c_void_p(ptr), 1 if is_device else 0, C.byref(m)))
    return m.value


def tau_set_solution(h: int, u, is_device: bool, m: int):
    ptr = _ptr(u) if is_device else np.ascontiguousarray(u, dtype=np.float64).ctypes.data
    _check(lib().tau_set_solution(C.c_void_p(h), C.c_void_p(ptr), 1 if is_device else 0, C.c_int64(m)))


def tau_get_stats(h: int, allow_notconv: bool = True) -> tau_stats:
    s = tau_stats()
    _check(lib().tau_get_stats(C.c_void_p(h), C.byref(s)), (TAU_ENOTCONV,) if allow_notconv else ())
    return s


def tau_get_iters(h: int, cap: int) -> np.ndarray:
    arr = np.zeros(cap, dtype=np.int32)
    _check(lib().tau_get_iters(C.c_void_p(h), arr.ctypes.data_as(C.POINTER(C.c_int)), C.c_int64(cap)))
    return arr


def tau_destroy(h: int):
    _check(lib().tau_destroy(C.c_void_p(h)))


def tau_apply_A(h: int, m: int, x, y):
    _check(lib().tau_apply_A(C.c_void_p(h), C.c_int64(m), C.c_void_p(_ptr(x)), C.c_void_p(_ptr(y))))


def tau_apply_Minv(h: int, r, z):
    _check(lib().tau_apply_Minv(C.c_void_p(h), C.c_void_p(_ptr(r)), C.c_void_p(_ptr(z))))


def tau_apply_MinvA(h: int, m: int, x, z):
    _check(lib().tau_apply_MinvA(C.c_void_p(h), C.c_int64(m), C.c_void_p(_ptr(x)), C.c_void_p(_ptr(z))))


def tau_rhs(h: int, m: int, u, b):
    _check(lib().tau_rhs(C.c_void_p(h), C.c_int64(m), C.c_void_p(_ptr(u)), C.c_void_p(_ptr(b))))


def tau_dst(h: int, x, y):
    _check(lib().tau_dst(C.c_void_p(h), C.c_void_p(_ptr(x)), C.c_void_p(_ptr(y))))


def tau_toeplitz_mode(h: int, dim: int, x, y):
    _check(lib().tau_toeplitz_mode(C.c_void_p(h), C.c_int(dim), C.c_void_p(_ptr(x)), C.c_void_p(_ptr(y))))


def tau_apply_A_f32(h: int, m: int, x, y):
    _check(lib().tau_apply_A_f32(C.c_void_p(h), C.c_int64(m), C.c_void_p(_ptr(x, "float32")),
                                 C.c_void_p(_ptr(y, "float32"))))


def tau_apply_Minv_f32(h: int, r, z):
    _check(lib().tau_apply_Minv_f32(C.c_void_p(h), C.c_void_p(_ptr(r, "float32")), C.c_void_p(_ptr(z, "float32"))))


def tau_get_ebar(h: int):
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(lib().tau_get_ebar(C.c_void_p(h), C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def tau_measure_fp64_peak(stream=None) -> float:
    v = C.c_double()
    _check(lib().tau_measure_fp64_peak(C.c_void_p(_stream(stream)), C.byref(v)))
    return v.value


def tau_choose_precision(desc: tau_problem_desc) -> int:
    """TAU_MIXED or TAU_DF64 for this problem (host only; desc.e_min must be set)."""
    v = C.c_int(-1)
    _check(lib().tau_choose_precision(C.byref(desc), C.byref(v)))
    return v.value


def tau_selftest_bounded_wait(stream=None) -> bool:
    """True when a device wait on an mbarrier that nothing arrives at gave up as it must."""
    v = C.c_int(-1)
    _check(lib().tau_selftest_bounded_wait(C.c_void_p(_stream(stream)), C.byref(v)))
    return v.value == 1


def tau_inject_wait_timeout(h: int):
    _check(lib().tau_inject_wait_timeout(C.c_void_p(h)))


def tau_apply_A_noalloc(desc: tau_problem_desc, e, x, y, stream=None):
    """y = A x without a problem handle and without device allocation (static scratch)."""
    _check(lib().tau_apply_A_noalloc(C.byref(desc), C.c_void_p(_ptr(e)), C.c_void_p(_ptr(x)),
                                     C.c_void_p(_ptr(y)), C.c_void_p(_stream(stream))))


def tau_batch_create(handles: Sequence[int], stream=None) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    b = C.c_void_p()
    _check(lib().tau_batch_create(arr, C.c_int(len(handles)), C.c_void_p(_stream(stream)), C.byref(b)))
    return b.value


def tau_batch_step(b: int, count: int = 1):
    _check(lib().tau_batch_step(C.c_void_p(b), C.c_int64(count)))


def tau_batch_sync(b: int, allow_notconv: bool = False):
    return _check(lib().tau_batch_sync(C.c_void_p(b)), (TAU_ENOTCONV,) if allow_notconv else ())


def tau_batch_get_info(b: int) -> tau_batch_info:
    info = tau_batch_info()
    _check(lib().tau_batch_get_info(C.c_void_p(b), C.byref(info)))
    return info


def tau_batch_destroy(b: int):
    _check(lib().tau_batch_destroy(C.c_void_p(b)))


def tau_server_create(budget_bytes: int, max_active: int, steps_per_launch: int = 4) -> int:
    h = C.c_void_p()
    _check(lib().tau_server_create(C.c_int64(budget_bytes), C.c_int(max_active), C.c_int(steps_per_launch),
                                   C.byref(h)))
    return h.value


def tau_server_submit(s: int, desc: tau_problem_desc, tables: dict) -> int:
    e = _FieldHolder(tables["e_tc"], tables["e_sp"])
    f = _FieldHolder(tables["f_tc"], tables["f_sp"])
    p = _FieldHolder(tables["psi_tc"], tables["psi_sp"])
    rid = C.c_int64()
    _check(lib().tau_server_submit(C.c_void_p(s), C.byref(desc), C.byref(e.f), C.byref(f.f), C.byref(p.f),
                                   C.byref(rid)))
    return rid.value


def tau_server_poll(s: int, rid: int) -> tau_request_info:
    info = tau_request_info()
    _check(lib().tau_server_poll(C.c_void_p(s), C.c_int64(rid), C.byref(info)))
    return info


def tau_server_wait(s: int, rid: int, timeout_s: float = 600.0) -> tau_request_info:
    info = tau_request_info()
    _check(lib().tau_server_wait(C.c_void_p(s), C.c_int64(rid), C.c_double(timeout_s), C.byref(info)))
    return info


def tau_server_result(s: int, rid: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _check(lib().tau_server_result(C.c_void_p(s), C.c_int64(rid), C.c_void_p(out.ctypes.data), C.c_int64(n)),
           (TAU_ENOTCONV,))
    return out


def tau_server_release(s: int, rid: int):
    _check(lib().tau_server_release(C.c_void_p(s), C.c_int64(rid)))


def tau_server_summary(s: int) -> tau_server_stats:
    out = tau_server_stats()
    _check(lib().tau_server_summary(C.c_void_p(s), C.byref(out)))
    return out


def tau_server_destroy(s: int):
    _check(lib().tau_server_destroy(C.c_void_p(s)))


class Problem:
    """Owner of one tau_problem: create, set fields, set up; destroyed with the object."""

    def __init__(self, workload, precision: int = TAU_FP64, route=(0, 0, 0), stream=None, e_bounds=None, **mixed):
        self.workload = workload
        self.prob = workload.prob
        self.handle = tau_create(make_desc(self.prob, precision, route, e_bounds, **mixed), stream)
        try:
            tau_set_fields(self.handle, workload.field_tables())
            tau_setup(self.handle)
        except Exception:
            tau_destroy(self.handle)
            self.handle = None
            raise

    def close(self):
        if getattr(self, "handle", None):
            tau_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, count: int = 1):
        tau_step(self.handle, count)

    def solve(self, allow_notconv: bool = False):
        return tau_solve(self.handle, allow_notconv)

    def solution(self):
        import torch
        out = torch.empty(self.prob.n_tot, dtype=torch.float64, device="cuda")
        tau_get_solution(self.handle, out, True)
        return out

    def stats(self) -> tau_stats:
        return tau_get_stats(self.handle)

    def iters(self) -> np.ndarray:
        return tau_get_iters(self.handle, self.prob.M)
