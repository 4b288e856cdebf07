"""CPU-side checks of the boundary: the library builds, loads and exports every
function include/tau_rsfde.h declares; the binding marshals structs and reports
argument errors; the product path has no CPU fallback."""

import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tau_rsfde.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2404_10221_gb300 import build, tau
    build.build()
    return tau.lib()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tau_[A-Za-z0-9_]+)\s*\(", txt)))


def test_header_declares_expected_calls():
    names = declared_functions()
    for must in ["tau_create", "tau_set_fields", "tau_setup", "tau_step", "tau_solve", "tau_get_solution",
                 "tau_destroy", "tau_apply_A", "tau_apply_Minv", "tau_dst", "tau_toeplitz_mode", "tau_rhs"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_layout_matches_c_compiler(tmp_path):
    """The ctypes mirrors have the sizes and field offsets a C compiler gives the header."""
    import shutil
    import subprocess
    from paper_2404_10221_gb300 import tau
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = {
        "tau_problem_desc": ["d", "n", "L", "R", "alpha", "kappa", "T", "M", "tol", "max_iter", "x0_mode",
                             "precision", "route", "e_min", "e_max", "refine_tol", "inner_max_iter",
                             "max_sweeps", "inner_tol", "method", "tc", "autotune"],
        "tau_field": ["rank", "n_times", "time_coef", "space"],
        "tau_stats": ["steps_done", "total_iters", "last_iters", "max_iters_step", "last_relres", "ebar",
                      "e_hat", "e_check", "route", "graph", "device_bytes", "kernels_prologue",
                      "kernels_per_iter", "kernels_epilogue", "kernels_total", "total_sweeps", "lines_per_cta",
                      "lines_per_cta_f32", "tc_dims", "route_source", "route_ms", "route_alt_ms",
                      "resid_precision"],
        "tau_request_info": ["id", "state", "status", "t_submit", "t_admit", "t_finish", "unknowns", "steps",
                             "gmres_iters", "device_bytes"],
        "tau_server_stats": ["completed", "failed", "queued", "active", "device_bytes_in_use", "latency_p50_s",
                               "latency_p99_s", "latency_mean_s", "unknowns_steps", "span_s", "throughput",
                               "group_launches", "group_rebuilds", "group_request_steps"],
    }
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "tau_rsfde.h"', "int main(void){"]
    for st, fields in checks.items():
        src.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fields:
            src.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    src.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for st, fields in checks.items():
        cls = getattr(tau, st)
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f in fields:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_invalid_desc_rejected_before_any_device_call(lib):
    from paper_2404_10221_gb300 import tau, workloads
    wl = workloads.c2_2d(n=7, M=2)
    bad = [("alpha", 0, 1.0), ("alpha", 1, 2.0), ("kappa", 0, -1.0)]
    for field, i, v in bad:
        d = tau.make_desc(wl.prob)
        getattr(d, field)[i] = v
        with pytest.raises(tau.TauError) as ei:
            tau.tau_create(d, 0)
        assert ei.value.status == tau.TAU_EINVAL
    d = tau.make_desc(wl.prob)
    d.d = 4
    with pytest.raises(tau.TauError):
        tau.tau_create(d, 0)
    d = tau.make_desc(wl.prob)
    d.max_iter = 0
    with pytest.raises(tau.TauError):
        tau.tau_create(d, 0)
    # empty or oversized grids, a degenerate time grid or domain, unknown selectors
    def edits():
        yield "n[0] = 0", lambda d: d.n.__setitem__(0, 0)
        yield "n[1] = 2^20 + 1", lambda d: d.n.__setitem__(1, (1 << 20) + 1)
        yield "n_tot > 2^31", lambda d: (setattr(d, "d", 3), d.n.__setitem__(0, 2048), d.n.__setitem__(1, 2048),
                                         d.n.__setitem__(2, 2048))
        yield "T = 0", lambda d: setattr(d, "T", 0.0)
        yield "M = 0", lambda d: setattr(d, "M", 0)
        yield "R <= L", lambda d: d.R.__setitem__(0, d.L[0])
        yield "all kappa 0", lambda d: (d.kappa.__setitem__(0, 0.0), d.kappa.__setitem__(1, 0.0))
        yield "tol = 0", lambda d: setattr(d, "tol", 0.0)
        yield "x0_mode", lambda d: setattr(d, "x0_mode", 3)
        yield "precision", lambda d: setattr(d, "precision", 7)
        yield "method", lambda d: setattr(d, "method", 9)
        yield "tc", lambda d: setattr(d, "tc", 5)
        yield "autotune", lambda d: setattr(d, "autotune", 4)
    for what, edit in edits():
        d = tau.make_desc(wl.prob)
        edit(d)
        with pytest.raises(tau.TauError) as ei:
            tau.tau_create(d, 0)
        assert ei.value.status == tau.TAU_EINVAL, what
    # the two-sided and Strang circulant methods run in FP64 only
    for method in (tau.TAU_TPGM, tau.TAU_SPGM):
        d = tau.make_desc(wl.prob, precision=tau.TAU_MIXED, method=method)
        with pytest.raises(tau.TauError) as ei:
            tau.tau_create(d, 0)
        assert ei.value.status == tau.TAU_EUNSUPPORTED
    d = tau.make_desc(wl.prob, route=(1, 0, 0))
    d.n[0] = 6                       # FFT route needs n+1 = 2^p
    with pytest.raises(tau.TauError) as ei:
        tau.tau_create(d, 0)
    assert ei.value.status in (tau.TAU_EUNSUPPORTED, tau.TAU_ECUDA)


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2404_10221_gb300 import tau
    assert lib.tau_setup(None) == tau.TAU_EINVAL
    assert lib.tau_step(None, 1) == tau.TAU_EINVAL
    assert lib.tau_destroy(None) == tau.TAU_OK
    assert b"NULL" in lib.tau_last_error() or lib.tau_last_error() != b""


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    from paper_2404_10221_gb300 import tau
    monkeypatch.setattr(tau, "_lib", None)
    monkeypatch.setattr(tau, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        tau.lib()


def test_make_desc_marshals_problem():
    from paper_2404_10221_gb300 import tau, workloads
    wl = workloads.c3_3d(n=15, M=7)
    d = tau.make_desc(wl.prob)
    assert d.d == 3 and list(d.n) == [15, 15, 15] and d.M == 7
    assert list(d.alpha) == [1.2, 1.5, 1.9]
    assert math.isnan(d.e_min) and math.isnan(d.e_max)


def test_choose_precision_policy(lib):
    """tau_choose_precision runs on the host (no GPU).  Its verdicts agree with what the GPU solves
    showed: the FP32 inner solve of the mixed form converges on the 1-D workload at n = 5000
    (policy value 0.022) and on the 1023^2 and 255^3 workloads, and cannot resolve the operator of
    the 1-D workload at n = 65535 (eta ~ 3e6, value 1.05), where the double-float form is needed."""
    from paper_2404_10221_gb300 import tau
    from paper_2404_10221_gb300 import workloads as W
    cases = [(W.c1_1d(n=5000, M=3), tau.TAU_MIXED), (W.c1_1d(n=65535, M=3), tau.TAU_DF64),
             (W.c2_2d(), tau.TAU_MIXED), (W.c3_3d(), tau.TAU_MIXED), (W.c1_1d(), tau.TAU_MIXED)]
    for wl, want in cases:
        d = tau.make_desc(wl.prob, e_bounds=(1.0, 3.0))
        assert tau.tau_choose_precision(d) == want, wl.prob.n
    # the boundary moves with e_min: a 25x larger e_min brings n = 65535 under the bound
    d = tau.make_desc(W.c1_1d(n=65535, M=3).prob, e_bounds=(25.0, 30.0))
    assert tau.tau_choose_precision(d) == tau.TAU_MIXED
    # e_min unset (NaN) or not positive, or a bad order: argument errors, no GPU touched
    for bounds in (None, (0.0, 1.0), (-1.0, 1.0)):
        d = tau.make_desc(W.c1_1d(n=127).prob, e_bounds=bounds)
        with pytest.raises(tau.TauError):
            tau.tau_choose_precision(d)
    d = tau.make_desc(W.c1_1d(n=127).prob, e_bounds=(1.0, 2.0))
    d.alpha[0] = 2.0
    with pytest.raises(tau.TauError):
        tau.tau_choose_precision(d)


def test_noalloc_refuses_a_forced_route_before_any_device_call(lib):
    """tau_apply_A_noalloc picks its own route (FFT for n_i + 1 = 2^p, else dense sums); a caller
    that forces one gets TAU_EINVAL instead of a silently different route.  The check runs before
    any CUDA call, so non-null placeholder pointers suffice here."""
    import ctypes as C
    from paper_2404_10221_gb300 import tau, workloads
    wl = workloads.c2_2d(n=63, M=2)
    for route in (tau.TAU_ROUTE_FFT, tau.TAU_ROUTE_DENSE, tau.TAU_ROUTE_CHIRP, tau.TAU_ROUTE_LONG):
        d = tau.make_desc(wl.prob, route=(0, route, 0))
        fake = C.c_void_p(16)
        st = lib.tau_apply_A_noalloc(C.byref(d), fake, fake, fake, None)
        assert st == tau.TAU_EINVAL, route
        assert b"TAU_ROUTE_AUTO" in lib.tau_last_error()
