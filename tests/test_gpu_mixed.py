"""Mixed-precision form: FP64 iterative refinement around an FP32 flexible GMRES.

FP32 operators are compared with the FP64 oracle at single-precision tolerances; whole solves
must agree with the FP64 oracle (and with the plain FP64 GPU path) to a relative 2-norm of 1e-8,
the accuracy bar the precision form is held to.
"""

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS32 = float(np.finfo(np.float32).eps)
MIXED_RTOL = 1e-8


def _tau():
    from paper_2404_10221_gb300 import tau
    return tau


def _wl(d, n, M=3, x0_mode=0):
    if d == 1:
        wl = W.c1_1d(n=n[0], M=M)
    elif d == 2:
        base = W.c2_2d(n=n[0], M=M)
        base.prob.n = list(n)
        wl = W.manufactured(f"2d_{n}", base.prob, base.e.terms, 2, 2, 1.0)
    else:
        base = W.c3_3d(n=n[0], M=M)
        base.prob.n = list(n)
        wl = W.manufactured(f"3d_{n}", base.prob, base.e.terms, 2, 2, 1.0)
    wl.prob.x0_mode = x0_mode
    return wl


def _f32(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to("cuda")


def minv_rtol32(prob, ebar):
    eta = O.etas(prob)
    l1 = [2 * O.fcd_weights(prob.alpha[i], prob.n[i])[0] for i in range(prob.d)]
    kappa_q = sum(eta[i] * l1[i] for i in range(prob.d)) / O.mu_tensor(prob, ebar).min()
    return 1e-5 + 4 * EPS32 * kappa_q


@pytest.mark.parametrize("d,n", [(1, (127,)), (1, (100,)), (2, (31, 63)), (2, (20, 9)), (3, (15, 7, 31))])
def test_fp32_operators_parity(d, n):
    tau = _tau()
    wl = _wl(d, n)
    pr = wl.prob
    # the FP32 line passes (the tensor-core DST has its own bound, tests/test_gpu_tc.py)
    p = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_OFF)
    t = wl.field_tables()
    ebar = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])[0]
    x = W.random_vector(pr.n_tot, 31)
    y = torch.empty(pr.n_tot, dtype=torch.float32, device="cuda")
    m = 1
    tau.tau_apply_A_f32(p.handle, m, _f32(x), y)
    torch.cuda.synchronize()
    e = O.eval_field_interior(pr, t["e_tc"][m], t["e_sp"])
    ref = O.apply_A(pr, e, x.astype(np.float32).astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    tau.tau_apply_Minv_f32(p.handle, _f32(x), y)
    torch.cuda.synchronize()
    ref = O.apply_Minv(pr, ebar, x.astype(np.float32).astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= minv_rtol32(pr, ebar)
    p.close()


@pytest.mark.parametrize("case", [
    (1, (127,), 32, 0),
    (1, (40,), 4, 1),
    (2, (31, 31), 4, 0),
    (2, (15, 63), 3, 1),
    (3, (7, 7, 7), 3, 0),
    (3, (15, 7, 31), 2, 0),
])
def test_mixed_solve_matches_fp64_oracle(case):
    tau = _tau()
    d, n, M, x0 = case
    wl = _wl(d, n, M=M, x0_mode=x0)
    p = tau.Problem(wl, precision=tau.TAU_MIXED)
    p.solve()
    u = p.solution().cpu().numpy()
    st = p.stats()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run()
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= MIXED_RTOL, rel
    assert st.steps_done == M and st.total_sweeps >= M


def test_mixed_full_size_2d_against_plain_fp64_path():
    """The 1023^2 workload: three steps of the mixed form against the plain FP64 GPU path."""
    tau = _tau()
    wl = W.c2_2d()
    a = tau.Problem(wl)
    a.step(3)
    ua = a.solution().cpu().numpy()
    a.close()
    b = tau.Problem(wl, precision=tau.TAU_MIXED)
    b.step(3)
    ub = b.solution().cpu().numpy()
    st = b.stats()
    b.close()
    rel = np.linalg.norm(ub - ua) / np.linalg.norm(ua)
    assert rel <= MIXED_RTOL, rel
    assert st.steps_done == 3


def test_mixed_notconv_reported_when_sweeps_capped():
    tau = _tau()
    wl = _wl(2, (31, 31), M=2)
    p = tau.Problem(wl, precision=tau.TAU_MIXED, refine_tol=1e-15, max_sweeps=1, inner_max_iter=2)
    st = p.solve(allow_notconv=True)
    assert st == tau.TAU_ENOTCONV
    p.close()


def test_mixed_resume_matches_straight_run():
    """From the second step on the mixed form forms each right-hand side from the previous step's
    FP64 residual; a solution set by the caller (checkpoint resume) drops back to the line passes.
    Both routes give the same march within the form's rounding."""
    tau = _tau()
    wl = _wl(3, (15, 7, 31), M=6)
    a = tau.Problem(wl, precision=tau.TAU_MIXED)
    a.solve()
    ua = a.solution().cpu().numpy()
    a.close()
    b = tau.Problem(wl, precision=tau.TAU_MIXED)
    b.step(3)
    mid = b.solution().cpu().numpy()
    b.close()
    c = tau.Problem(wl, precision=tau.TAU_MIXED)
    tau.tau_set_solution(c.handle, mid, False, 3)
    c.step(3)
    uc = c.solution().cpu().numpy()
    c.close()
    assert np.linalg.norm(uc - ua) <= 1e-10 * np.linalg.norm(ua)
