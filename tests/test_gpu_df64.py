"""TAU_DF64: the plain method in double-float arithmetic (pairs of FP32 numbers) on the FP32 pipes.
Held to the plain FP64 path's bar: relative 2-norm <= 1e-10 against the FP64 oracle at GMRES tol
1e-12, iteration counts within +-1."""

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOLVE_RTOL = 1e-10


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


@pytest.mark.parametrize("case", [
    (1, (127,), 32, 0),
    (1, (40,), 4, 1),          # dense route, previous-step initial guess
    (2, (31, 31), 4, 0),
    (2, (15, 63), 3, 1),
    (2, (12, 31), 3, 0),       # mixed routes
    (3, (7, 7, 7), 3, 0),
    (3, (15, 7, 31), 2, 0),
])
def test_df64_solve_matches_oracle(case):
    tau = _tau()
    d, n, M, x0 = case
    wl = _wl(d, n, M=M, x0_mode=x0)
    p = tau.Problem(wl, precision=tau.TAU_DF64)
    p.solve()
    u = p.solution().cpu().numpy()
    its = p.iters()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run()
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= SOLVE_RTOL, rel
    assert np.all(np.abs(its - np.array(ref.iters)) <= 1), (its, ref.iters)


def test_df64_full_size_2d_against_plain_fp64():
    tau = _tau()
    wl = W.c2_2d()
    a = tau.Problem(wl)
    a.step(3)
    ua = a.solution().cpu().numpy()
    ia = a.iters()[:3]
    a.close()
    b = tau.Problem(wl, precision=tau.TAU_DF64)
    b.step(3)
    ub = b.solution().cpu().numpy()
    ib = b.iters()[:3]
    b.close()
    assert np.linalg.norm(ub - ua) <= SOLVE_RTOL * np.linalg.norm(ua)
    assert np.all(np.abs(ib - ia) <= 1), (ia, ib)


def test_df64_checkpoint_roundtrip_is_exact_to_fp64():
    tau = _tau()
    wl = _wl(2, (31, 15), M=4)
    p = tau.Problem(wl, precision=tau.TAU_DF64)
    p.step(2)
    u = p.solution().cpu().numpy()
    tau.tau_set_solution(p.handle, u, False, 2)
    u2 = p.solution().cpu().numpy()
    p.close()
    # a double -> double-float -> double round trip keeps about 48 bits
    assert np.max(np.abs(u2 - u)) <= 2.0 ** -46 * np.max(np.abs(u))
