"""Two-sided τ-preconditioned GMRES (TPGM, Eq. (Pls)) on the GPU against the oracle's two-sided
solver: relative 2-norm <= 1e-10 at GMRES tol 1e-12, iteration counts within +-1."""

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
    (1, (127,), 8, 0),
    (1, (40,), 4, 1),          # dense route, previous-step initial guess
    (2, (31, 31), 4, 0),
    (2, (15, 63), 3, 1),
    (2, (12, 31), 3, 0),       # mixed routes
    (3, (7, 7, 7), 3, 0),
    (3, (15, 7, 31), 2, 1),
])
def test_tpgm_solve_matches_oracle(case):
    tau = _tau()
    d, n, M, x0 = case
    wl = _wl(d, n, M=M, x0_mode=x0)
    p = tau.Problem(wl, method=tau.TAU_TPGM)
    p.solve()
    u = p.solution().cpu().numpy()
    its = p.iters()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables(), sided=2)
    ref.run()
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= SOLVE_RTOL, rel
    assert np.all(np.abs(its - np.array(ref.iters)) <= 1), (its, ref.iters)


def test_tpgm_full_size_2d_against_one_sided():
    # both methods converge to A^{-1} b; the paper reports similar iteration numbers (Tables 2-4)
    tau = _tau()
    wl = W.c2_2d()
    a = tau.Problem(wl)
    a.step(2)
    ua = a.solution().cpu().numpy()
    ia = a.iters()[:2]
    a.close()
    b = tau.Problem(wl, method=tau.TAU_TPGM)
    b.step(2)
    ub = b.solution().cpu().numpy()
    ib = b.iters()[:2]
    b.close()
    assert np.linalg.norm(ub - ua) <= SOLVE_RTOL * np.linalg.norm(ua)
    assert np.all(np.abs(ib - ia) <= 3), (ia, ib)


def test_tpgm_in_a_batch_equals_alone():
    tau = _tau()
    rng = W.SplitMix64(4242)
    wls = [W.random_2d(rng, sizes=(15, 31, 63), M=3) for _ in range(3)]
    alone = []
    for wl in wls:
        p = tau.Problem(wl, method=tau.TAU_TPGM)
        p.solve()
        alone.append(p.solution().cpu().numpy())
        p.close()
    probs = [tau.Problem(wl, method=tau.TAU_TPGM if k != 1 else tau.TAU_OPGM) for k, wl in enumerate(wls)]
    bt = tau.tau_batch_create([p.handle for p in probs])
    tau.tau_batch_step(bt, 3)
    tau.tau_batch_sync(bt)
    tau.tau_batch_destroy(bt)
    for k, (ua, p) in enumerate(zip(alone, probs)):
        ub = p.solution().cpu().numpy()
        if k != 1:
            assert np.array_equal(ua, ub)
        else:
            assert np.linalg.norm(ub - ua) <= SOLVE_RTOL * np.linalg.norm(ua)
        p.close()


def test_tpgm_needs_fp64():
    tau = _tau()
    wl = _wl(1, (15,), M=2)
    with pytest.raises(tau.TauError):
        tau.Problem(wl, precision=tau.TAU_MIXED, method=tau.TAU_TPGM)
