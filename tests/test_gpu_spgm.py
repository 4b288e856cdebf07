"""The Strang circulant comparison method (SPGM, Table 1, Eq. (Pcir)) on the GPU against the
oracle's SPGM: relative 2-norm <= 1e-10 at GMRES tol 1e-12, iteration counts within +-1."""

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    (1, (15,), 6, 0),
    (1, (40,), 4, 1),          # dense τ route, previous-step initial guess
    (2, (15, 15), 3, 0),
    (2, (12, 31), 3, 1),       # mixed τ routes
    (3, (7, 5, 7), 2, 0),
    (2, (70, 90), 2, 0),       # Hartley tiles of more than 8 x 128 values (16 lines of 70 or 90)
])
def test_spgm_solve_matches_oracle(case):
    tau = _tau()
    d, n, M, x0 = case
    wl = _wl(d, n, M=M, x0_mode=x0)
    p = tau.Problem(wl, method=tau.TAU_SPGM)
    p.solve()
    u = p.solution().cpu().numpy()
    its = p.iters()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables(), sided=3)
    ref.run()
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= 1e-10, rel
    assert np.all(np.abs(its - np.array(ref.iters)) <= 1), (its, ref.iters)


def test_spgm_needs_more_iterations_than_opgm_in_2d():
    # Table 3: the Strang circulant preconditioner needs far more iterations than the τ one in 2-D
    tau = _tau()
    wl = W.paper_example(2, [1.7, 1.9], 63, 4096)
    a = tau.Problem(wl)
    a.step(3)
    b = tau.Problem(wl, method=tau.TAU_SPGM)
    b.step(3)
    ia, ib = a.iters()[:3], b.iters()[:3]
    assert np.linalg.norm(b.solution().cpu().numpy() - a.solution().cpu().numpy()) <= 1e-8 * np.linalg.norm(
        a.solution().cpu().numpy())
    a.close()
    b.close()
    assert np.mean(ib) >= 2.0 * np.mean(ia), (ia, ib)


def test_spgm_needs_fp64():
    tau = _tau()
    with pytest.raises(tau.TauError):
        tau.Problem(_wl(1, (15,), M=2), precision=tau.TAU_DF64, method=tau.TAU_SPGM)
