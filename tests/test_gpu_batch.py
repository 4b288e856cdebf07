"""Batched form: many independent instances (uneven n, alpha, kappa, e) advanced by one graph
launch per step.  Each instance must give the same result alone and in the batch (the batch only
overlaps the instances' kernels; their arithmetic is unchanged), and agree with the oracle."""

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tau():
    from paper_2404_10221_gb300 import tau
    return tau


def _instances(count, sizes, M, seed):
    rng = W.SplitMix64(seed)
    return [W.random_2d(rng, sizes=sizes, M=M) for _ in range(count)]


def _alone(wl, precision):
    tau = _tau()
    p = tau.Problem(wl, precision=precision)
    p.solve()
    u = p.solution().cpu().numpy()
    its = p.iters()
    p.close()
    return u, its


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_alone(precision):
    tau = _tau()
    wls = _instances(7, (15, 31, 63, 127), 4, 10221 + precision)
    alone = [_alone(wl, precision) for wl in wls]
    probs = [tau.Problem(wl, precision=precision) for wl in wls]
    b = tau.tau_batch_create([p.handle for p in probs])
    tau.tau_batch_step(b, wls[0].prob.M)
    tau.tau_batch_sync(b)
    tau.tau_batch_destroy(b)
    for (ua, ia), p in zip(alone, probs):
        ub = p.solution().cpu().numpy()
        assert np.array_equal(ua, ub)
        assert np.array_equal(ia, p.iters())
        p.close()


def test_batch_matches_oracle_and_mixes_dimensions():
    tau = _tau()
    wls = _instances(3, (15, 31), 3, 777)
    one_d = W.c1_1d(n=63, M=3)
    three_d = W.c3_3d(n=7, M=3)
    wls += [one_d, three_d]
    probs = [tau.Problem(wl) for wl in wls]
    b = tau.tau_batch_create([p.handle for p in probs])
    tau.tau_batch_step(b, 3)
    assert tau.tau_batch_sync(b) == tau.TAU_OK
    tau.tau_batch_destroy(b)
    for wl, p in zip(wls, probs):
        u = p.solution().cpu().numpy()
        ref = O.OracleSolver(wl.prob, wl.field_tables())
        ref.run()
        assert np.linalg.norm(u - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
        p.close()


def test_batch_rejects_mismatched_steps():
    tau = _tau()
    a = tau.Problem(W.c1_1d(n=15, M=3))
    c = tau.Problem(W.c1_1d(n=15, M=4))
    with pytest.raises(tau.TauError):
        tau.tau_batch_create([a.handle, c.handle])
    a.close()
    c.close()


def test_batch_of_uneven_3d_instances():
    # d = 3 with uneven n_i per axis, FFT and dense routes mixed, in one batch
    tau = _tau()
    shapes = [(15, 7, 31), (7, 15, 3), (31, 3, 7), (12, 7, 15)]
    wls = []
    for k, n in enumerate(shapes):
        base = W.c3_3d(n=n[0], M=3)
        base.prob.n = list(n)
        base.prob.alpha = [1.2 + 0.1 * k, 1.5, 1.8 - 0.1 * k]
        wls.append(W.manufactured(f"3d_{n}", base.prob, base.e.terms, 2, 2, 1.0))
    alone = [_alone(wl, 0) for wl in wls]
    probs = [tau.Problem(wl) for wl in wls]
    b = tau.tau_batch_create([p.handle for p in probs])
    tau.tau_batch_step(b, 3)
    assert tau.tau_batch_sync(b) == tau.TAU_OK
    tau.tau_batch_destroy(b)
    for wl, (ua, ia), p in zip(wls, alone, probs):
        ub = p.solution().cpu().numpy()
        assert np.array_equal(ua, ub)
        ref = O.OracleSolver(wl.prob, wl.field_tables())
        ref.run()
        assert np.linalg.norm(ub - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
        p.close()
