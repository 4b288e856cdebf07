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


# ---- grouped execution: one launch per kernel for all problems of a group ----------------------

def _mixed_instances(shapes, M, seed, d=2, x0_mode=0):
    """Mixed-precision instances with uneven n per axis and random alpha, kappa, e amplitude."""
    rng = W.SplitMix64(seed)
    out = []
    for n in shapes:
        if d == 2:
            wl = W.random_2d(rng, sizes=(n[0],), M=M)
            wl.prob.n = list(n)
            wl = W.manufactured(wl.name, wl.prob, wl.e.terms, 2, 2, 1.0)
        else:
            base = W.c3_3d(n=n[0], M=M)
            base.prob.n = list(n)
            base.prob.alpha = [1.1 + 0.8 * rng.uniform() for _ in range(3)]
            wl = W.manufactured("g3", base.prob, base.e.terms, 2, 2, 1.0)
        wl.prob.x0_mode = x0_mode
        out.append(wl)
    return out


def _expected_groups(probs, grouped=True):
    """(groups, problems in them): problems group by (d, residual precision, x0 mode), at least two
    to a group; the residual precision is the one tau_setup chose for each problem."""
    keys = {}
    for p in probs:
        st = p.stats()
        k = (p.prob.d, int(st.resid_precision), int(p.prob.x0_mode))
        keys[k] = keys.get(k, 0) + 1
    if not grouped:
        return 0, 0
    big = [v for v in keys.values() if v >= 2]
    return len(big), sum(big)


def _run_batch(wls, **kw):
    tau = _tau()
    probs = [tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_OFF) for wl in wls]
    b = tau.tau_batch_create([p.handle for p in probs])
    info = tau.tau_batch_get_info(b)
    assert (info.groups, info.grouped_problems) == _expected_groups(probs, kw.get("grouped", True)), info
    tau.tau_batch_step(b, wls[0].prob.M)
    tau.tau_batch_sync(b)
    tau.tau_batch_destroy(b)
    out = [(p.solution().cpu().numpy(), p.iters(), int(p.stats().total_sweeps)) for p in probs]
    for p in probs:
        p.close()
    return info, out


def _alone_mixed(wl):
    tau = _tau()
    p = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_OFF)
    p.solve()
    r = (p.solution().cpu().numpy(), p.iters(), int(p.stats().total_sweeps))
    p.close()
    return r


def test_grouped_batch_equals_alone_and_oracle():
    """Nine uneven 2-D instances, sizes from 3 to 127 per axis (so some finish their loops long
    before others): one group, every kernel one launch for all nine, results bit-identical to each
    instance alone (same kernels, tiles and reduction order) and within the form's bar of the
    oracle."""
    shapes = [(3, 5), (127, 63), (15, 31), (63, 63), (7, 127), (31, 15), (127, 127), (5, 3), (63, 7)]
    wls = _mixed_instances(shapes, 4, 4242)
    info, got = _run_batch(wls)
    assert info.groups >= 1 and info.grouped_problems >= len(wls) - 1, info
    assert info.launches_per_inner_iter > 0
    for wl, (ub, ib, sb) in zip(wls, got):
        ua, ia, sa = _alone_mixed(wl)
        assert np.array_equal(ua, ub)
        assert np.array_equal(ia, ib) and sa == sb
        ref = O.OracleSolver(wl.prob, wl.field_tables())
        ref.run()
        assert np.linalg.norm(ub - ref.u) <= 1e-8 * np.linalg.norm(ref.u)


def test_grouped_batch_mixes_dimensions_and_precisions():
    """2-D and 3-D mixed instances form one group each; a plain FP64 instance and a 1-D one take
    their own branches; x0 = previous step in a third group.  All match their runs alone."""
    tau = _tau()
    wls2 = _mixed_instances([(15, 31), (31, 15), (63, 31)], 3, 11)
    wls3 = _mixed_instances([(7, 15, 11), (15, 7, 7)], 3, 12, d=3)
    wlsp = _mixed_instances([(31, 31), (15, 63)], 3, 13, x0_mode=1)
    plain = W.c2_2d(n=31, M=3)
    one_d = W.c1_1d(n=63, M=3)
    mixed = wls2 + wls3 + wlsp
    alone = [_alone_mixed(wl) for wl in mixed]
    probs = [tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_OFF) for wl in mixed]
    probs += [tau.Problem(plain), tau.Problem(one_d, precision=tau.TAU_MIXED, tc=tau.TAU_TC_OFF)]
    b = tau.tau_batch_create([p.handle for p in probs])
    info = tau.tau_batch_get_info(b)
    tau.tau_batch_step(b, 3)
    assert tau.tau_batch_sync(b) == tau.TAU_OK
    tau.tau_batch_destroy(b)
    groups, grouped = _expected_groups(probs[:len(mixed)])
    assert (info.groups, info.grouped_problems) == (groups, grouped), info
    assert groups >= 2 and info.branches == groups + len(probs) - grouped, info
    for (ua, ia, _), p in zip(alone, probs):
        assert np.array_equal(ua, p.solution().cpu().numpy())
        assert np.array_equal(ia, p.iters())
    for wl, p in zip([plain, one_d], probs[len(mixed):]):
        ref = O.OracleSolver(wl.prob, wl.field_tables())
        ref.run()
        u = p.solution().cpu().numpy()
        assert np.linalg.norm(u - ref.u) <= 1e-8 * np.linalg.norm(ref.u)
    for p in probs:
        p.close()


def test_grouping_off_gives_the_same_results(monkeypatch):
    shapes = [(15, 31), (63, 15), (31, 31), (7, 63)]
    wls = _mixed_instances(shapes, 3, 99)
    info_g, got_g = _run_batch(wls)
    monkeypatch.setenv("TAU_BATCH_GROUPS", "0")
    info_b, got_b = _run_batch(wls, grouped=False)
    assert info_g.groups >= 1 and info_b.groups == 0 and info_b.branches == len(wls)
    for (ug, ig, _), (ub, ib, _) in zip(got_g, got_b):
        assert np.array_equal(ug, ub) and np.array_equal(ig, ib)


def test_grouped_batch_with_tuned_tiles_equals_alone(monkeypatch):
    """With the tile autotuner on, problems of different shapes may run different line-pass
    kernels (128 or 256 threads per CTA, different lines per CTA) at the same position of the step;
    the group then splits that position into one grouped launch per kernel.  Results stay
    bit-identical to each problem alone (the tuner's choices are recorded per shape, so the alone
    runs take the same tiles)."""
    monkeypatch.setenv("TAU_AUTOTUNE", "1")
    shapes = [(255, 63), (127, 255), (63, 63), (255, 255), (31, 127)]
    wls = _mixed_instances(shapes, 3, 515)
    info, got = _run_batch(wls)
    assert info.groups >= 1
    for wl, (ub, ib, sb) in zip(wls, got):
        ua, ia, sa = _alone_mixed(wl)
        assert np.array_equal(ua, ub)
        assert np.array_equal(ia, ib) and sa == sb
