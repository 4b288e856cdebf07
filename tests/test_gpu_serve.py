"""Served form: the continuous-batching request loop.

Requests of mixed dimension, size and precision are submitted together; each result must be the
same as solving that request alone (the loop only overlaps the requests' work on the device), and
admission must follow the device-memory budget."""

import numpy as np
import pytest

from paper_2404_10221_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tau():
    from paper_2404_10221_gb300 import tau
    return tau


def _mix(seed=20240416):
    rng = W.SplitMix64(seed)
    wls = []
    for k in range(6):
        wl = W.random_2d(rng, sizes=(15, 31, 63), M=3 + k % 3)
        wls.append(wl)
    wls.append(W.c1_1d(n=127, M=5))
    wls.append(W.c3_3d(n=15, M=3))
    precs = [0, 1, 0, 1, 0, 1, 0, 1]
    return wls, precs


def _alone(wl, precision):
    """The request solved alone, as the server runs it (mixed: inner solve on the line passes)."""
    tau = _tau()
    p = tau.Problem(wl, precision=precision, tc=tau.TAU_TC_OFF if precision == tau.TAU_MIXED else 0,
                    autotune=tau.TAU_TUNE_RECORDED)
    p.solve()
    u = p.solution().cpu().numpy()
    p.close()
    return u


def test_results_same_alone_and_in_the_mix():
    tau = _tau()
    wls, precs = _mix()
    s = tau.tau_server_create(8 << 30, 8, 2)
    ids = [tau.tau_server_submit(s, tau.make_desc(wl.prob, precision=pr), wl.field_tables())
           for wl, pr in zip(wls, precs)]
    infos = [tau.tau_server_wait(s, i, 300.0) for i in ids]
    assert all(inf.state == tau.TAU_REQ_DONE and inf.status == tau.TAU_OK for inf in infos)
    mixed = [tau.tau_server_result(s, i, wl.prob.n_tot) for i, wl in zip(ids, wls)]
    summ = tau.tau_server_summary(s)
    tau.tau_server_destroy(s)
    assert summ.completed == len(wls) and summ.failed == 0
    assert 0 < summ.latency_p50_s <= summ.latency_p99_s
    for wl, pr, um in zip(wls, precs, mixed):
        ua = _alone(wl, pr)
        assert np.array_equal(ua, um)


def test_admission_follows_memory_budget():
    tau = _tau()
    wls = [W.c2_2d(n=63, M=4) for _ in range(3)]
    desc = tau.make_desc(wls[0].prob)
    # estimate of one request: (max_iter + 11) n 8 bytes + 1 MiB; a budget for one at a time
    one = (desc.max_iter + 11) * wls[0].prob.n_tot * 8 + (1 << 20)
    s = tau.tau_server_create(int(one * 1.5), 8, 1)
    ids = [tau.tau_server_submit(s, desc, wl.field_tables()) for wl in wls]
    infos = [tau.tau_server_wait(s, i, 300.0) for i in ids]
    tau.tau_server_destroy(s)
    assert all(inf.state == tau.TAU_REQ_DONE for inf in infos)
    for a, b in zip(infos, infos[1:]):
        assert b.t_admit >= a.t_finish - 1e-6       # admitted only after memory was returned


def test_oversized_request_fails_fast():
    tau = _tau()
    wl = W.c2_2d(n=255, M=2)
    s = tau.tau_server_create(1 << 20, 4, 1)
    rid = tau.tau_server_submit(s, tau.make_desc(wl.prob), wl.field_tables())
    info = tau.tau_server_wait(s, rid, 10.0)
    tau.tau_server_destroy(s)
    assert info.state == tau.TAU_REQ_FAILED and info.status == tau.TAU_ENOMEM


def test_requests_share_launches_and_late_arrivals_join():
    """Mixed 2-D requests of different sizes and step counts batch their iterations together (shared
    launches of one group graph, rebuilt as requests finish or arrive); requests submitted while the
    first ones run are admitted and join; every result equals the request solved alone."""
    import time
    tau = _tau()
    rng = W.SplitMix64(777)
    early = [W.random_2d(rng, sizes=(31, 63, 127), M=6 + 2 * k) for k in range(4)]
    late = [W.random_2d(rng, sizes=(31, 63), M=4 + k) for k in range(3)]
    s = tau.tau_server_create(8 << 30, 16, 2)
    desc = lambda wl: tau.make_desc(wl.prob, precision=tau.TAU_MIXED)
    ids_e = [tau.tau_server_submit(s, desc(wl), wl.field_tables()) for wl in early]
    t_end = time.time() + 60
    while tau.tau_server_poll(s, ids_e[0]).state == tau.TAU_REQ_QUEUED and time.time() < t_end:
        time.sleep(0.001)
    ids_l = [tau.tau_server_submit(s, desc(wl), wl.field_tables()) for wl in late]
    ids = ids_e + ids_l
    infos = [tau.tau_server_wait(s, i, 300.0) for i in ids]
    res = [tau.tau_server_result(s, i, wl.prob.n_tot) for i, wl in zip(ids, early + late)]
    summ = tau.tau_server_summary(s)
    tau.tau_server_destroy(s)
    assert all(inf.state == tau.TAU_REQ_DONE and inf.status == tau.TAU_OK for inf in infos)
    assert summ.group_launches > 0 and summ.group_rebuilds >= 2, (summ.group_launches, summ.group_rebuilds)
    assert summ.group_request_steps > summ.group_launches
    # at least one late request was admitted before the last early one finished
    assert min(infos[len(early) + k].t_admit for k in range(len(late))) < max(inf.t_finish for inf in infos[:len(early)])
    for wl, u in zip(early + late, res):
        assert np.array_equal(_alone(wl, tau.TAU_MIXED), u)


def test_served_results_match_the_oracle():
    """Requests of each kind the server handles (shared launches for small mixed requests, a
    double-float request, a plain FP64 one, a 1-D one on its own stream) against the oracle: the
    form's bar for the mixed and double-float requests, the plain bar for FP64."""
    import oracle as O
    tau = _tau()
    rng = W.SplitMix64(4040)
    wls = [W.random_2d(rng, sizes=(31, 63), M=3) for _ in range(3)]
    wls += [W.c3_3d(n=15, M=3), W.c1_1d(n=127, M=3), W.c2_2d(n=31, M=3)]
    precs = [tau.TAU_MIXED, tau.TAU_MIXED, tau.TAU_MIXED, tau.TAU_MIXED, tau.TAU_DF64, tau.TAU_FP64]
    s = tau.tau_server_create(8 << 30, 8, 2)
    ids = [tau.tau_server_submit(s, tau.make_desc(wl.prob, precision=pr), wl.field_tables())
           for wl, pr in zip(wls, precs)]
    infos = [tau.tau_server_wait(s, i, 300.0) for i in ids]
    got = [tau.tau_server_result(s, i, wl.prob.n_tot) for i, wl in zip(ids, wls)]
    tau.tau_server_destroy(s)
    assert all(inf.state == tau.TAU_REQ_DONE and inf.status == tau.TAU_OK for inf in infos)
    for wl, pr, u in zip(wls, precs, got):
        ref = O.OracleSolver(wl.prob, wl.field_tables())
        ref.run()
        bar = 1e-10 if pr == tau.TAU_FP64 else 1e-8
        assert np.linalg.norm(u - ref.u) <= bar * np.linalg.norm(ref.u), (wl.prob.n, pr)
