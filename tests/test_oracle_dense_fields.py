"""The oracle's grid-array field form (fields of any shape, §1 Eq. (RSFDE)) pinned to its
separable-table form: the same separable workload given both ways yields the same right-hand sides
and the same time march, on uneven grids where a transposed axis or a shifted padded index would
show.  It also pins the array layout (x_1 fastest) against eval_field's."""

import numpy as np

import oracle as O
from paper_2404_10221_gb300 import workloads as W


def _as_arrays(wl):
    t = wl.field_tables()
    prob = wl.prob
    e = np.stack([O.eval_field_interior(prob, t["e_tc"][m], t["e_sp"]) for m in range(prob.M)])
    f = np.stack([O.eval_field(prob, t["f_tc"][m], t["f_sp"]).reshape(-1) for m in range(prob.M)])
    psi = O.eval_field_interior(prob, t["psi_tc"][0], t["psi_sp"])
    return t, {"e_dense": e, "f_dense": f, "psi_dense": psi}


def test_array_fields_reproduce_table_fields_2d_and_3d():
    for wl in (W.c2_2d(n=13, M=3), W.c3_3d(n=5, M=2)):
        wl.prob.n = [13, 9] if wl.prob.d == 2 else [5, 7, 4]
        wl = W.manufactured("uneven", wl.prob, wl.e.terms, 2, 2, 1.0)
        t, arr = _as_arrays(wl)
        a = O.OracleSolver(wl.prob, t)
        b = O.OracleSolver(wl.prob, arr)
        assert abs(a.ebar - b.ebar) <= 1e-15 * a.ebar
        for m in range(wl.prob.M):
            assert np.array_equal(a.e_at(m), b.e_at(m))
            np.testing.assert_allclose(b.F_at(m), a.F_at(m), rtol=0, atol=1e-14 * np.abs(a.F_at(m)).max())
        a.run()
        b.run()
        assert a.iters == b.iters
        assert np.linalg.norm(a.u - b.u) <= 1e-13 * np.linalg.norm(a.u)


def test_time_independent_e_and_zero_f_arrays():
    prob = W.Problem(d=2, n=[6, 5], alpha=[1.3, 1.7], kappa=[1.0, 0.4], M=2)
    arr = W.dense_fields(prob, time_dependent_e=False, with_f=False)
    s = O.OracleSolver(prob, arr)
    assert np.array_equal(s.e_at(0), s.e_at(1))
    assert np.all(s.F_at(1) == 0.0)
    # zero source: b = (B E - S) u, so one step equals the direct solve of that system
    s.step()
    e = s.e_at(0)
    u0 = arr["psi_dense"]
    b = O.rhs_b(prob, e, u0, np.zeros(prob.n_tot))
    np.testing.assert_allclose(s.u, O.step_direct(prob, e, b), rtol=0, atol=1e-10 * np.abs(s.u).max())


def test_dense_field_layout_is_x1_fastest():
    prob = W.Problem(d=2, n=[4, 3], alpha=[1.5, 1.5], kappa=[1.0, 1.0], M=1)
    arr = W.dense_fields(prob)
    x = prob.grid(0)[1:-1]
    y = prob.grid(1)[1:-1]
    t = prob.half_times()[0]
    # node (j1, j2) sits at index j2 * n_1 + j1
    for j2 in range(3):
        for j1 in range(4):
            want = 1.0 + x[j1] * y[j2] * np.exp(-t * x[j1])
            assert arr["e_dense"][0][j2 * 4 + j1] == want
