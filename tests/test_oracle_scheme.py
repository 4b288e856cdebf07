"""Pins for the whole scheme (§2 time marching, §4 experiments): spatial
convergence order on the paper's manufactured solutions, the Iter columns and
(soft) the Error columns of Tables 2-4, and GMRES time-marching vs the direct
solve of every step."""

import os

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def _error(wl, direct=True, steps=None):
    s = O.OracleSolver(wl.prob, wl.field_tables())
    s.run(steps=steps, direct=direct)
    return O.l2_error(wl.prob, s.u, wl.exact(wl.prob.T)), s


@pytest.mark.parametrize("alpha", [1.3, 1.5, 1.9])
def test_example1_fourth_order_and_table2(alpha):
    rows = [r for r in _load("table2_example1.txt") if r[0] == alpha]
    errs = {}
    for a, M, Np1, err_paper, it_opgm, _ in rows[:2]:
        wl = W.paper_example(1, [alpha], int(Np1) - 1, int(M))
        errs[int(Np1)], _ = _error(wl)
    ratio = errs[16] / errs[32]
    paper_ratio = rows[0][3] / rows[1][3]
    # hard pin: 4th order in h with the paper's own ratio (Table 2) within 10 %
    assert 14.0 < ratio < 20.0
    assert abs(ratio / paper_ratio - 1) < 0.10
    # soft pin: magnitude within one decade of the printed Error column
    assert 0.1 < errs[16] / rows[0][3] < 10


@pytest.mark.parametrize("row", _load("table2_example1.txt"))
def test_example1_iterations_table2(row):
    alpha, M, Np1, _, it_paper, _ = row
    wl = W.paper_example(1, [alpha], int(Np1) - 1, int(M))
    s = O.OracleSolver(wl.prob, wl.field_tables())
    s.run(steps=40)
    assert abs(np.mean(s.iters) - it_paper) <= 1.0


@pytest.mark.parametrize("row", _load("table2_example1.txt"))
def test_example1_two_sided_iterations_table2(row):
    # the TPGM column of Table 2: GMRES on Eq. (Pls)
    alpha, M, Np1, _, _, it_paper = row
    wl = W.paper_example(1, [alpha], int(Np1) - 1, int(M))
    s = O.OracleSolver(wl.prob, wl.field_tables(), sided=2)
    s.run(steps=40)
    assert abs(np.mean(s.iters) - it_paper) <= 1.0


@pytest.mark.parametrize("row", _load("table3_example2.txt"))
def test_example2_iterations_table3(row):
    a1, a2, M, Np1, _, it_paper = row
    wl = W.paper_example(2, [a1, a2], int(Np1) - 1, int(M))
    s = O.OracleSolver(wl.prob, wl.field_tables())
    s.run(steps=6)
    assert abs(np.mean(s.iters) - it_paper) <= 1.0


@pytest.mark.parametrize("row", _load("table4_example3.txt"))
def test_example3_iterations_table4(row):
    a1, a2, a3, M, Np1, _, it_paper = row
    wl = W.paper_example(3, [a1, a2, a3], int(Np1) - 1, int(M))
    s = O.OracleSolver(wl.prob, wl.field_tables())
    s.run(steps=3)
    assert abs(np.mean(s.iters) - it_paper) <= 1.0


def test_example2_fourth_order_table3():
    rows = _load("table3_example2.txt")[2:4]           # (1.3, 1.5), N+1 = 16, 32
    errs = []
    for a1, a2, M, Np1, err_paper, _ in rows:
        wl = W.paper_example(2, [a1, a2], int(Np1) - 1, 256)
        errs.append(_error(wl)[0])
    ratio = errs[0] / errs[1]
    paper_ratio = rows[0][4] / rows[1][4]
    assert 14.0 < ratio < 20.0
    assert abs(ratio / paper_ratio - 1) < 0.15
    assert 0.1 < errs[0] / rows[0][4] < 10


def test_gmres_march_matches_direct_march():
    wl = W.c1_1d(n=31, M=8)
    _, sg = _error(wl, direct=False)
    _, sd = _error(wl, direct=True)
    assert np.linalg.norm(sg.u - sd.u) <= 1e-10 * np.linalg.norm(sd.u)


def test_x0_previous_mode_same_solution():
    wl = W.c2_2d(n=7, M=4)
    s0 = O.OracleSolver(wl.prob, wl.field_tables())
    s0.run()
    wl.prob.x0_mode = 1
    s1 = O.OracleSolver(wl.prob, wl.field_tables())
    s1.run()
    assert np.linalg.norm(s0.u - s1.u) <= 1e-10 * np.linalg.norm(s0.u)
