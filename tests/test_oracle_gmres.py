"""Pins for the oracle's GMRES (Lemma Krylov, stopping rule of §4) and the
paper's convergence statements (Theorem GMRES, Theorem one-sidethm)."""

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W


def _system(d=2, n=(6, 5), seed=0):
    if d == 1:
        wl = W.c1_1d(n=n[0], M=8)
    elif d == 2:
        wl = W.c2_2d(n=n[0], M=8)
        wl.prob.n = list(n)
        wl = W.manufactured("t", wl.prob, wl.e.terms, 2, 2, 1.0)
    else:
        wl = W.c3_3d(n=n[0], M=8)
    p = wl.prob
    t = wl.field_tables()
    ebar = O.ebar_from_tables(p, t["e_tc"], t["e_sp"])[0]
    e = O.eval_field_interior(p, t["e_tc"][0], t["e_sp"])
    b = W.random_vector(p.n_tot, seed + 1)
    return p, e, b, ebar, t


@pytest.mark.parametrize("d,n", [(1, (15,)), (2, (6, 5)), (3, (4, 4, 4))])
def test_gmres_matches_direct_solve(d, n):
    p, e, b, ebar, _ = _system(d, n)
    res = O.gmres(lambda v: O.apply_A(p, e, v), b, np.zeros_like(b), 1e-13, 200,
                  lambda v: O.apply_Minv(p, ebar, v))
    x_dir = np.linalg.solve(O.dense_A(p, e), b)
    assert np.linalg.norm(res.x - x_dir) <= 1e-10 * np.linalg.norm(x_dir)
    # residual estimates are non-increasing (GMRES minimises over nested spaces)
    assert all(res.res[i + 1] <= res.res[i] * (1 + 1e-12) for i in range(len(res.res) - 1))
    # estimate equals the true preconditioned residual norm at the end
    r = O.apply_Minv(p, ebar, b - O.apply_A(p, e, res.x))
    assert abs(np.linalg.norm(r) - res.res[-1]) <= 1e-10 * res.res[0]


def test_gmres_basis_orthonormal():
    # Arnoldi basis of a well-converging run is orthonormal to working precision.
    p, e, b, ebar, _ = _system(2, (5, 4))
    res = O.gmres(lambda v: O.apply_A(p, e, v), b, np.zeros_like(b), 1e-30, 3,
                  lambda v: O.apply_Minv(p, ebar, v))
    V = res.basis
    assert V.shape[0] == 4
    assert np.allclose(V @ V.T, np.eye(V.shape[0]), atol=1e-12)


def test_a_form_equals_paper_form():
    # P^{-1} Ã = (B P)^{-1} A and P^{-1} b̃ = (B P)^{-1} b: same Krylov space and iterates.
    p, e, b, ebar, _ = _system(2, (5, 6))
    x0 = np.zeros_like(b)
    a = O.gmres(lambda v: O.apply_A(p, e, v), b, x0, 1e-12, 50, lambda v: O.apply_Minv(p, ebar, v))
    q = O.gmres_paper_form(p, e, b, x0, ebar, 1e-12, 50)
    assert a.iters == q.iters
    assert np.allclose(a.res, q.res, rtol=1e-9, atol=1e-14 * a.res[0])
    assert np.linalg.norm(a.x - q.x) <= 1e-11 * np.linalg.norm(q.x)


def test_one_sided_vs_two_sided_and_theorem_bound():
    # Theorem one-sidethm: ||r_j|| <= ebar^{-1/2} ||r̃_j|| with u^(0) = P^{-1/2} ũ^(0) = 0;
    # Theorem GMRES: ||r̃_k|| / ||r̃_0|| <= (2 + c) c^k.
    p, e, b, ebar, t = _system(2, (6, 5))
    _, ehat, echeck = O.ebar_from_tables(p, t["e_tc"], t["e_sp"])
    one = O.gmres_paper_form(p, e, b, np.zeros_like(b), ebar, 1e-14, 40)
    two = O.two_sided_gmres(p, e, b, ebar, 1e-14, 40)
    k = min(len(one.res), len(two.res))
    for j in range(1, k):
        assert one.res[j] <= two.res[j] / np.sqrt(ebar) * (1 + 1e-8) + 1e-15
    c = O.theorem_c(ehat, echeck)
    assert c < 1
    for j in range(1, len(two.res)):
        assert two.res[j] / two.res[0] <= (2 + c) * c ** j


def test_iteration_count_mesh_independent():
    # Theorem GMRES: the rate does not depend on N; iteration counts stay flat.
    its = []
    for n in (7, 15, 31):
        wl = W.paper_example(2, [1.3, 1.5], n, 4096)
        s = O.OracleSolver(wl.prob, wl.field_tables())
        s.run(steps=2)
        its.append(max(s.iters))
    assert max(its) - min(its) <= 1


@pytest.mark.parametrize("d,n", [(1, (9,)), (2, (6, 5)), (3, (3, 4, 3))])
def test_pmh_squares_to_P_inverse(d, n):
    # P^{-1/2} on the sine basis, applied twice, is P^{-1} of the dense assembly of Eq. (Pa)
    p, e, b, ebar, _ = _system(d, n)
    mu, beta = O.mu_tensor(p, ebar), O.beta_tensor(p)
    half = np.sqrt(beta / mu)
    r = O.apply_sine_diag(p, O.apply_sine_diag(p, b, half), half)
    ref = np.linalg.solve(O.dense_P(p, ebar), b)
    assert np.linalg.norm(r - ref) <= 1e-12 * np.linalg.norm(ref)
    # P^{-1/2} B^{-1} on the sine basis equals the dense eigh-based P^{-1/2} times B^{-1}
    pb = O.apply_sine_diag(p, b, 1.0 / np.sqrt(beta * mu))
    Bm = O.dense_B(p)
    w, Q = np.linalg.eigh(0.5 * (O.dense_P(p, ebar) + O.dense_P(p, ebar).T))
    ref2 = (Q * w ** -0.5) @ Q.T @ np.linalg.solve(Bm, b)
    assert np.linalg.norm(pb - ref2) <= 1e-11 * np.linalg.norm(ref2)


@pytest.mark.parametrize("d,n", [(1, (9,)), (2, (6, 5)), (3, (3, 4, 3))])
def test_two_sided_structured_equals_dense_form(d, n):
    # the structured TPGM runs the same Krylov iteration as the dense eigh-based form of Eq. (Pls)
    p, e, b, ebar, _ = _system(d, n)
    s = O.two_sided_structured(p, e, b, ebar, 1e-12, 60)
    q = O.two_sided_gmres(p, e, b, ebar, 1e-12, 60)
    assert s.iters == q.iters
    assert np.allclose(s.res, q.res, rtol=1e-8, atol=1e-13 * q.res[0])
    w, Q = np.linalg.eigh(0.5 * (O.dense_P(p, ebar) + O.dense_P(p, ebar).T))
    u_dense = (Q * w ** -0.5) @ Q.T @ q.x
    assert np.linalg.norm(s.x - u_dense) <= 1e-10 * np.linalg.norm(u_dense)
    x_dir = np.linalg.solve(O.dense_A(p, e), b)
    assert np.linalg.norm(s.x - x_dir) <= 1e-10 * np.linalg.norm(x_dir)


def test_two_sided_time_march_matches_one_sided():
    # both solvers converge to the same u^(m) (A^{-1} b each step); iteration counts are close
    # (Tables 2-4: OPGM and TPGM take similar iteration numbers)
    wl = W.paper_example(2, [1.3, 1.5], 15, 64)
    one = O.OracleSolver(wl.prob, wl.field_tables())
    two = O.OracleSolver(wl.prob, wl.field_tables(), sided=2)
    one.run(steps=3)
    two.run(steps=3)
    assert np.linalg.norm(one.u - two.u) <= 1e-10 * np.linalg.norm(one.u)
    assert all(abs(a - b) <= 2 for a, b in zip(one.iters, two.iters))
