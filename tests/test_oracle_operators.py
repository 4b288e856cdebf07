"""Pins for the oracle's operators: dense Kronecker assembly vs structured mode
products (Eqs. (tls), (Salpha), (Ha)), the preconditioner M = ebar B + tau(S)
and its DST diagonalisation (Eqs. (Pa), (tauSalpha), (diag), Lemma le:eig),
the commutation remark of §3, Lemma PSPD, and the right-hand side of
Appendix A."""

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

CASES = [
    (1, [1], [1.5], [1.0]),
    (1, [7], [1.3], [2.0]),
    (1, [16], [1.9], [0.5]),
    (2, [3, 4], [1.4, 1.8], [1.0, 0.5]),
    (2, [5, 2], [1.1, 1.7], [0.3, 1.2]),
    (3, [3, 2, 4], [1.2, 1.5, 1.9], [1.0, 1.0, 0.5]),
]


def _prob(d, n, alpha, kappa, M=4):
    return W.Problem(d=d, n=list(n), alpha=list(alpha), kappa=list(kappa), T=1.0, M=M)


@pytest.mark.parametrize("case", CASES)
def test_structured_A_matches_dense(case):
    p = _prob(*case)
    e = W.random_positive(p.n_tot, 1)
    x = W.random_vector(p.n_tot, 2)
    A = O.dense_A(p, e)
    assert np.allclose(O.apply_A(p, e, x), A @ x, rtol=1e-13, atol=1e-12)
    # S symmetric (sum of Kronecker products of symmetric factors)
    S = O.dense_S(p)
    assert np.allclose(S, S.T)
    assert np.allclose(O.apply_S(p, x), S @ x, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("case", CASES)
def test_Minv_dst_matches_dense_solve(case):
    p = _prob(*case)
    ebar = 1.7
    r = W.random_vector(p.n_tot, 5)
    M = O.dense_M(p, ebar)
    z_dense = np.linalg.solve(M, r)
    z = O.apply_Minv(p, ebar, r)
    assert np.linalg.norm(z - z_dense) <= 1e-13 * np.linalg.norm(z_dense) * p.n_tot


@pytest.mark.parametrize("case", CASES)
def test_mu_are_eigenvalues_of_M(case):
    p = _prob(*case)
    ebar = 0.9
    M = O.dense_M(p, ebar)
    assert np.allclose(M, M.T)
    ev = np.sort(np.linalg.eigvalsh(M))
    mu = np.sort(O.mu_tensor(p, ebar))
    assert np.allclose(ev, mu, rtol=1e-12)


@pytest.mark.parametrize("case", CASES)
def test_commutation_and_P_spd(case):
    p = _prob(*case)
    B = O.dense_B(p)
    tS = O.dense_tauS(p)
    # §3: B tau(S) = tau(S) B, hence B^{-1/2} tau(S) B^{-1/2} = B^{-1} tau(S)
    assert np.allclose(B @ tS, tS @ B, atol=1e-12 * np.abs(tS).max())
    w, Q = np.linalg.eigh(B)
    Bmh = (Q * w ** -0.5) @ Q.T
    assert np.allclose(Bmh @ tS @ Bmh, np.linalg.solve(B, tS), atol=1e-11 * np.abs(tS).max())
    # Lemma PSPD and ||P^{-1}|| <= 1/ebar (proof of Theorem one-sidethm)
    ebar = 1.3
    P = O.dense_P(p, ebar)
    assert np.allclose(P, P.T, atol=1e-11 * np.abs(P).max())
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0
    assert np.linalg.norm(np.linalg.inv(P), 2) <= 1.0 / ebar * (1 + 1e-12)


def test_rhs_1d_matches_appendix_A():
    # 1-D: F = B f + (alpha_1/24) f_0, f_0 = [f(L),0..0,f(R)].
    p = _prob(1, [9], [1.3], [1.0])
    rng = np.random.default_rng(7)
    fpad = rng.standard_normal(11)
    f0 = np.zeros(9)
    f0[0], f0[-1] = fpad[0], fpad[-1]
    F_app = O.tridiag_B(1.3, 9) @ fpad[1:-1] + (1.3 / 24) * f0
    assert np.allclose(O.rhs_F(p, fpad), F_app, rtol=1e-14, atol=1e-14)


def test_rhs_2d_matches_appendix_A():
    # 2-D form of Appendix A, written out term by term.
    N, a1, a2 = 5, 1.4, 1.8
    p = _prob(2, [N, N], [a1, a2], [1.0, 1.0])
    rng = np.random.default_rng(11)
    fp = rng.standard_normal((N + 2, N + 2))     # fp[j2, j1]
    B1, B2 = O.tridiag_B(a1, N), O.tridiag_B(a2, N)
    f_int = fp[1:-1, 1:-1].reshape(-1)
    f1 = np.zeros((N, N))
    f1[:, 0] = fp[1:-1, 0]
    f1[:, -1] = fp[1:-1, -1]
    g1 = fp[0, 1:-1]
    g2 = fp[-1, 1:-1]
    g3 = np.zeros(N)
    g3[0], g3[-1] = fp[0, 0], fp[0, -1]
    g4 = np.zeros(N)
    g4[0], g4[-1] = fp[-1, 0], fp[-1, -1]
    F = np.kron(B2, B1) @ f_int + np.kron(B2, a1 / 24 * np.eye(N)) @ f1.reshape(-1)
    blk = np.zeros((N, N))
    blk[0], blk[-1] = B1 @ g1, B1 @ g2
    F += a2 / 24 * blk.reshape(-1)
    blk = np.zeros((N, N))
    blk[0], blk[-1] = g3, g4
    F += a1 * a2 / 24 ** 2 * blk.reshape(-1)
    assert np.allclose(O.rhs_F(p, fp), F, rtol=1e-14, atol=1e-14)


def test_rhs_b_definition():
    p = _prob(2, [4, 3], [1.4, 1.8], [1.0, 0.5])
    e = W.random_positive(p.n_tot, 3)
    u = W.random_vector(p.n_tot, 4)
    F = W.random_vector(p.n_tot, 5)
    b = O.rhs_b(p, e, u, F)
    ref = (O.dense_B(p) @ np.diag(e) - O.dense_S(p)) @ u + p.dt * F
    assert np.allclose(b, ref, rtol=1e-13, atol=1e-13)


def test_field_tables_evaluate_separable_sum():
    wl = W.c2_2d(n=6, M=3)
    t = wl.field_tables()
    p = wl.prob
    m = 1
    tm = p.half_times()[m]
    ev = O.eval_field_interior(p, t["e_tc"][m], t["e_sp"])
    x = p.grid(0)[1:-1]
    y = p.grid(1)[1:-1]
    ref = 2 + np.outer(np.cos(np.pi * y), np.sin(np.pi * x)) * (1 + tm)
    assert np.allclose(ev, ref.reshape(-1), rtol=1e-14)
