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


def test_rhs_3d_matches_appendix_A_structure():
    """3-D F of reading R6 written out as Appendix A structures it: the interior term
    (B_3 ⊗ B_2 ⊗ B_1) f_int, then the boundary values of the padded grid entering through the faces
    (weight alpha_i/24 times the B of the two other axes), the edges (alpha_i alpha_j / 24^2 times the
    B of the third axis) and the corners (alpha_1 alpha_2 alpha_3 / 24^3).  Uneven sizes and random
    padded values, so a wrong axis, sign or weight in any term fails."""
    n1, n2, n3 = 4, 3, 5
    a = [1.3, 1.6, 1.9]
    p = _prob(3, [n1, n2, n3], a, [1.0, 1.0, 1.0])
    rng = np.random.default_rng(23)
    fp = rng.standard_normal((n3 + 2, n2 + 2, n1 + 2))      # fp[j3, j2, j1]
    B = [O.tridiag_B(a[0], n1), O.tridiag_B(a[1], n2), O.tridiag_B(a[2], n3)]
    w = [ai / 24.0 for ai in a]
    sl = slice(1, -1)

    def kron3(M3, M2, M1):
        return np.kron(M3, np.kron(M2, M1))

    def ends(n, lo, hi):
        # a vector over one axis holding boundary data at its two ends (the node next to each face)
        v = np.zeros(n)
        v[0], v[-1] = lo, hi
        return v

    F = kron3(B[2], B[1], B[0]) @ fp[sl, sl, sl].reshape(-1)
    # faces: for each axis, the two boundary planes, pushed to the adjacent interior layer
    for ax in range(3):
        G = np.zeros((n3, n2, n1))
        for side, idx in ((0, 0), (-1, -1)):
            if ax == 0:
                G[:, :, idx] += fp[sl, sl, 0 if side == 0 else -1]
            elif ax == 1:
                G[:, idx, :] += fp[sl, 0 if side == 0 else -1, sl]
            else:
                G[idx, :, :] += fp[0 if side == 0 else -1, sl, sl]
        Ms = [B[0], B[1], B[2]]
        Ms[ax] = w[ax] * np.eye([n1, n2, n3][ax])
        F += kron3(Ms[2], Ms[1], Ms[0]) @ G.reshape(-1)
    # edges: two axes on the boundary, the third interior
    for ax_free in range(3):
        axs = [i for i in range(3) if i != ax_free]
        G = np.zeros((n3, n2, n1))
        for s0 in (0, -1):
            for s1 in (0, -1):
                src = [None, None, None]
                dst = [slice(None), slice(None), slice(None)]
                src[ax_free] = sl
                for axb, sb in zip(axs, (s0, s1)):
                    src[axb] = 0 if sb == 0 else -1
                    dst[axb] = 0 if sb == 0 else -1
                # fp indexed [j3, j2, j1]; G likewise
                G[tuple(dst[::-1])] += fp[tuple(src[::-1])]
        Ms = [w[0] * np.eye(n1), w[1] * np.eye(n2), w[2] * np.eye(n3)]
        Ms[ax_free] = B[ax_free]
        F += kron3(Ms[2], Ms[1], Ms[0]) @ G.reshape(-1)
    # corners
    G = np.zeros((n3, n2, n1))
    for c3 in (0, -1):
        for c2 in (0, -1):
            for c1 in (0, -1):
                G[c3, c2, c1] += fp[c3, c2, c1]
    F += (w[0] * w[1] * w[2]) * G.reshape(-1)
    assert np.allclose(O.rhs_F(p, fp), F, rtol=1e-14, atol=1e-14)


def test_ebar_from_tables_closed_form_and_direct_evaluation():
    """Eqs. (bard), (dhat) on the 1-D workload e = 1 + 0.5 sin(pi x)(1 + t): over the interior grid
    (n odd, so x = 1/2 is a node) and t_{m+1/2}, the largest value is 1 + 0.5 (1 + t_{M-1/2}) and the
    smallest 1 + 0.5 sin(pi h)(1 + t_{1/2}); and on a 2-D workload the bounds equal those of e
    evaluated node by node from the workload's own closures."""
    wl = W.c1_1d(n=127, M=16)
    p = wl.prob
    t = wl.field_tables()
    ebar, ehat, echeck = O.ebar_from_tables(p, t["e_tc"], t["e_sp"])
    ts = p.half_times()
    h = p.h(0)
    assert abs(ehat - (1 + 0.5 * (1 + ts[-1]))) <= 1e-15
    assert abs(echeck - (1 + 0.5 * np.sin(np.pi * h) * (1 + ts[0]))) <= 1e-15
    assert abs(ebar - 0.5 * (ehat + echeck)) <= 1e-15
    wl2 = W.c2_2d(n=15, M=5)
    wl2.prob.n = [15, 9]
    wl2 = W.manufactured("e2", wl2.prob, wl2.e.terms, 2, 2, 1.0)
    p2 = wl2.prob
    t2 = wl2.field_tables()
    _, hi, lo = O.ebar_from_tables(p2, t2["e_tc"], t2["e_sp"])
    x = p2.grid(0)[1:-1]
    y = p2.grid(1)[1:-1]
    vals = []
    for tm in p2.half_times():
        for yy in y:
            for xx in x:
                vals.append(sum(tf(tm) * sf[0](xx) * sf[1](yy) for tf, sf in wl2.e.terms))
    assert abs(hi - max(vals)) <= 1e-14 and abs(lo - min(vals)) <= 1e-14
