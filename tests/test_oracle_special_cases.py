"""Special cases that reduce the scheme to something known (§2-§3), as pins for the oracle.

- kappa = 0: no fractional term, so S = 0, A = B E and M = ebar B.
- Constant e = c: ebar = c, so A - M = S - τ(S), the Hankel part of every fractional factor; the
  preconditioner is exact up to it.
- alpha = 2 (the limit of the weights: s_0 = 2, s_1 = -1, s_k = 0 for k >= 2): every Toeplitz
  factor is tridiagonal and so equal to its τ matrix, the scheme is the classical fourth-order
  compact one (B = I + (1/12) tridiag(1, -2, 1)), and with constant e, M = A: preconditioned GMRES
  converges in one iteration.
"""

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W


def _prob(n, alpha, kappa, M=10):
    d = len(n)
    return W.Problem(d=d, n=list(n), alpha=list(alpha), kappa=list(kappa), T=1.0, M=M)


@pytest.mark.parametrize("n", [(9,), (5, 4), (3, 4, 2)])
def test_kappa_zero_leaves_B_E(n):
    d = len(n)
    p = _prob(n, [1.3, 1.6, 1.8][:d], [0.0] * d)
    N = int(np.prod(n))
    e = 1.0 + W.random_vector(N, 3) ** 2
    x = W.random_vector(N, 4)
    assert np.abs(O.dense_S(p)).max() == 0.0
    assert np.allclose(O.dense_A(p, e), O.dense_B(p) @ np.diag(e), rtol=0, atol=1e-14)
    assert np.allclose(O.apply_A(p, e, x), O.apply_B(p, e * x), rtol=0, atol=1e-13)
    ebar = 1.7
    z = O.apply_Minv(p, ebar, x)
    assert np.allclose(z, np.linalg.solve(ebar * O.dense_B(p), x), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [(12,), (6, 5), (4, 3, 3)])
def test_constant_e_leaves_only_the_hankel_part(n):
    d = len(n)
    p = _prob(n, [1.3, 1.6, 1.8][:d], [1.0, 0.7, 0.4][:d])
    N = int(np.prod(n))
    c = 2.5
    A = O.dense_A(p, np.full(N, c))
    M = O.dense_M(p, c)
    S, tS = O.dense_S(p), O.dense_tauS(p)
    assert np.allclose(A - M, S - tS, rtol=0, atol=1e-12 * np.abs(S).max())
    # along one dimension, T - τ(T) is the Hankel matrix H(T) of the weights
    t = O.fcd_weights(p.alpha[0], n[0])
    T = O.toeplitz_S(p.alpha[0], n[0])
    assert np.allclose(T - O.tau_of(t), O.hankel_H(t), rtol=0, atol=1e-14)


@pytest.mark.parametrize("n", [(15,), (7, 6), (4, 5, 3)])
def test_alpha_two_makes_the_preconditioner_exact(n):
    d = len(n)
    p = _prob(n, [2.0] * d, [1.0, 0.5, 0.8][:d])
    for i in range(d):
        t = O.fcd_weights(2.0, n[i])
        assert t[0] == pytest.approx(2.0) and t[1] == pytest.approx(-1.0) and np.all(np.abs(t[2:]) < 1e-15)
        assert np.allclose(O.tau_of(t), O.toeplitz_S(2.0, n[i]), rtol=0, atol=1e-15)
        Bi = O.tridiag_B(2.0, n[i])
        lap = 2 * np.eye(n[i]) - np.eye(n[i], k=1) - np.eye(n[i], k=-1)
        assert np.allclose(Bi, np.eye(n[i]) - lap / 12.0, rtol=0, atol=1e-15)
    N = int(np.prod(n))
    c = 1.5
    e = np.full(N, c)
    assert np.allclose(O.dense_A(p, e), O.dense_M(p, c), rtol=0, atol=1e-12)
    b = W.random_vector(N, 5)
    res = O.gmres(lambda v: O.apply_A(p, e, v), b, np.zeros_like(b), 1e-12, 20,
                  lambda v: O.apply_Minv(p, c, v))
    assert res.iters == 1
    x = np.linalg.solve(O.dense_A(p, e), b)
    assert np.linalg.norm(res.x - x) <= 1e-12 * np.linalg.norm(x)
