"""Pins for the oracle's FCD weights, the discrete Riesz operator and the
quasi-compact operator (§2), and for the closed-form Riesz derivative the
manufactured sources use (§1)."""

import math

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

ALPHAS = [1.1, 1.3, 1.5, 1.7, 1.9]


@pytest.mark.parametrize("alpha", ALPHAS)
def test_recurrence_matches_gamma_form(alpha):
    # §2: closed Gamma form of s_j vs the recurrence below Eq. (eq0).
    s = O.fcd_weights(alpha, 60)
    g = O.fcd_weights_gamma(alpha, 60)
    assert np.allclose(s, g, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("alpha", ALPHAS)
def test_weight_signs_and_zero_sum(alpha):
    # Eq. (As1): s_0 > 0, s_k < 0, s_0 + 2 sum s_k = 0 (partial sums decrease to 0+).
    s = O.fcd_weights(alpha, 20001)
    assert s[0] > 0 and np.all(s[1:] < 0)
    partial = s[0] + 2 * np.cumsum(s[1:])
    assert np.all(partial > 0)
    assert np.all(np.diff(partial) < 0)
    # tail of sum_k s_k behaves like k^{-alpha}: partial sum at K is O(K^{-alpha})
    K = 20000
    assert partial[-1] < 5.0 * K ** (-alpha)


def test_alpha_two_is_classical_second_difference():
    # alpha -> 2: s = (2, -1, 0, ...), i.e. S = -tridiag(1,-2,1) (textbook 3-point Laplacian).
    s = O.fcd_weights(2.0, 8)
    assert np.allclose(s, [2.0, -1.0, 0, 0, 0, 0, 0, 0], atol=1e-15)


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_generating_function(alpha):
    # FCD symbol: s_0 + 2 sum_k s_k cos(k theta) = |2 sin(theta/2)|^alpha.
    K = 200000
    s = O.fcd_weights(alpha, K)
    k = np.arange(1, K)
    for theta in [0.3, 1.0, 2.0, 3.0]:
        val = s[0] + 2 * np.sum(s[1:] * np.cos(k * theta))
        assert abs(val - abs(2 * math.sin(theta / 2)) ** alpha) < 2e-6


def test_riesz_closed_form_alpha2_is_second_derivative():
    # sigma_2 = 1/2, left and right RL derivatives of order 2 are both d^2/dx^2.
    x = np.linspace(0.05, 0.95, 19)
    R = W.riesz_bump(2, 2, 2.0)(x)
    # u = x^2 (1-x)^2 = x^2 - 2x^3 + x^4, u'' = 2 - 12 x + 12 x^2
    assert np.allclose(R, 2 - 12 * x + 12 * x ** 2, rtol=1e-13, atol=1e-13)


def test_riesz_closed_form_vs_quadrature():
    # §1 definition of the RL derivatives evaluated by quadrature with the
    # algebraic weight, second derivative by central differences.
    integrate = pytest.importorskip("scipy.integrate")
    alpha = 1.5
    u = W.bump(4, 4)

    def I_left(x):
        return integrate.quad(u, 0.0, x, weight="alg", wvar=(0.0, 1.0 - alpha), epsabs=1e-14, epsrel=1e-13)[0]

    def I_right(x):
        return integrate.quad(u, x, 1.0, weight="alg", wvar=(1.0 - alpha, 0.0), epsabs=1e-14, epsrel=1e-13)[0]

    sigma = -1.0 / (2 * math.cos(alpha * math.pi / 2))
    dlt = 2e-3
    R = W.riesz_bump(4, 4, alpha)
    for x in [0.2, 0.45, 0.7]:
        d2 = 0.0
        for I in (I_left, I_right):
            d2 += (I(x + dlt) - 2 * I(x) + I(x - dlt)) / dlt ** 2
        num = sigma * d2 / math.gamma(2 - alpha)
        assert abs(num - R(x)) < 1e-5 * max(1.0, abs(R(x)))


@pytest.mark.parametrize("alpha", [1.3, 1.5, 1.9])
def test_fcd_second_order_and_quasicompact_fourth_order(alpha):
    # delta^alpha u = d^alpha u + O(h^2); delta^alpha u = 𝓗_alpha d^alpha u + O(h^4)
    # (§2 and Appendix B), on the interior part of (0,1) away from the boundary layer.
    u = W.bump(4, 4)
    R = W.riesz_bump(4, 4, alpha)
    e2, e4 = [], []
    for Np1 in (32, 64, 128):
        h = 1.0 / Np1
        x = np.arange(Np1 + 1) * h
        d = O.fcd_apply_line(alpha, h, u(x))
        Rx = R(x)
        xi = x[1:-1]
        m = (xi >= 0.25) & (xi <= 0.75)
        e2.append(np.abs(d - Rx[1:-1])[m].max())
        Hex = (alpha / 24) * Rx[:-2] + (1 - alpha / 12) * Rx[1:-1] + (alpha / 24) * Rx[2:]
        e4.append(np.abs(d - Hex)[m].max())
    r2 = [e2[i] / e2[i + 1] for i in range(2)]
    r4 = [e4[i] / e4[i + 1] for i in range(2)]
    assert all(3.6 < r < 4.4 for r in r2), r2
    assert all(14.0 < r < 18.0 for r in r4), r4


def test_fcd_line_matches_toeplitz_matrix():
    # delta^alpha on a function vanishing on the boundary is -h^{-alpha} S_alpha (Eq. (eq0)).
    alpha, n = 1.7, 9
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(3)
    u = np.zeros(n + 2)
    u[1:-1] = rng.standard_normal(n)
    d = O.fcd_apply_line(alpha, h, u)
    assert np.allclose(d, -O.toeplitz_S(alpha, n) @ u[1:-1] / h ** alpha, rtol=1e-13, atol=1e-12)
