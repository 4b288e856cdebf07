"""Pins for the oracle's tau-algebra pieces (§3): H(T), tau(T), the sine
matrix, the eigenvalues q (Eq. (q)), beta (Lemma Heig), Lemma tauT."""

import math

import numpy as np
import pytest

import oracle as O

SIZES = [1, 2, 3, 4, 5, 8, 17, 32]


def test_hankel_structure_brute_force():
    # H(T) printed in Eq. (tau): first row (t_2..t_{N-1}, 0, 0), constant along
    # anti-diagonals, persymmetric (symmetric about the anti-diagonal).
    n = 7
    t = np.arange(10.0, 10.0 + n)          # distinct entries t_0..t_6
    H = O.hankel_H(t)
    assert np.allclose(H[0], list(t[2:n]) + [0.0, 0.0])
    assert np.allclose(H[-1], [0.0, 0.0] + list(t[2:n][::-1]))
    for i in range(n):
        for j in range(n):
            if i + 1 < n and j - 1 >= 0:
                assert H[i, j] == H[i + 1, j - 1]
            assert H[i, j] == H[n - 1 - j, n - 1 - i]
    assert np.allclose(H, H.T)


@pytest.mark.parametrize("n", SIZES)
def test_sine_matrix_orthogonal_symmetric(n):
    S = O.sine_matrix(n)
    assert np.allclose(S, S.T, atol=1e-15)
    assert np.allclose(S @ S, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("alpha", [1.1, 1.5, 1.9])
@pytest.mark.parametrize("n", SIZES)
def test_tau_diagonalised_by_sine(alpha, n):
    # Eq. (diag): tau(T) = S Q S with Q = diag(q_i) of Eq. (q).
    t = O.fcd_weights(alpha, n)
    S = O.sine_matrix(n)
    D = S @ O.tau_of(t) @ S
    q = O.tau_eigs_q(t)
    assert np.allclose(np.diag(D), q, rtol=1e-12, atol=1e-13)
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-13 * max(1.0, np.abs(q).max())
    # independent route: eigenvalues by a symmetric eigensolver
    assert np.allclose(np.sort(np.linalg.eigvalsh(O.tau_of(t))), np.sort(q), rtol=1e-12, atol=1e-13)


def test_tridiagonal_toeplitz_is_tau():
    # §3: a tridiagonal Toeplitz matrix is already a tau matrix: H(T) = 0.
    t = np.array([2.0, -1.0, 0.0, 0.0, 0.0, 0.0])
    assert np.allclose(O.hankel_H(t), 0.0)
    assert np.allclose(O.tau_of(t), O.toeplitz_S(2.0, 6))


@pytest.mark.parametrize("alpha", [1.1, 1.5, 1.9])
@pytest.mark.parametrize("n", [3, 8, 31])
def test_beta_eigs_lemma_heig(alpha, n):
    B = O.tridiag_B(alpha, n)
    S = O.sine_matrix(n)
    beta = O.beta_eigs(alpha, n)
    assert np.allclose(S @ B @ S, np.diag(beta), atol=1e-14)
    assert np.all(beta > 1 - alpha / 6) and np.all(beta < 1)
    assert np.all(beta > 2.0 / 3.0)
    ev = np.linalg.eigvalsh(B)
    cond_half = math.sqrt(ev.max() / ev.min())
    assert cond_half <= math.sqrt(6) / 2


@pytest.mark.parametrize("alpha", [1.1, 1.5, 1.9])
@pytest.mark.parametrize("n", [4, 16, 40])
def test_lemma_tauT(alpha, n):
    # tau(T) SPD and ||tau^{-1/2} H tau^{-1/2}||_2 < 1/2 (Lemma tauT).
    t = O.fcd_weights(alpha, n)
    tau = O.tau_of(t)
    w, Q = np.linalg.eigh(tau)
    assert w.min() > 0
    th = (Q * w ** -0.5) @ Q.T
    nrm = np.linalg.norm(th @ O.hankel_H(t) @ th, 2)
    assert nrm < 0.5


def test_toeplitz_S_spd():
    for alpha in [1.1, 1.5, 1.9]:
        assert np.linalg.eigvalsh(O.toeplitz_S(alpha, 25)).min() > 0


@pytest.mark.parametrize("n", [1, 2, 7, 31, 100])
def test_row_helpers_match_the_whole_matrices(n):
    # sine_rows, toeplitz_rows and tau_eigs_q_at (the sampled forms used at sizes where the whole
    # matrices do not fit) agree with sine_matrix, toeplitz_S and tau_eigs_q row by row.
    ks1 = np.arange(1, n + 1)
    assert np.array_equal(O.sine_rows(n, ks1), O.sine_matrix(n))
    assert np.array_equal(O.toeplitz_rows(1.37, n, ks1 - 1), O.toeplitz_S(1.37, n))
    t = O.fcd_weights(1.63, n)
    assert np.allclose(O.tau_eigs_q_at(t, ks1), O.tau_eigs_q(t), rtol=1e-14, atol=1e-14)


def test_row_helpers_closed_forms_at_large_n():
    # Large-n special cases fixed by the mathematics: row k of S at the middle mode of an odd
    # N + 1 = 2m alternates 0, +-sqrt(2/(N+1)) ... ; q of the tridiagonal t = (2, -1) is
    # 2 - 2 cos(pi k/(N+1)) (the second-difference matrix, alpha = 2).
    n = 65535
    row = O.sine_rows(n, np.array([(n + 1) // 2]))[0]          # k = (N+1)/2: sin(pi j / 2)
    j = np.arange(1, n + 1)
    ref = math.sqrt(2.0 / (n + 1)) * np.where(j % 2 == 1, np.where(j % 4 == 1, 1.0, -1.0), 0.0)
    assert np.allclose(row, ref, atol=1e-15)
    t = np.zeros(n)
    t[0], t[1] = 2.0, -1.0
    ks = np.array([1, 17, 40000, n])
    assert np.allclose(O.tau_eigs_q_at(t, ks), 2.0 - 2.0 * np.cos(np.pi * ks / (n + 1)), atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 100, 127, 255, 256])
def test_sine_matrix_row_mirror(n):
    """The rows of the DST-I matrix satisfy S[n-1-k][j] = (-1)^j S[k][j] (0-based j, k), so the
    product splits into even-j and odd-j sums E, O over the first ceil(n/2) rows:
    y[k] = E_k + O_k and y[n-1-k] = E_k - O_k (the middle row of an odd n is its own mirror, where
    O vanishes).  The tensor-core DST multiplies only those rows; this pins the identity on the
    oracle's sine matrix and the reconstruction on a random vector."""
    S = O.sine_matrix(n)
    sign = (-1.0) ** np.arange(n)
    assert np.allclose(S[::-1, :], S * sign[None, :], atol=1e-15, rtol=0)
    h = (n + 1) // 2
    x = np.random.default_rng(n).standard_normal(n)
    E = S[:h, 0::2] @ x[0::2]
    Od = S[:h, 1::2] @ x[1::2]
    y = np.empty(n)
    y[:h] = E + Od
    km = n - 1 - np.arange(h)
    mirror = km > np.arange(h)
    y[km[mirror]] = (E - Od)[mirror]
    if n % 2:
        assert abs(Od[h - 1]) <= 1e-14 * np.abs(x).sum()
    assert np.allclose(y, S @ x, atol=1e-13, rtol=0)
