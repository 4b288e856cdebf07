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
