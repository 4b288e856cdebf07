"""The error model behind the host-side precision policy (tau_choose_precision), checked on the CPU.

The policy takes the mixed form when 2^-23 max_i eta_i 2 s_0(alpha_i) / e_min <= 0.05.  Its model:
on the smooth vectors of a converging solve, the FP32 rounding error of A x is about
eps_32 eta ||s||_1 |x|, while the Toeplitz sum cancels (the fractional weights sum to zero,
Eq. (As1)) and leaves a result of order e |x|.  Here A x of the 1-D workload, B(e∘x) + eta T x
(Eq. (tls)), is evaluated in FP32 (single-precision FFTs of a power-of-two circulant embedding of
T) and in FP64 on the manufactured solution's profile x^2 (1-x)^2, for n from 1023 to 65535 (eta
from 5e3 to 3e6).  The FP32 relative error must track the policy value: the ratio between the two
stays within [0.05, 1] at every n, and the error stays below 1e-2 wherever the library picks the
mixed form.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

sf = pytest.importorskip("scipy.fft")


@pytest.fixture(scope="module")
def tau():
    from paper_2404_10221_gb300 import build, tau
    build.build()
    tau.lib()
    return tau


def toeplitz_product(s, x, dtype):
    """T x for the symmetric Toeplitz T with first column s, through a circulant of length 2^p >= 2n,
    every operation in `dtype`."""
    n = len(x)
    L = 1 << int(math.ceil(math.log2(2 * n)))
    c = np.zeros(L, dtype)
    c[:n] = s
    c[L - n + 1:] = s[1:][::-1]
    xp = np.zeros(L, dtype)
    xp[:n] = x
    y = sf.irfft(sf.rfft(c) * sf.rfft(xp), n=L)
    assert y.dtype == dtype
    return y[:n]


def apply_A_1d(alpha, eta, e, x, dtype):
    ex = (e * x).astype(dtype)
    b = ex * dtype(1 - alpha / 12)
    b[1:] += ex[:-1] * dtype(alpha / 24)
    b[:-1] += ex[1:] * dtype(alpha / 24)
    s = O.fcd_weights(alpha, len(x)).astype(dtype)
    return b + dtype(eta) * toeplitz_product(s, x.astype(dtype), dtype)


def test_fp32_matvec_error_tracks_the_policy_value(tau):
    for n in (1023, 5000, 20000, 65535):
        wl = W.c1_1d(n=n, M=3)
        pr = wl.prob
        a = pr.alpha[0]
        h = (pr.R[0] - pr.L[0]) / (n + 1)
        eta = pr.kappa[0] * (pr.T / pr.M) / (2.0 * h ** a)
        xs = np.linspace(pr.L[0] + h, pr.R[0] - h, n)
        x = xs ** 2 * (1 - xs) ** 2
        e = 1.0 + 0.5 * np.sin(np.pi * xs)           # e of the workload at t = 0 (e_min = 1)
        y64 = apply_A_1d(a, eta, e, x, np.float64)
        y32 = apply_A_1d(a, eta, e, x, np.float32).astype(np.float64)
        rel = np.linalg.norm(y32 - y64) / np.linalg.norm(y64)
        s0 = O.fcd_weights(a, 1)[0]
        value = 2.0 ** -23 * eta * 2.0 * s0 / 1.0
        assert 0.05 <= rel / value <= 1.0, (n, rel, value)
        choice = tau.tau_choose_precision(tau.make_desc(pr, e_bounds=(1.0, 1.5)))
        if choice == tau.TAU_MIXED:
            assert rel <= 1e-2, (n, rel)
        else:
            assert choice == tau.TAU_DF64 and rel > 1e-2, (n, rel)
