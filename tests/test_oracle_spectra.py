"""Spectral diagnostics of §3 (Figs. 1–3, Theorem GMRES), oracle tier: the preconditioned spectrum
clusters while Ã's spreads with N, and the numerical range of the two-sided matrix stays inside the
angle Theorem GMRES allows.  tests/golden/spectra_examples.txt is the regression record
(written by tests/golden/make_spectra.py from the oracle)."""

import os

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "spectra_examples.txt")
COLS = ["spread_A", "spread_PA", "re_PA_min", "re_PA_max", "v", "r", "sin_theta"]


def _summary(d, alpha, n):
    wl = W.paper_example(d, list(alpha), n, 64)
    p, t = wl.prob, wl.field_tables()
    ebar, ehat, echeck = O.ebar_from_tables(p, t["e_tc"], t["e_sp"])
    e = O.eval_field_interior(p, t["e_tc"][0], t["e_sp"])
    return O.spectral_summary(p, e, ebar), O.theorem_c(ehat, echeck)


def test_numerical_range_bounds_exact_cases():
    # SPD: W(A) = [lambda_min, lambda_max]
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    A = Q @ np.diag([0.5, 1.0, 2.0, 2.5, 3.0]) @ Q.T
    v, r = O.numerical_range_bounds(A)
    assert abs(v - 0.5) < 1e-12 and abs(r - 3.0) < 1e-12
    # Jordan block [[1, 2], [0, 1]]: W is the disc of radius 1 about 1 (touches 0)
    v, r = O.numerical_range_bounds(np.array([[1.0, 2.0], [0.0, 1.0]]))
    assert abs(v) < 1e-12 and abs(r - 2.0) < 1e-12


def test_preconditioned_spectrum_clusters():
    # Figs. 1–2: Ã's eigenvalues spread like N^alpha, P^{-1} Ã's stay clustered near 1
    sp = [_summary(1, (1.5,), n)[0] for n in (7, 15, 31)]
    for a, b in zip(sp, sp[1:]):
        assert b["spread_A"] > 2.0 * a["spread_A"]
    for s in sp + [_summary(2, (1.3, 1.5), 7)[0]]:
        assert s["spread_PA"] < 1.5
        assert 0.5 < s["re_PA_min"] <= s["re_PA_max"] < 1.1


@pytest.mark.parametrize("d,alpha,n", [(1, (1.5,), 15), (1, (1.9,), 31), (2, (1.3, 1.5), 7)])
def test_numerical_range_within_theorem_bound(d, alpha, n):
    s, c = _summary(d, alpha, n)
    assert 0 < s["v"] <= s["r"]          # 0 is not in W(Ă)
    assert s["sin_theta"] <= c


def test_spectra_golden_record():
    with open(GOLDEN) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for r in rows:
        d, alpha, n = int(r[0]), tuple(float(x) for x in r[1].split(",")), int(r[2])
        s, c = _summary(d, alpha, n)
        want = [float(x) for x in r[3:3 + len(COLS)]]
        got = [s[k] for k in COLS]
        assert np.allclose(got, want, rtol=1e-8, atol=1e-12), (r[:3], got, want)
        assert abs(c - float(r[-1])) <= 1e-12
