"""The autotuner's measured choices: the route of each dimension (the GEMM-or-FFT decision of the
line passes: dense O(n) mode products against FFT or chirp-z transforms), timed on the device at
setup, kept per device and shape, and persisted to the autotune file so a later process reuses it.

The library reads TAU_TUNE_CACHE once per process, so each measurement here runs in a fresh
Python process with its own cache file."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
from paper_2404_10221_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np, torch
from paper_2404_10221_gb300 import tau, workloads as W
wl = W.c2_2d(n=1000, M=2)
wl.prob.n = [1000, 100]
wl = W.manufactured("tune", wl.prob, wl.e.terms, 2, 2, 1.0)
p = tau.Problem(wl)
st = p.stats()
p.solve()
u = p.solution().cpu().numpy()
p.close()
np.save({out!r}, u)
print(json.dumps({{"route": list(st.route[:2]), "source": list(st.route_source[:2]),
                  "ms": list(st.route_ms[:2]), "alt": list(st.route_alt_ms[:2])}}))
"""


def _child(cache, out):
    env = dict(os.environ, TAU_TUNE_CACHE=str(cache), TAU_AUTOTUNE="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, out=str(out))], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_route_choice_is_measured_recorded_and_reused(tmp_path):
    from paper_2404_10221_gb300 import tau
    cache = tmp_path / "autotune.txt"
    a = _child(cache, tmp_path / "a.npy")
    # both dimensions have two candidates (n = 1000 and n = 100: chirp-z or dense); both measured
    assert a["source"] == [1, 1], a
    for i in range(2):
        assert 0.0 < a["ms"][i] <= a["alt"][i], a
        assert a["route"][i] in (tau.TAU_ROUTE_CHIRP, tau.TAU_ROUTE_DENSE)
    # n = 1000: the dense route's O(n) sums per element lose to the O(log n) chirp-z transforms
    assert a["route"][0] == tau.TAU_ROUTE_CHIRP, a
    text = cache.read_text()
    assert text.startswith("# tau_rsfde autotune")
    assert text.count("route|") == 2 and "lpb|" in text
    # a second process reads the record instead of measuring again, and takes the same routes
    b = _child(cache, tmp_path / "b.npy")
    assert b["source"] == [2, 2], b
    assert b["route"] == a["route"] and b["ms"] == pytest.approx(a["ms"], rel=1e-5)
    ua, ub = np.load(tmp_path / "a.npy"), np.load(tmp_path / "b.npy")
    assert np.array_equal(ua, ub)
    # the tuned solve against the oracle (plain FP64 bar)
    wl = W.c2_2d(n=1000, M=2)
    wl.prob.n = [1000, 100]
    wl = W.manufactured("tune", wl.prob, wl.e.terms, 2, 2, 1.0)
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run()
    assert np.linalg.norm(ua - ref.u) / np.linalg.norm(ref.u) <= 1e-10


def test_route_record_of_another_build_is_ignored(tmp_path):
    cache = tmp_path / "autotune.txt"
    cache.write_text("# tau_rsfde autotune some other build\nroute|x|0|0|1000|1|100\t2 1 2\n")
    a = _child(cache, tmp_path / "a.npy")
    assert a["source"] == [1, 1], a
    assert "some other build" not in cache.read_text()
