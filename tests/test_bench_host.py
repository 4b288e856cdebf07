"""Host-side pieces of bench.py that need no GPU: the DRAM traffic of the dominant kernel is
reported only for the kernel sources it was captured on, and the algorithmic FLOP count of one
preconditioned matvec is the figure the roofline uses."""

import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_is_null_once_a_captured_source_changes(tmp_path, monkeypatch):
    # a copy of the tree where one hashed file differs by one byte from the sources as they stand:
    # no traffic figure
    rel = next(iter(bench.TRAFFIC_CAPTURE["sha256"]))
    fake_root = tmp_path / "repo"
    for r in bench.TRAFFIC_CAPTURE["sha256"]:
        dst = fake_root / r
        dst.parent.mkdir(parents=True, exist_ok=True)
        data = open(os.path.join(ROOT, r), "rb").read()
        dst.write_bytes(data + (b" " if r == rel else b""))
    monkeypatch.setattr(bench, "__file__", str(fake_root / "bench.py"))
    assert bench.captured_traffic() is None


def test_matvec_flop_count():
    """4.87e8 algorithmic FLOPs per preconditioned matvec on 1023^2 (the roofline's unit); the count
    grows as n^2 log n."""
    f1, f2 = bench.pass_flops_2d(1023), bench.pass_flops_2d(2047)
    assert abs(f1 - 4.87e8) / 4.87e8 < 0.01
    assert 4.0 < f2 / f1 < 4.0 * math.log2(4096) / math.log2(2048) * 1.05
