"""The allocation-free matvec entry point against the regular one and against the oracle.

tau_apply_A_noalloc serves callers that cannot allocate device memory: a host application whose
pool owns the device, a plugin that must keep the device's memory footprint unchanged, or a
latency-critical loop that cannot afford a cudaMalloc (which may synchronise the device).  Its
scratch lives in one static device array shared by all calls.  This file is collected last so that
a run stopping at the first failure has already run every other test; it also passes on its own
in a fresh process.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_RTOL = 1e-12   # the operator tolerance of the parity tests


def _case(n, seed):
    import oracle as O
    from paper_2404_10221_gb300 import tau, workloads as W
    d = len(n)
    base = {1: W.c1_1d, 2: W.c2_2d, 3: W.c3_3d}[d](n=n[0], M=5)
    base.prob.n = list(n)
    base.prob.max_iter = 2
    wl = W.manufactured(f"na_{d}d", base.prob, base.e.terms, 2, 2, 1.0)
    t = wl.field_tables()
    m = 2
    e = O.eval_field_interior(wl.prob, t["e_tc"][m], t["e_sp"])
    x = W.random_vector(wl.prob.n_tot, seed)
    return tau, wl, m, e, x


def _regular(tau, wl, m, x):
    p = tau.Problem(wl)
    y = torch.empty(wl.prob.n_tot, dtype=torch.float64, device="cuda")
    tau.tau_apply_A(p.handle, m, torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    out = y.cpu().numpy()
    p.close()
    return out


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_apply_A_noalloc_matches_apply_A_two_calls_in_a_row():
    results = []
    # two calls in a row on different problems: the second must not see the first's scratch
    for n, seed in [((63, 31), 5), ((15, 7, 31), 6)]:
        tau, wl, m, e, x = _case(n, seed)
        desc = tau.make_desc(wl.prob)
        y = torch.full((wl.prob.n_tot,), float("nan"), dtype=torch.float64, device="cuda")
        tau.tau_apply_A_noalloc(desc, torch.from_numpy(e).cuda(), torch.from_numpy(x).cuda(), y)
        torch.cuda.synchronize()
        results.append((tau, wl, m, x, y.cpu().numpy()))
    for tau, wl, m, x, got in results:
        ref = _regular(tau, wl, m, x)
        assert _rel(got, ref) <= OP_RTOL


# Shapes that take both of the entry point's routes: n + 1 a power of two (FFT) and any other n
# (dense sums), in 1-D, 2-D and 3-D, up to its limits (n_i = 4095, 262,144 grid points).
SHAPES = [(4095,), (1000,), (100, 37), (1000, 255), (63, 63, 63), (31, 5, 17)]


@pytest.mark.parametrize("n", SHAPES)
def test_apply_A_noalloc_matches_oracle_on_a_side_stream(n):
    import oracle as O
    tau, wl, m, e, x = _case(n, 7)
    desc = tau.make_desc(wl.prob)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ed = torch.from_numpy(e).cuda()
        xd = torch.from_numpy(x).cuda()
        y = torch.full((wl.prob.n_tot,), float("nan"), dtype=torch.float64, device="cuda")
        tau.tau_apply_A_noalloc(desc, ed, xd, y, stream=side.cuda_stream)
    side.synchronize()
    got = y.cpu().numpy()
    ref = O.apply_A(wl.prob, e, x)
    assert _rel(got, ref) <= OP_RTOL, "vs oracle"
    assert _rel(got, _regular(tau, wl, m, x)) <= OP_RTOL, "vs tau_apply_A"


def test_apply_A_noalloc_leaves_free_device_memory_unchanged():
    """After a first call (which looks up the scratch address), further calls allocate nothing."""
    tau, wl, m, e, x = _case((127, 63), 8)
    desc = tau.make_desc(wl.prob)
    ed = torch.from_numpy(e).cuda()
    xd = torch.from_numpy(x).cuda()
    y = torch.empty(wl.prob.n_tot, dtype=torch.float64, device="cuda")
    tau.tau_apply_A_noalloc(desc, ed, xd, y)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        tau.tau_apply_A_noalloc(desc, ed, xd, y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_apply_A_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2404_10221_gb300 import tau, workloads as W
    wl = W.c2_2d(n=1023, M=2)
    desc = tau.make_desc(wl.prob)
    e = torch.ones(8, dtype=torch.float64, device="cuda")
    with pytest.raises(tau.TauError) as ei:
        tau.tau_apply_A_noalloc(desc, e, e, e)
    assert ei.value.status == tau.TAU_EINVAL
    assert "static scratch limit" in str(ei.value)
