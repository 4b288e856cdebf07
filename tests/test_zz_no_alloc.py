"""The allocation-free matvec entry point against the regular one.

tau_apply_A_noalloc serves callers that cannot allocate device memory (a host application's
pool owns the device, a plugin must keep the memory footprint unchanged, or a latency-critical
loop cannot afford a possibly synchronising cudaMalloc).  Its scratch lives in one static device
array shared by all calls.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_RTOL = 1e-12   # the operator tolerance of the parity tests


def _case(d, n, seed):
    import oracle as O
    from paper_2404_10221_gb300 import tau, workloads as W
    if d == 2:
        base = W.c2_2d(n=n[0], M=5)
    else:
        base = W.c3_3d(n=n[0], M=5)
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


def test_apply_A_noalloc_matches_apply_A_two_calls_in_a_row():
    results = []
    # two calls in a row on different problems: the second must not see the first's scratch
    for d, n, seed in [(2, (63, 31), 5), (3, (15, 7, 31), 6)]:
        tau, wl, m, e, x = _case(d, n, seed)
        desc = tau.make_desc(wl.prob)
        y = torch.full((wl.prob.n_tot,), float("nan"), dtype=torch.float64, device="cuda")
        tau.tau_apply_A_noalloc(desc, torch.from_numpy(e).cuda(), torch.from_numpy(x).cuda(), y)
        torch.cuda.synchronize()
        results.append((tau, wl, m, x, y.cpu().numpy()))
    for tau, wl, m, x, got in results:
        ref = _regular(tau, wl, m, x)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= OP_RTOL, rel


def test_apply_A_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2404_10221_gb300 import tau, workloads as W
    wl = W.c2_2d(n=1023, M=2)
    desc = tau.make_desc(wl.prob)
    e = torch.ones(8, dtype=torch.float64, device="cuda")
    with pytest.raises(tau.TauError) as ei:
        tau.tau_apply_A_noalloc(desc, e, e, e)
    assert ei.value.status == tau.TAU_EINVAL
    assert "static scratch limit" in str(ei.value)
