"""Fields given to the library as device arrays (tau_set_fields_device): any positive e(x,t) and any
f(x,t) of the problem statement (§1, Eq. (RSFDE)), sampled at t_{m+1/2} on the grid, not only the
separable expansions of tau_set_fields.  The library reads e of step m and forms
F = (⊗ 𝓗_{alpha_l}) f (Eq. (2.2), Appendix A) from f on the padded grid on the device; the oracle
takes the same arrays.  Bars: FP64 solves 1e-10 relative with iterations ±1; the mixed form 1e-8."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
from paper_2404_10221_gb300 import workloads as W


def _tau():
    from paper_2404_10221_gb300 import tau
    return tau


def _prob(n, M, alpha=(1.4, 1.8, 1.6), kappa=(1.0, 0.5, 0.8)):
    d = len(n)
    return W.Problem(d=d, n=list(n), alpha=list(alpha[:d]), kappa=list(kappa[:d]), T=1.0, M=M, tol=1e-12)


def _solve(prob, fields, precision=0, steps=None):
    tau = _tau()
    h = tau.tau_create(tau.make_desc(prob, precision=precision))
    dev = {k: (None if v is None else torch.from_numpy(np.ascontiguousarray(v)).cuda())
           for k, v in fields.items()}
    try:
        tau.tau_set_fields_device(h, dev["e_dense"], dev["f_dense"], dev["psi_dense"])
        tau.tau_setup(h)
        tau.tau_step(h, prob.M if steps is None else steps)
        tau.tau_sync(h)
        u = torch.empty(prob.n_tot, dtype=torch.float64, device="cuda")
        tau.tau_get_solution(h, u, True)
        its = tau.tau_get_iters(h, prob.M)
        torch.cuda.synchronize()
        return u.cpu().numpy(), its
    finally:
        tau.tau_destroy(h)


def _oracle(prob, fields, steps=None):
    ref = O.OracleSolver(prob, fields)
    ref.run(steps)
    return ref


@pytest.mark.parametrize("n,M", [((63, 47), 4), ((15, 9, 11), 3), ((127,), 5)])
def test_non_separable_fields_match_oracle(n, M):
    prob = _prob(n, M)
    fields = W.dense_fields(prob)
    u, its = _solve(prob, fields)
    ref = _oracle(prob, fields)
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= 1e-10, rel
    assert np.all(np.abs(its[:M] - np.array(ref.iters)) <= 1), (its, ref.iters)


def test_time_independent_e_and_zero_source():
    """e_step = 0 (one slab for every step) and f = NULL (F = 0)."""
    prob = _prob((31, 33), 3)
    fields = W.dense_fields(prob, time_dependent_e=False, with_f=False)
    u, its = _solve(prob, fields)
    ref = _oracle(prob, fields)
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-10


def test_mixed_form_with_device_fields():
    tau = _tau()
    prob = _prob((63, 63), 3)
    fields = W.dense_fields(prob)
    u, _ = _solve(prob, fields, precision=tau.TAU_MIXED)
    ref = _oracle(prob, fields)
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-8


def test_separable_fields_as_tables_or_as_arrays_agree():
    """The same separable workload through both field forms lands on the same solution (the only
    difference is the rounding order of F)."""
    tau = _tau()
    wl = W.c2_2d(n=63, M=3)
    t = wl.field_tables()
    prob = wl.prob
    e = np.stack([O.eval_field_interior(prob, t["e_tc"][m], t["e_sp"]) for m in range(prob.M)])
    f = np.stack([O.eval_field(prob, t["f_tc"][m], t["f_sp"]).reshape(-1) for m in range(prob.M)])
    psi = O.eval_field_interior(prob, t["psi_tc"][0], t["psi_sp"])
    u_dev, _ = _solve(prob, {"e_dense": e, "f_dense": f, "psi_dense": psi})
    p = tau.Problem(wl)
    p.solve()
    u_tab = p.solution().cpu().numpy()
    p.close()
    assert np.linalg.norm(u_dev - u_tab) / np.linalg.norm(u_tab) <= 1e-12


def test_bad_strides_rejected():
    tau = _tau()
    prob = _prob((15, 7), 2)
    h = tau.tau_create(tau.make_desc(prob))
    try:
        e = torch.ones(prob.M, prob.n_tot, dtype=torch.float64, device="cuda")
        with pytest.raises(tau.TauError) as ei:
            tau.tau_set_fields_device(h, e, e_step=prob.n_tot + 1)
        assert ei.value.status == tau.TAU_EINVAL
        f = torch.ones(17 * 9, dtype=torch.float64, device="cuda")
        with pytest.raises(tau.TauError) as ei:
            tau.tau_set_fields_device(h, e, f, f_step=5)
        assert ei.value.status == tau.TAU_EINVAL
        with pytest.raises(tau.TauError) as ei:
            tau.tau_setup(h)
        assert ei.value.status == tau.TAU_ESTATE
    finally:
        tau.tau_destroy(h)
