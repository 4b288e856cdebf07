"""Long-line route (d = 1): the chirp route's convolutions as four-step FFTs over global memory.

Against the FP64 oracle where its dense matrices fit (n <= 5000): operators to a relative 2-norm
of 1e-12 (M^{-1} with the conditioning allowance), solves to 1e-10 with iteration counts within
+-1.  At n up to 65535 (the served 1-D range) on sampled outputs the oracle computes one by one
(rows of S, of the Toeplitz factor, q at single modes), and through properties: S S x = x,
mode-wise mu_k (S M^{-1} x)_k = (S x)_k, and the preconditioned residual of a whole step.
"""

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_RTOL = 1e-12
SOLVE_RTOL = 1e-10
EPS = np.finfo(np.float64).eps


def _tau():
    from paper_2404_10221_gb300 import tau
    return tau


def _wl(n, M=3, x0_mode=0, max_iter=100):
    wl = W.c1_1d(n=n, M=M)
    wl.prob.x0_mode = x0_mode
    wl.prob.max_iter = max_iter
    return wl


def _long():
    tau = _tau()
    return (tau.TAU_ROUTE_LONG, 0, 0)


def _cuda(x, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).to("cuda")


def _host(y):
    return y.detach().cpu().numpy().astype(np.float64)


def _cmp(got, ref, rtol=OP_RTOL):
    got = _host(got) if hasattr(got, "detach") else got
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= rtol, f"rel 2-norm {rel:.3e}"
    assert np.abs(got - ref).max() <= 10 * rtol * np.abs(ref).max()


def _kappa_q(prob, ebar):
    eta = O.etas(prob)
    l1 = 2 * O.fcd_weights(prob.alpha[0], prob.n[0])[0]
    return eta[0] * l1 / O.mu_tensor(prob, ebar).min()


FORCED = [1, 2, 3, 5, 40, 127, 1000, 4095]


@pytest.mark.parametrize("n", FORCED + [4096, 5000])
def test_operators_vs_oracle(n):
    tau = _tau()
    wl = _wl(n, max_iter=4)
    pr = wl.prob
    p = tau.Problem(wl, route=_long())
    assert p.stats().route[0] == tau.TAU_ROUTE_LONG
    x = W.random_vector(n, 51)
    xd = _cuda(x)
    y = torch.empty_like(xd)
    tau.tau_dst(p.handle, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.sine_matrix(n) @ x)
    tau.tau_toeplitz_mode(p.handle, 0, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.toeplitz_S(pr.alpha[0], n) @ x)
    t = wl.field_tables()
    ebar = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])[0]
    e = O.eval_field_interior(pr, t["e_tc"][1], t["e_sp"])
    tau.tau_apply_A(p.handle, 1, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_A(pr, e, x))
    tau.tau_rhs(p.handle, 1, xd, y)
    torch.cuda.synchronize()
    F = O.rhs_F(pr, O.eval_field(pr, t["f_tc"][1], t["f_sp"]))
    _cmp(y, O.rhs_b(pr, e, x, F))
    tau.tau_apply_Minv(p.handle, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_Minv(pr, ebar, x), OP_RTOL + 4 * EPS * _kappa_q(pr, ebar))
    tau.tau_apply_MinvA(p.handle, 1, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_Minv(pr, ebar, O.apply_A(pr, e, x)), OP_RTOL + 4 * EPS * _kappa_q(pr, ebar))
    p.close()


@pytest.mark.parametrize("n", [50000, 65535])
def test_operators_sampled_at_served_sizes(n):
    """The top of the served 1-D range: sampled rows against the oracle, and the τ solve through
    S S x = x and mu_k (S M^{-1} x)_k = (S x)_k at sampled modes."""
    tau = _tau()
    wl = _wl(n, max_iter=4)
    pr = wl.prob
    p = tau.Problem(wl)
    assert p.stats().route[0] == tau.TAU_ROUTE_LONG
    rng = np.random.default_rng(n)
    ks = np.unique(np.concatenate([[1, 2, n // 2, n - 1, n], rng.integers(1, n + 1, 59)]))
    x = W.random_vector(n, 52)
    xd = _cuda(x)
    y = torch.empty_like(xd)
    z = torch.empty_like(xd)
    # DST-I rows
    tau.tau_dst(p.handle, xd, y)
    torch.cuda.synchronize()
    sx = _host(y)
    ref = O.sine_rows(n, ks) @ x
    assert np.abs(sx[ks - 1] - ref).max() <= 1e-12 * np.abs(ref).max() + 1e-13 * np.linalg.norm(x)
    tau.tau_dst(p.handle, y, z)
    torch.cuda.synchronize()
    assert np.linalg.norm(_host(z) - x) <= 1e-12 * np.linalg.norm(x)
    # Toeplitz rows
    tau.tau_toeplitz_mode(p.handle, 0, xd, y)
    torch.cuda.synchronize()
    ref = O.toeplitz_rows(pr.alpha[0], n, ks - 1) @ x
    got = _host(y)[ks - 1]
    assert np.abs(got - ref).max() <= 1e-12 * np.linalg.norm(x)
    # A rows: B(e∘x) + eta T x (Eq. (tls), d = 1)
    t = wl.field_tables()
    e = O.eval_field_interior(pr, t["e_tc"][0], t["e_sp"])
    tau.tau_apply_A(p.handle, 0, xd, y)
    torch.cuda.synchronize()
    ex = np.concatenate([[0.0], e * x, [0.0]])
    a = pr.alpha[0]
    ba = (1 - a / 12) * ex[ks] + (a / 24) * (ex[ks - 1] + ex[ks + 1])
    refA = ba + O.etas(pr)[0] * ref
    got = _host(y)[ks - 1]
    assert np.abs(got - refA).max() <= 1e-12 * O.etas(pr)[0] * np.linalg.norm(x)
    # tau solve at sampled modes: mu_k (S M^{-1} x)_k = (S x)_k
    ebar = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])[0]
    q = O.tau_eigs_q_at(O.fcd_weights(a, n), ks)
    mu = ebar * O.beta_eigs(a, n)[ks - 1] + O.etas(pr)[0] * q
    tau.tau_apply_Minv(p.handle, xd, y)
    tau.tau_dst(p.handle, y, z)
    torch.cuda.synchronize()
    lhs = mu * _host(z)[ks - 1]
    # q_k near k = 1 is a sum of O(1) terms with an absolute FP64 error ~ eps ||s||_1 (see the
    # M^{-1} tolerance of the FFT-route tests): allowance 4 eps eta 2 s_0 / min mu
    kq = O.etas(pr)[0] * 2 * O.fcd_weights(a, 1)[0] / mu.min()
    assert np.abs(lhs - sx[ks - 1]).max() <= (OP_RTOL + 4 * EPS * kq) * np.abs(sx).max()
    p.close()


@pytest.mark.parametrize("case", [
    (127, 4, 0, True),      # forced: the 1-D workload's size
    (1000, 3, 1, True),
    (5000, 3, 0, False),    # automatic choice
    (300, 3, 1, False),
])
def test_solve_parity(case):
    tau = _tau()
    n, M, x0, forced = case
    wl = _wl(n, M=M, x0_mode=x0)
    p = tau.Problem(wl, route=_long() if forced else (0, 0, 0))
    assert p.stats().route[0] == tau.TAU_ROUTE_LONG
    p.solve()
    u = p.solution().cpu().numpy()
    its = p.iters()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run()
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= SOLVE_RTOL, rel
    assert np.all(np.abs(its - np.array(ref.iters)) <= 1), (its, ref.iters)


def test_long_matches_fft_route():
    tau = _tau()
    wl = _wl(4095, M=3)
    a = tau.Problem(wl, route=(tau.TAU_ROUTE_FFT, 0, 0))
    assert a.stats().route[0] == tau.TAU_ROUTE_FFT
    a.solve()
    ua, ia = a.solution().cpu().numpy(), a.iters()
    a.close()
    b = tau.Problem(wl, route=_long())
    b.solve()
    ub, ib = b.solution().cpu().numpy(), b.iters()
    b.close()
    assert np.linalg.norm(ub - ua) <= 1e-11 * np.linalg.norm(ua)
    assert np.all(np.abs(ia - ib) <= 1)


def test_full_step_preconditioned_residual_at_65535():
    """One step at n = 65535: ||M^{-1}(b - A u^1)|| <= tol ||M^{-1} b|| up to rounding, with b, A and
    M^{-1} the library's own operators (each checked against the oracle above).  Forming b - A u in
    FP64 leaves a floor of about eps eta ||s||_1 ||u||_inf per entry (eta ~ 2e6 here), so the bound
    is 1e-9 rather than the GMRES tolerance 1e-12; a wrong solve gives O(1)."""
    tau = _tau()
    wl = _wl(65535, M=4)
    p = tau.Problem(wl)
    u0 = p.solution()
    b = torch.empty_like(u0)
    tau.tau_rhs(p.handle, 0, u0, b)
    p.step(1)
    u1 = p.solution()
    Au = torch.empty_like(u0)
    tau.tau_apply_A(p.handle, 0, u1, Au)
    r = b - Au
    z = torch.empty_like(u0)
    z0 = torch.empty_like(u0)
    tau.tau_apply_Minv(p.handle, r, z)
    tau.tau_apply_Minv(p.handle, b, z0)
    torch.cuda.synchronize()
    its = int(p.iters()[0])
    p.close()
    assert 1 <= its <= 30
    assert (torch.linalg.norm(z) / torch.linalg.norm(z0)).item() <= 1e-9


@pytest.mark.parametrize("prec", ["mixed", "df64"])
def test_precision_forms(prec):
    tau = _tau()
    precision = tau.TAU_MIXED if prec == "mixed" else tau.TAU_DF64
    bar = 1e-8 if prec == "mixed" else SOLVE_RTOL
    wl = _wl(5000, M=3)
    p = tau.Problem(wl, precision=precision)
    assert p.stats().route[0] == tau.TAU_ROUTE_LONG
    p.solve()
    u = p.solution().cpu().numpy()
    its = p.iters()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run()
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= bar, rel
    if prec == "df64":
        assert np.all(np.abs(its - np.array(ref.iters)) <= 1), (its, ref.iters)


def test_double_float_at_65535_against_fp64():
    """At n = 65535, eta ~ 3e6: the FP32 inner solve of the mixed form cannot resolve the operator
    (eps_32 eta ||s||_1 ~ 0.4), the double-float form (~48 bits) can."""
    tau = _tau()
    wl = _wl(65535, M=3)
    a = tau.Problem(wl)
    a.solve()
    ua = a.solution()
    ia = a.iters()
    a.close()
    b = tau.Problem(wl, precision=tau.TAU_DF64)
    assert b.stats().route[0] == tau.TAU_ROUTE_LONG
    b.solve()
    ub = b.solution()
    ib = b.iters()
    b.close()
    assert (torch.linalg.norm(ub - ua) / torch.linalg.norm(ua)).item() <= 1e-9
    assert np.all(np.abs(ia - ib) <= 1), (ia, ib)


def test_two_sided_on_long_route():
    tau = _tau()
    wl = _wl(5000, M=2)
    a = tau.Problem(wl)
    a.solve()
    ua = a.solution().cpu().numpy()
    a.close()
    b = tau.Problem(wl, method=tau.TAU_TPGM)
    assert b.stats().route[0] == tau.TAU_ROUTE_LONG
    b.solve()
    ub = b.solution().cpu().numpy()
    b.close()
    assert np.linalg.norm(ub - ua) <= 1e-10 * np.linalg.norm(ua)


def test_route_rejections():
    tau = _tau()
    base = W.c2_2d(n=63, M=2)
    with pytest.raises(tau.TauError) as ei:
        tau.Problem(base, route=(tau.TAU_ROUTE_LONG, 0, 0))
    assert ei.value.status == tau.TAU_EUNSUPPORTED
    with pytest.raises(tau.TauError) as ei:
        tau.Problem(_wl(127, M=2), route=_long(), method=tau.TAU_SPGM)
    assert ei.value.status == tau.TAU_EUNSUPPORTED


def test_served_long_request_same_as_alone():
    tau = _tau()
    wls = [_wl(20000, M=3), _wl(5000, M=4), W.c2_2d(n=200, M=3)]
    precs = [tau.TAU_MIXED, tau.TAU_FP64, tau.TAU_MIXED]
    s = tau.tau_server_create(8 << 30, 8, 2)
    ids = [tau.tau_server_submit(s, tau.make_desc(wl.prob, precision=pr), wl.field_tables())
           for wl, pr in zip(wls, precs)]
    infos = [tau.tau_server_wait(s, i, 300.0) for i in ids]
    assert all(inf.state == tau.TAU_REQ_DONE and inf.status == tau.TAU_OK for inf in infos)
    got = [tau.tau_server_result(s, i, wl.prob.n_tot) for i, wl in zip(ids, wls)]
    tau.tau_server_destroy(s)
    for wl, pr, um in zip(wls, precs, got):
        # alone as the server runs it: mixed requests on the line passes, recorded tuning choices
        p = tau.Problem(wl, precision=pr, tc=tau.TAU_TC_OFF if pr == tau.TAU_MIXED else 0,
                        autotune=tau.TAU_TUNE_RECORDED)
        p.solve()
        ua = p.solution().cpu().numpy()
        p.close()
        assert np.array_equal(ua, um)
