"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element on the same seeded inputs.

Operators: FP64, relative 2-norm <= 1e-12 and max |diff| <= 1e-11 max |ref|
(FFT rounding is O(eps log n) ~ 1e-14).  Whole solves: relative 2-norm <= 1e-10
at GMRES tol 1e-12 with per-step iteration counts within +-1 of the oracle.
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


def minv_rtol(prob, ebar):
    """Tolerance for operators that divide by mu (M^{-1}, M^{-1}A).

    The small tau eigenvalues q_k (~(pi k/(n+1))^alpha) come out of a sum of O(1) terms of
    size ||s||_1, so any FP64 evaluation of them carries an absolute error of order
    eps ||s||_1; in mu_k it is multiplied by eta_i.  The resulting relative change of M^{-1} is
    bounded by kappa_q eps with kappa_q = sum_i eta_i ||s^(i)||_1 / min_k mu_k.
    """
    eta = O.etas(prob)
    l1 = [2 * O.fcd_weights(prob.alpha[i], prob.n[i])[0] for i in range(prob.d)]
    mu_min = O.mu_tensor(prob, ebar).min()
    kappa_q = sum(eta[i] * l1[i] for i in range(prob.d)) / mu_min
    return OP_RTOL + 4 * EPS * kappa_q


def _tau():
    from paper_2404_10221_gb300 import tau
    return tau


def _wl(d, n, M=3, seed=0, max_iter=100, x0_mode=0, tol=1e-12):
    """Workload with the C2/C3 coefficient shapes and per-dimension sizes n."""
    if d == 1:
        wl = W.c1_1d(n=n[0], M=M, tol=tol)
    elif d == 2:
        base = W.c2_2d(n=n[0], M=M, tol=tol)
        base.prob.n = list(n)
        wl = W.manufactured(f"2d_{n}", base.prob, base.e.terms, 2, 2, 1.0)
    else:
        base = W.c3_3d(n=n[0], M=M, tol=tol)
        base.prob.n = list(n)
        wl = W.manufactured(f"3d_{n}", base.prob, base.e.terms, 2, 2, 1.0)
    wl.prob.max_iter = max_iter
    wl.prob.x0_mode = x0_mode
    return wl


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _cmp(got, ref, rtol=OP_RTOL):
    got = got.detach().cpu().numpy() if hasattr(got, "detach") else got
    nr = np.linalg.norm(ref)
    rel = np.linalg.norm(got - ref) / nr
    assert rel <= rtol, f"rel 2-norm {rel:.3e}"
    assert np.abs(got - ref).max() <= 10 * rtol * np.abs(ref).max()


SHAPES = [
    (1, (1,)), (1, (3,)), (1, (7,)), (1, (127,)), (1, (1023,)), (1, (4095,)),
    (1, (5,)), (1, (100,)),                    # dense route (n+1 not a power of two)
    (2, (15, 7)), (2, (31, 63)), (2, (20, 9)), (2, (63, 5)),
    (3, (7, 15, 3)), (3, (5, 6, 7)), (3, (15, 15, 15)),
]


@pytest.fixture(scope="module")
def problems():
    cache = {}

    def get(d, n):
        key = (d, tuple(n))
        if key not in cache:
            wl = _wl(d, n, max_iter=4)
            # one-dimensional lines of n >= 1023 would take the long-line route automatically; this
            # file covers the one-CTA routes
            fft = all(((m + 1) & m) == 0 for m in n)
            route = (_tau().TAU_ROUTE_FFT, 0, 0) if d == 1 and fft else (0, 0, 0)
            cache[key] = (wl, _tau().Problem(wl, route=route))
        return cache[key]

    yield get
    for _, p in cache.values():
        p.close()


@pytest.mark.parametrize("d,n", SHAPES)
def test_dst_parity(problems, d, n):
    wl, p = problems(d, n)
    x = W.random_vector(wl.prob.n_tot, 11)
    y = torch.empty(wl.prob.n_tot, dtype=torch.float64, device="cuda")
    _tau().tau_dst(p.handle, _cuda(x), y)
    torch.cuda.synchronize()
    X = x.reshape(O.tau_oracle._shape(wl.prob))
    for i in range(d):
        X = O.mode_product(X, O.sine_matrix(n[i]), d - 1 - i)
    _cmp(y, X.reshape(-1))


@pytest.mark.parametrize("d,n", SHAPES)
def test_toeplitz_mode_parity(problems, d, n):
    wl, p = problems(d, n)
    x = W.random_vector(wl.prob.n_tot, 12)
    for dim in range(d):
        y = torch.empty(wl.prob.n_tot, dtype=torch.float64, device="cuda")
        _tau().tau_toeplitz_mode(p.handle, dim, _cuda(x), y)
        torch.cuda.synchronize()
        X = x.reshape(O.tau_oracle._shape(wl.prob))
        ref = O.mode_product(X, O.toeplitz_S(wl.prob.alpha[dim], n[dim]), d - 1 - dim).reshape(-1)
        _cmp(y, ref)


@pytest.mark.parametrize("d,n", SHAPES)
def test_apply_A_rhs_Minv_parity(problems, d, n):
    tau = _tau()
    wl, p = problems(d, n)
    pr = wl.prob
    t = wl.field_tables()
    ebar, ehat, echeck = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])
    g = tau.tau_get_ebar(p.handle)
    assert abs(g[0] - ebar) <= 1e-14 * ebar and abs(g[1] - ehat) <= 1e-14 * ehat
    x = W.random_vector(pr.n_tot, 13)
    xd = _cuda(x)
    y = torch.empty_like(xd)
    for m in (0, pr.M - 1):
        e = O.eval_field_interior(pr, t["e_tc"][m], t["e_sp"])
        tau.tau_apply_A(p.handle, m, xd, y)
        torch.cuda.synchronize()
        _cmp(y, O.apply_A(pr, e, x))
        tau.tau_rhs(p.handle, m, xd, y)
        torch.cuda.synchronize()
        F = O.rhs_F(pr, O.eval_field(pr, t["f_tc"][m], t["f_sp"]))
        _cmp(y, O.rhs_b(pr, e, x, F))
        tau.tau_apply_MinvA(p.handle, m, xd, y)
        torch.cuda.synchronize()
        _cmp(y, O.apply_Minv(pr, ebar, O.apply_A(pr, e, x)), minv_rtol(pr, ebar))
    tau.tau_apply_Minv(p.handle, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_Minv(pr, ebar, x), minv_rtol(pr, ebar))


def _solve_both(wl):
    tau = _tau()
    p = tau.Problem(wl)
    p.solve()
    u = p.solution().cpu().numpy()
    its = p.iters()
    st = p.stats()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run()
    return u, its, ref, st


@pytest.mark.parametrize("case", [
    (1, (127,), 32, 0),      # the 1-D workload in full
    (1, (31,), 6, 1),        # previous-step initial guess
    (1, (40,), 4, 0),        # dense route
    (2, (31, 31), 4, 0),
    (2, (15, 63), 3, 1),
    (2, (12, 31), 3, 0),     # mixed routes
    (3, (7, 7, 7), 3, 0),
    (3, (15, 7, 3), 2, 1),
])
def test_solve_parity(case):
    d, n, M, x0 = case
    wl = _wl(d, n, M=M, x0_mode=x0)
    u, its, ref, st = _solve_both(wl)
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= SOLVE_RTOL, f"rel {rel:.3e}"
    assert np.all(np.abs(its - np.array(ref.iters)) <= 1), (its, ref.iters)
    assert st.steps_done == M


def test_solve_parity_paper_example1_iterations():
    # Example 1 (Table 2, alpha = 1.5, N+1 = 32, tol 1e-9): GPU and oracle iterate alike.
    wl = W.paper_example(1, [1.5], 31, 4096)
    wl.prob.M = 4096
    tau = _tau()
    p = tau.Problem(wl)
    p.step(40)
    its = p.iters()[:40]
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run(steps=40)
    assert np.all(np.abs(its - np.array(ref.iters)) <= 1)


def test_full_size_2d_operators_and_five_steps():
    """The 2-D workload at its full size (1023^2 unknowns, M = 100): operators in full and the
    first five time steps against the oracle, for the plain FP64 path (1e-10, iterations +-1) and
    for the mixed-precision form (1e-8)."""
    tau = _tau()
    wl = W.c2_2d()
    pr = wl.prob
    p = tau.Problem(wl)
    t = wl.field_tables()
    ebar = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])[0]
    x = W.random_vector(pr.n_tot, 21)
    xd = _cuda(x)
    y = torch.empty_like(xd)
    e0 = O.eval_field_interior(pr, t["e_tc"][0], t["e_sp"])
    tau.tau_apply_A(p.handle, 0, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_A(pr, e0, x))
    tau.tau_apply_Minv(p.handle, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_Minv(pr, ebar, x), minv_rtol(pr, ebar))
    p.step(5)
    u = p.solution().cpu().numpy()
    its = p.iters()[:5]
    p.close()
    q = tau.Problem(wl, precision=tau.TAU_MIXED)
    q.step(5)
    umx = q.solution().cpu().numpy()
    q.close()
    ref = O.OracleSolver(pr, t)
    ref.run(steps=5)
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= SOLVE_RTOL, rel
    assert np.all(np.abs(its - np.array(ref.iters)) <= 1), (its, ref.iters)
    rel_mx = np.linalg.norm(umx - ref.u) / np.linalg.norm(ref.u)
    assert rel_mx <= 1e-8, rel_mx


def test_full_size_3d_mixed_step_against_oracle():
    """The 3-D workload at its full size (255^3 = 16.6M unknowns) in the mixed-precision form with
    its measured tensor-core choices: one Crank-Nicolson step against the oracle's structured tier
    (the form's bar, 1e-8)."""
    tau = _tau()
    wl = W.c3_3d()
    q = tau.Problem(wl, precision=tau.TAU_MIXED)
    q.step(1)
    u = q.solution().cpu().numpy()
    q.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run(steps=1)
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= 1e-8, rel


def test_full_size_3d_operators():
    """3-D at 255^3 (16.6M unknowns): A and M^{-1} in full against the oracle."""
    tau = _tau()
    wl = W.c3_3d()
    wl.prob.max_iter = 2
    pr = wl.prob
    p = tau.Problem(wl)
    t = wl.field_tables()
    ebar = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])[0]
    x = W.random_vector(pr.n_tot, 22)
    xd = _cuda(x)
    y = torch.empty_like(xd)
    e0 = O.eval_field_interior(pr, t["e_tc"][0], t["e_sp"])
    tau.tau_apply_A(p.handle, 0, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_A(pr, e0, x))
    tau.tau_apply_Minv(p.handle, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_Minv(pr, ebar, x), minv_rtol(pr, ebar))
    p.close()


def test_properties_dst_involution_and_minv_inverse():
    """S_d S_d = I and M (M^{-1} r) = r through the library at 1023^2."""
    tau = _tau()
    wl = W.c2_2d(M=2)
    wl.prob.max_iter = 2
    p = tau.Problem(wl)
    x = _cuda(W.random_vector(wl.prob.n_tot, 23))
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    tau.tau_dst(p.handle, x, y)
    tau.tau_dst(p.handle, y, z)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(z - x) / torch.linalg.norm(x)).item() <= 1e-13
    p.close()


def test_checkpoint_resume_matches_straight_run():
    tau = _tau()
    wl = _wl(2, (31, 15), M=6)
    a = tau.Problem(wl)
    a.solve()
    ua = a.solution().cpu().numpy()
    a.close()
    b = tau.Problem(wl)
    b.step(3)
    mid = b.solution().cpu().numpy()
    b.close()
    c = tau.Problem(wl)
    tau.tau_set_solution(c.handle, mid, False, 3)
    c.step(3)
    uc = c.solution().cpu().numpy()
    c.close()
    assert np.linalg.norm(uc - ua) <= 1e-13 * np.linalg.norm(ua)


def test_notconv_reported():
    tau = _tau()
    wl = _wl(2, (31, 31), M=2, max_iter=2, tol=1e-14)
    p = tau.Problem(wl)
    st = p.solve(allow_notconv=True)
    assert st == tau.TAU_ENOTCONV
    assert np.all(p.iters() == 2)
    p.close()


# Dense-route tiles that hold more than one round of 8 x 128 outputs (lines per CTA x n > 1024):
# lines of 65..127 points across a strided axis (16 or 8 lines per CTA), and single lines longer
# than 1024 points.  Every dense output reads the whole line, so the outputs must not overwrite
# it before all of them are computed.
DENSE_TILES = [
    ((251, 129, 76), (0, 0, 0)),          # chirp, chirp, dense (the rules' routes)
    ((251, 129, 76), (2, 2, 2)),          # dense on every axis
    ((90, 70), (2, 2)),                   # dense, 16 lines of 70 per CTA on the strided axis
    ((1500, 37), (2, 2)),                 # one dense line of 1500 per CTA
    ((2000,), (2,)),                      # 1-D, one line of 2000
]


@pytest.mark.parametrize("n,route", DENSE_TILES)
def test_dense_route_tiles_beyond_one_round(n, route):
    tau = _tau()
    d = len(n)
    wl = _wl(d, n, max_iter=4)
    pr = wl.prob
    p = tau.Problem(wl, route=tuple(route) + (0,) * (3 - d), autotune=tau.TAU_TUNE_OFF)
    st = p.stats()
    if route[0] == 2:
        assert all(r == tau.TAU_ROUTE_DENSE for r in st.route[:d])
    t = wl.field_tables()
    ebar = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])[0]
    x = W.random_vector(pr.n_tot, 31)
    xd = _cuda(x)
    y = torch.empty_like(xd)
    from oracle import tau_oracle as OT
    for dim in range(d):
        tau.tau_toeplitz_mode(p.handle, dim, xd, y)
        torch.cuda.synchronize()
        T = O.toeplitz_S(pr.alpha[dim], pr.n[dim])
        _cmp(y, O.mode_product(x.reshape(OT._shape(pr)), T, OT._axis(pr, dim)).reshape(-1))
    tau.tau_dst(p.handle, xd, y)
    torch.cuda.synchronize()
    X = x.reshape(OT._shape(pr))
    for i in range(d):
        X = O.mode_product(X, O.sine_matrix(pr.n[i]), OT._axis(pr, i))
    _cmp(y, X.reshape(-1))
    e0 = O.eval_field_interior(pr, t["e_tc"][0], t["e_sp"])
    tau.tau_apply_A(p.handle, 0, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_A(pr, e0, x))
    tau.tau_apply_Minv(p.handle, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_Minv(pr, ebar, x), minv_rtol(pr, ebar))
    p.close()


def test_3d_chirp_and_dense_step_against_oracle():
    """One Crank-Nicolson step of a 3-D grid whose axes take the chirp (251, 129) and dense (76)
    routes, plain FP64 (1e-10, iterations +-1) and mixed (1e-8), against the oracle."""
    tau = _tau()
    wl = _wl(3, (251, 129, 76), M=115)
    wl.prob.alpha = [1.82, 1.84, 1.68]
    wl.prob.kappa = [0.35, 0.3, 0.96]
    wl = W.manufactured("3d_chirp_dense", wl.prob, wl.e.terms, 2, 2, 1.0)
    p = tau.Problem(wl)
    p.step(1)
    u = p.solution().cpu().numpy()
    its = p.iters()[:1]
    p.close()
    q = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_OFF)
    q.step(1)
    umx = q.solution().cpu().numpy()
    q.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run(steps=1)
    assert np.linalg.norm(u - ref.u) <= SOLVE_RTOL * np.linalg.norm(ref.u)
    assert abs(int(its[0]) - ref.iters[0]) <= 1, (its, ref.iters)
    assert np.linalg.norm(umx - ref.u) <= 1e-8 * np.linalg.norm(ref.u)
