"""Chirp route: any n_i < 4096 (n_i + 1 not a power of two) through a power-of-two circulant
embedding for the Toeplitz products and a chirp-z convolution for the DST-I.

Held to the FFT route's bar against the FP64 oracle: operators to a relative 2-norm of 1e-12
(M^{-1} with the same conditioning allowance), whole solves to 1e-10 at GMRES tol 1e-12 with
iteration counts within +-1; the FP32 and double-float forms to their own bars.
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
EPS32 = float(np.finfo(np.float32).eps)


def _tau():
    from paper_2404_10221_gb300 import tau
    return tau


def _wl(d, n, M=3, x0_mode=0, max_iter=100):
    if d == 1:
        wl = W.c1_1d(n=n[0], M=M)
    elif d == 2:
        base = W.c2_2d(n=n[0], M=M)
        base.prob.n = list(n)
        wl = W.manufactured(f"2d_{n}", base.prob, base.e.terms, 2, 2, 1.0)
    else:
        base = W.c3_3d(n=n[0], M=M)
        base.prob.n = list(n)
        wl = W.manufactured(f"3d_{n}", base.prob, base.e.terms, 2, 2, 1.0)
    wl.prob.x0_mode = x0_mode
    wl.prob.max_iter = max_iter
    return wl


def _cuda(x, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).to("cuda")


def _cmp(got, ref, rtol=OP_RTOL):
    got = got.detach().cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= rtol, f"rel 2-norm {rel:.3e}"
    assert np.abs(got - ref).max() <= 10 * rtol * np.abs(ref).max()


def _kappa_q(prob, ebar):
    eta = O.etas(prob)
    l1 = [2 * O.fcd_weights(prob.alpha[i], prob.n[i])[0] for i in range(prob.d)]
    return sum(eta[i] * l1[i] for i in range(prob.d)) / O.mu_tensor(prob, ebar).min()


def _chirp(d):
    tau = _tau()
    return tuple([tau.TAU_ROUTE_CHIRP] * d + [0] * (3 - d))


# forced chirp route: tiny lines (M = 2, 4: the first DIF stage reads the whole line), lines
# whose n is a power of two (convolution length exactly 2n), and n up to the route's limit
FORCED_1D = [1, 2, 3, 5, 40, 127, 130, 256, 1000, 1500, 2048, 4000, 4094]


@pytest.mark.parametrize("n", FORCED_1D)
def test_dst_and_toeplitz_forced_chirp_1d(n):
    tau = _tau()
    wl = _wl(1, (n,), max_iter=4)
    p = tau.Problem(wl, route=_chirp(1))
    assert p.stats().route[0] == tau.TAU_ROUTE_CHIRP
    x = W.random_vector(n, 41)
    xd = _cuda(x)
    y = torch.empty_like(xd)
    tau.tau_dst(p.handle, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.sine_matrix(n) @ x)
    tau.tau_toeplitz_mode(p.handle, 0, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.toeplitz_S(wl.prob.alpha[0], n) @ x)
    p.close()


SHAPES = [
    (1, (130,)), (1, (1000,)), (1, (3000,)),
    (2, (300, 129)), (2, (1023, 200)), (2, (130, 5)), (2, (6, 256)),
    (3, (130, 7, 129)), (3, (15, 200, 3)),
]


@pytest.fixture(scope="module")
def problems():
    cache = {}

    def get(d, n):
        key = (d, tuple(n))
        if key not in cache:
            wl = _wl(d, n, max_iter=4)
            # one-dimensional problems would take the long-line route automatically
            cache[key] = (wl, _tau().Problem(wl, route=_chirp(1) if d == 1 else (0, 0, 0)))
        return cache[key]

    yield get
    for _, p in cache.values():
        p.close()


def test_auto_route_choice():
    tau = _tau()
    # d = 1: FFT for n + 1 = 2^p <= 512, dense below 128, the long-line route otherwise
    cases = [((127,), tau.TAU_ROUTE_FFT), ((511,), tau.TAU_ROUTE_FFT), ((100,), tau.TAU_ROUTE_DENSE),
             ((128,), tau.TAU_ROUTE_LONG), ((1023,), tau.TAU_ROUTE_LONG), ((4094,), tau.TAU_ROUTE_LONG)]
    for n, want in cases:
        p = tau.Problem(_wl(1, n, max_iter=2))
        assert p.stats().route[0] == want, (n, p.stats().route[0])
        p.close()
    # d >= 2: chirp for 128 <= n < 4096 with n + 1 not a power of two
    p = tau.Problem(_wl(2, (128, 4094), max_iter=2))
    assert p.stats().route[0] == tau.TAU_ROUTE_CHIRP and p.stats().route[1] == tau.TAU_ROUTE_CHIRP
    p.close()
    # double-float lines of n > 2047 do not fit in shared memory on the chirp route: dense instead
    p = tau.Problem(_wl(2, (3000, 5), max_iter=2), precision=tau.TAU_DF64)
    assert p.stats().route[0] == tau.TAU_ROUTE_DENSE
    p.close()
    with pytest.raises(tau.TauError) as ei:
        tau.Problem(_wl(1, (3000,), max_iter=2), precision=tau.TAU_DF64, route=_chirp(1))
    assert ei.value.status == tau.TAU_EUNSUPPORTED
    with pytest.raises(tau.TauError) as ei:
        tau.Problem(_wl(1, (4096,), max_iter=2), route=_chirp(1))
    assert ei.value.status == tau.TAU_EUNSUPPORTED


@pytest.mark.parametrize("d,n", SHAPES)
def test_operators_parity(problems, d, n):
    tau = _tau()
    wl, p = problems(d, n)
    pr = wl.prob
    shape = O.tau_oracle._shape(pr)
    x = W.random_vector(pr.n_tot, 42)
    xd = _cuda(x)
    y = torch.empty_like(xd)
    tau.tau_dst(p.handle, xd, y)
    torch.cuda.synchronize()
    X = x.reshape(shape)
    for i in range(d):
        X = O.mode_product(X, O.sine_matrix(n[i]), d - 1 - i)
    _cmp(y, X.reshape(-1))
    for dim in range(d):
        tau.tau_toeplitz_mode(p.handle, dim, xd, y)
        torch.cuda.synchronize()
        ref = O.mode_product(x.reshape(shape), O.toeplitz_S(pr.alpha[dim], n[dim]), d - 1 - dim)
        _cmp(y, ref.reshape(-1))
    t = wl.field_tables()
    ebar = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])[0]
    e = O.eval_field_interior(pr, t["e_tc"][1], t["e_sp"])
    tau.tau_apply_A(p.handle, 1, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_A(pr, e, x))
    tau.tau_apply_Minv(p.handle, xd, y)
    torch.cuda.synchronize()
    _cmp(y, O.apply_Minv(pr, ebar, x), OP_RTOL + 4 * EPS * _kappa_q(pr, ebar))


@pytest.mark.parametrize("case", [
    (1, (1000,), 4, 0),
    (1, (256,), 3, 1),
    (2, (300, 129), 3, 0),
    (2, (130, 31), 3, 1),
    (3, (130, 7, 15), 2, 0),
])
def test_solve_parity(case):
    tau = _tau()
    d, n, M, x0 = case
    wl = _wl(d, n, M=M, x0_mode=x0)
    p = tau.Problem(wl, route=_chirp(1) if d == 1 else (0, 0, 0))
    assert all(p.stats().route[i] == tau.TAU_ROUTE_CHIRP for i in range(d) if n[i] >= 128)
    p.solve()
    u = p.solution().cpu().numpy()
    its = p.iters()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run()
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= SOLVE_RTOL, rel
    assert np.all(np.abs(its - np.array(ref.iters)) <= 1), (its, ref.iters)


def test_forced_chirp_matches_fft_route_solve():
    """n + 1 = 2^p: the chirp route and the FFT route solve the same problem alike."""
    tau = _tau()
    wl = _wl(2, (127, 63), M=3)
    a = tau.Problem(wl)
    a.solve()
    ua = a.solution().cpu().numpy()
    ia = a.iters()
    a.close()
    b = tau.Problem(wl, route=_chirp(2))
    b.solve()
    ub = b.solution().cpu().numpy()
    ib = b.iters()
    b.close()
    assert np.linalg.norm(ub - ua) <= 1e-11 * np.linalg.norm(ua)
    assert np.all(np.abs(ia - ib) <= 1)


@pytest.mark.parametrize("d,n", [(1, (1000,)), (2, (300, 129)), (3, (130, 7, 15))])
def test_fp32_operators_parity(d, n):
    tau = _tau()
    wl = _wl(d, n, max_iter=4)
    pr = wl.prob
    p = tau.Problem(wl, precision=tau.TAU_MIXED, route=_chirp(1) if d == 1 else (0, 0, 0), tc=tau.TAU_TC_OFF)
    t = wl.field_tables()
    ebar = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])[0]
    x = W.random_vector(pr.n_tot, 43).astype(np.float32).astype(np.float64)
    y = torch.empty(pr.n_tot, dtype=torch.float32, device="cuda")
    tau.tau_apply_A_f32(p.handle, 1, _cuda(x, np.float32), y)
    torch.cuda.synchronize()
    e = O.eval_field_interior(pr, t["e_tc"][1], t["e_sp"])
    ref = O.apply_A(pr, e, x)
    got = y.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    tau.tau_apply_Minv_f32(p.handle, _cuda(x, np.float32), y)
    torch.cuda.synchronize()
    ref = O.apply_Minv(pr, ebar, x)
    got = y.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5 + 4 * EPS32 * _kappa_q(pr, ebar)
    p.close()


@pytest.mark.parametrize("prec", ["mixed", "df64"])
def test_precision_forms_on_chirp_route(prec):
    tau = _tau()
    precision = tau.TAU_MIXED if prec == "mixed" else tau.TAU_DF64
    bar = 1e-8 if prec == "mixed" else SOLVE_RTOL
    wl = _wl(2, (300, 129), M=3)
    p = tau.Problem(wl, precision=precision)
    assert p.stats().route[0] == tau.TAU_ROUTE_CHIRP and p.stats().route[1] == tau.TAU_ROUTE_CHIRP
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


def test_two_sided_method_on_chirp_route():
    tau = _tau()
    wl = _wl(2, (200, 31), M=2)
    a = tau.Problem(wl)
    a.solve()
    ua = a.solution().cpu().numpy()
    a.close()
    b = tau.Problem(wl, method=tau.TAU_TPGM)
    b.solve()
    ub = b.solution().cpu().numpy()
    b.close()
    assert np.linalg.norm(ub - ua) <= 1e-10 * np.linalg.norm(ua)


def test_batch_with_chirp_instances_same_as_alone():
    tau = _tau()
    shapes = [(300, 129), (130, 31), (127, 200), (200, 200)]
    wls = [_wl(2, n, M=3) for n in shapes]
    alone = []
    for wl in wls:
        p = tau.Problem(wl)
        p.solve()
        alone.append(p.solution().cpu().numpy())
        p.close()
    probs = [tau.Problem(wl) for wl in wls]
    b = tau.tau_batch_create([p.handle for p in probs])
    tau.tau_batch_step(b, 3)
    assert tau.tau_batch_sync(b) == tau.TAU_OK
    tau.tau_batch_destroy(b)
    for ua, p in zip(alone, probs):
        assert np.array_equal(ua, p.solution().cpu().numpy())
        p.close()
