"""Tensor-core (tcgen05, TF32) DST-I mode products of the mixed form's FP32 τ solve.

Two bars.  (1) Against the kernel's own stated arithmetic, emulated here on the oracle's sine matrix:
every mode product takes TF32-rounded inputs (nearest, ties away) and a TF32-rounded S, accumulates
in FP32 and writes FP32, so M^{-1} r must agree with that emulation up to the accumulation error.
The tensor cores do not round every addition of a sum as IEEE FP32 does (products of a K-group are
aligned to the largest one), so that error is relative to sum |S_kj x_j| rather than to the result,
which the DST's cancellation makes the larger: measured 6.7e-5 at 255^2 and 2.1e-4 at 63^3.  The
bound is 1e-3, half a TF32 rounding step: a wrong operand layout or index gives O(1).  (2) Against
the exact oracle M^{-1}: within the TF32 bound (about 2^-11 per rounding, a few roundings deep).
Whole mixed-precision solves with the tensor-core preconditioner still meet the form's 1e-8 bar.
"""

import numpy as np
import pytest

import oracle as O
from paper_2404_10221_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tau():
    from paper_2404_10221_gb300 import tau
    return tau


def _wl(d, n, M=3):
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
    return wl


def tf32(a):
    """Round to TF32 (10 mantissa bits), to nearest with ties away from zero, as cvt.rna.tf32.f32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    b = (b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return b.view(np.float32).astype(np.float64)


def emulated_minv(pr, ebar, r, tc_dims):
    """M^{-1} r with the line passes of the FP32 chain: DST along dims d-1..1, DST·(1/mu)·DST along
    dim 0, DST along 1..d-1; a dimension in tc_dims takes the tensor-core arithmetic (TF32 inputs,
    FP32 output), the others exact products rounded to FP32 (a stand-in for the FFT line pass)."""
    d = pr.d
    shape = O.tau_oracle._shape(pr)
    X = np.asarray(r, dtype=np.float32).astype(np.float64).reshape(shape)
    invmu = (1.0 / O.mu_tensor(pr, ebar)).astype(np.float32).astype(np.float64).reshape(shape)
    S = [O.sine_matrix(pr.n[i]) for i in range(d)]

    def dst(X, i, mul=None):
        tc = i in tc_dims
        Si = tf32(S[i]) if tc else S[i]
        Xi = tf32(X) if tc else X
        Y = O.mode_product(Xi, Si, d - 1 - i)
        if mul is not None:
            Y = Y.astype(np.float32).astype(np.float64) * mul
        return Y.astype(np.float32).astype(np.float64)

    for i in range(d - 1, 0, -1):
        X = dst(X, i)
    X = dst(dst(X, 0, invmu), 0)
    for i in range(1, d):
        X = dst(X, i)
    return X.reshape(-1)


SHAPES = [(1, (127,)), (1, (100,)), (1, (5,)), (1, (256,)), (2, (31, 63)), (2, (20, 9)), (2, (255, 255)),
          (2, (300, 129)), (2, (129, 17)), (3, (15, 7, 31)), (3, (63, 63, 63)), (3, (2, 3, 5))]


@pytest.mark.parametrize("d,n", SHAPES)
def test_tc_minv_f32(d, n):
    tau = _tau()
    wl = _wl(d, n)
    pr = wl.prob
    pr.max_iter = 4
    p = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_ON)
    t = wl.field_tables()
    ebar = O.ebar_from_tables(pr, t["e_tc"], t["e_sp"])[0]
    x = W.random_vector(pr.n_tot, 61).astype(np.float32)
    y = torch.empty(pr.n_tot, dtype=torch.float32, device="cuda")
    tau.tau_apply_Minv_f32(p.handle, torch.from_numpy(x).to("cuda"), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    p.close()
    tc_dims = {i for i in range(d) if n[i] <= 256}
    emu = emulated_minv(pr, ebar, x, tc_dims)
    rel = np.linalg.norm(got - emu) / np.linalg.norm(emu)
    assert rel <= 1e-3, f"vs emulated TF32 arithmetic: {rel:.3e}"
    ref = O.apply_Minv(pr, ebar, x.astype(np.float64))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-2, f"vs exact M^-1: {rel:.3e}"


@pytest.mark.parametrize("case", [
    (1, (127,), 6),
    (2, (63, 127), 3),
    (3, (63, 63, 63), 2),
    (3, (15, 7, 31), 3),
])
def test_mixed_solve_with_tc_meets_the_form_bar(case):
    tau = _tau()
    d, n, M = case
    wl = _wl(d, n, M=M)
    p = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_ON)
    p.solve()
    u = p.solution().cpu().numpy()
    st = p.stats()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run()
    rel = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert rel <= 1e-8, rel
    assert st.steps_done == M


def test_tc_and_line_pass_solves_agree_at_255_cubed_two_steps():
    """The 3-D workload at its full size: two mixed-precision steps with the tensor-core DST and with
    the FP32 line passes land within the form's bar of each other."""
    tau = _tau()
    wl = W.c3_3d(M=50)
    a = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_ON)
    a.step(2)
    ua = a.solution()
    a.close()
    b = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_OFF)
    b.step(2)
    ub = b.solution()
    b.close()
    assert (torch.linalg.norm(ua - ub) / torch.linalg.norm(ub)).item() <= 1e-8


def test_tc_dims_reported():
    tau = _tau()
    # low bits: dimensions whose τ-solve DST runs on the tensor cores; bit 8: the split-TF32 matvec
    # (every dimension n <= 256)
    for n, on_mask, mv in (((63, 63, 63), 7, True), ((300, 129), 2, False), ((1000,), 0, False)):
        d = len(n)
        wl = _wl(d, n, M=2)
        wl.prob.max_iter = 4
        p = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_ON)
        st = p.stats().tc_dims
        assert st & 0xFF == on_mask and bool(st & 0x100) == mv, (n, st)
        p.close()
        p = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_OFF)
        assert p.stats().tc_dims == 0
        p.close()
        p = tau.Problem(wl, precision=tau.TAU_MIXED)   # automatic: measured choices
        st = p.stats().tc_dims
        assert st & 0xFF in (0, on_mask) and (mv or not st & 0x100)
        p.close()


@pytest.mark.parametrize("d,n", [(1, (127,)), (1, (5,)), (1, (256,)), (2, (31, 63)), (2, (255, 255)),
                                 (2, (20, 9)), (2, (129, 17)), (3, (15, 7, 31)), (3, (63, 63, 63)),
                                 (3, (2, 3, 5))])
def test_tc_split_matvec_f32(d, n):
    """A x in FP32 with the Toeplitz products as split-TF32 tensor-core products: FP32-level
    accuracy, the bound of the FP32 line passes (1e-5 relative against the oracle)."""
    tau = _tau()
    wl = _wl(d, n)
    pr = wl.prob
    pr.max_iter = 4
    p = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_ON)
    assert p.stats().tc_dims & 0x100
    t = wl.field_tables()
    x = W.random_vector(pr.n_tot, 62).astype(np.float32)
    y = torch.empty(pr.n_tot, dtype=torch.float32, device="cuda")
    for m in (0, 1):
        tau.tau_apply_A_f32(p.handle, m, torch.from_numpy(x).to("cuda"), y)
        torch.cuda.synchronize()
        e = O.eval_field_interior(pr, t["e_tc"][m], t["e_sp"])
        ref = O.apply_A(pr, e, x.astype(np.float64))
        got = y.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 1e-5, f"m={m}: {rel:.3e}"
    p.close()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The tensor-core kernels wait on mbarriers with a poll limit.  A wait on a barrier that
    nothing arrives at must end with the error status, not hang, and the CUDA context must stay
    usable: a tensor-core M^-1 product right after it still meets its bound."""
    tau = _tau()
    assert tau.tau_selftest_bounded_wait() is True
    test_tc_minv_f32(2, (31, 63))


def test_expired_wait_is_reported_once_by_sync():
    """The error path of an expired wait: the device flag that a tensor-core kernel sets when a
    bounded wait runs out (set here through the test hook; no wait is made to run out) makes the
    next sync return TAU_ETIMEOUT; the report clears it, so the sync after that is clean and the
    problem keeps working (a solve after it meets the form's bar against the oracle)."""
    tau = _tau()
    wl = _wl(2, (31, 15), M=2)
    p = tau.Problem(wl, precision=tau.TAU_MIXED, tc=tau.TAU_TC_ON)
    assert tau.tau_sync(p.handle) == tau.TAU_OK
    tau.tau_inject_wait_timeout(p.handle)
    with pytest.raises(tau.TauError) as ei:
        tau.tau_sync(p.handle)
    assert ei.value.status == tau.TAU_ETIMEOUT
    assert tau.tau_sync(p.handle) == tau.TAU_OK
    p.solve()
    u = p.solution().cpu().numpy()
    p.close()
    ref = O.OracleSolver(wl.prob, wl.field_tables())
    ref.run()
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-8
