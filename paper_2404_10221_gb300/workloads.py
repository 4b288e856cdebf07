"""Seeded synthetic input generators for the τ-preconditioned GMRES path.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle.  It holds none of the method's arithmetic (no discretisation, no
preconditioner, no Krylov step): it only describes problems and samples the
coefficient, source and initial fields on the grid.

Fields are separable expansions
    g(x, t) = sum_r  c_r(t) * prod_i phi_{r,i}(x_i),
which covers every test problem of the paper (Examples 1-3, §4) and the
benchmark workloads.  A field is handed to either side as tables:
  * ``time_coef``  [n_times, R]   c_r at the requested times,
  * ``space[i]``   [R, n_i + 2]   phi_{r,i} at x_{i,0..n_i+1} (boundary included).

The manufactured sources need the Riesz derivative (§1, definition below
Eq. (RSFDE)) of the exact solutions; for polynomial bumps
phi(x) = x^p (1-x)^q on (0,1) it has the closed form obtained from the
Riemann-Liouville power rule  D^a x^k = Gamma(k+1)/Gamma(k+1-a) x^(k-a).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Sequence

import numpy as np

TimeFn = Callable[[np.ndarray], np.ndarray]
SpaceFn = Callable[[np.ndarray], np.ndarray]


# --------------------------------------------------------------------------
# problem description
# --------------------------------------------------------------------------
@dataclass
class Problem:
    """Parameters of the RSFDE (§1, Eq. (RSFDE)) and of the solver (§4)."""

    d: int
    n: List[int]                 # interior points N_i per dimension
    alpha: List[float]           # orders alpha_i in (1,2)
    kappa: List[float]           # diffusion coefficients kappa_i >= 0
    T: float = 1.0
    M: int = 1                   # Crank-Nicolson steps, dt = T/M
    L: List[float] = field(default_factory=lambda: [0.0, 0.0, 0.0])
    R: List[float] = field(default_factory=lambda: [1.0, 1.0, 1.0])
    tol: float = 1e-12
    max_iter: int = 100
    x0_mode: int = 0             # 0: zero initial guess, 1: previous step

    @property
    def dt(self) -> float:
        return self.T / self.M

    def h(self, i: int) -> float:
        return (self.R[i] - self.L[i]) / (self.n[i] + 1)

    def grid(self, i: int) -> np.ndarray:
        """x_{i,j}, j = 0..N_i+1 (boundary included)."""
        return self.L[i] + self.h(i) * np.arange(self.n[i] + 2, dtype=np.float64)

    @property
    def n_tot(self) -> int:
        return int(np.prod(self.n[: self.d]))

    def half_times(self) -> np.ndarray:
        """t_{m+1/2}, m = 0..M-1."""
        return (np.arange(self.M, dtype=np.float64) + 0.5) * self.dt


@dataclass
class SeparableField:
    """g(x,t) = sum_r c_r(t) prod_i phi_{r,i}(x_i)."""

    terms: List[tuple]   # (time_fn, [space_fn_1, ..., space_fn_d])

    @property
    def rank(self) -> int:
        return len(self.terms)

    def tables(self, prob: Problem, times: Sequence[float]):
        times = np.asarray(times, dtype=np.float64)
        R = self.rank
        tc = np.zeros((len(times), R), dtype=np.float64)
        space = []
        for r, (tf, _) in enumerate(self.terms):
            tc[:, r] = np.broadcast_to(tf(times), times.shape)
        for i in range(prob.d):
            x = prob.grid(i)
            s = np.zeros((R, prob.n[i] + 2), dtype=np.float64)
            for r, (_, sf) in enumerate(self.terms):
                s[r, :] = np.broadcast_to(sf[i](x), x.shape)
            space.append(s)
        return tc, space


def _const(c: float) -> TimeFn:
    return lambda t: np.full_like(np.asarray(t, dtype=np.float64), c)


def _one(x):
    return np.ones_like(x)


# --------------------------------------------------------------------------
# closed-form Riesz derivative of polynomial bumps (input generation only)
# --------------------------------------------------------------------------
def _poly_coeffs(p: int, q: int) -> np.ndarray:
    """Coefficients c_k of x^p (1-x)^q = sum_k c_k x^k."""
    c = np.zeros(p + q + 1)
    for j in range(q + 1):
        c[p + j] = math.comb(q, j) * (-1) ** j
    return c


def riesz_bump(p: int, q: int, alpha: float, scale: float = 1.0) -> SpaceFn:
    """Riesz derivative of scale * x^p (1-x)^q on (0,1) (zero outside).

    Left RL derivative from 0 uses the expansion in powers of x, the right
    one from 1 the expansion in powers of (1-x); sigma_alpha =
    -1/(2 cos(alpha*pi/2)) as in §1.
    """
    cl = _poly_coeffs(p, q)          # powers of x
    cr = _poly_coeffs(q, p)          # powers of y = 1-x
    sigma = -1.0 / (2.0 * math.cos(alpha * math.pi / 2.0))

    def f(x):
        x = np.asarray(x, dtype=np.float64)
        y = 1.0 - x
        xl = np.clip(x, 0.0, None)
        yl = np.clip(y, 0.0, None)
        out = np.zeros_like(x)
        for k, c in enumerate(cl):
            if c != 0.0:
                g = math.gamma(k + 1) / math.gamma(k + 1 - alpha)
                out = out + c * g * np.where(xl > 0, xl, 1.0) ** (k - alpha) * (xl > 0)
        for k, c in enumerate(cr):
            if c != 0.0:
                g = math.gamma(k + 1) / math.gamma(k + 1 - alpha)
                out = out + c * g * np.where(yl > 0, yl, 1.0) ** (k - alpha) * (yl > 0)
        return scale * sigma * out

    return f


def bump(p: int, q: int, scale: float = 1.0) -> SpaceFn:
    return lambda x: scale * np.asarray(x, dtype=np.float64) ** p * (1.0 - np.asarray(x, dtype=np.float64)) ** q


# --------------------------------------------------------------------------
# manufactured problems  u*(x,t) = exp(-t) prod_i phi(x_i)
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    prob: Problem
    e: SeparableField
    f: SeparableField
    psi: SeparableField
    exact: Callable[[float], np.ndarray] | None = None   # u*(G, t) on the interior grid

    def field_tables(self):
        """All tables both sides consume: e and f at t_{m+1/2}, psi at t=0."""
        th = self.prob.half_times()
        e_tc, e_sp = self.e.tables(self.prob, th)
        f_tc, f_sp = self.f.tables(self.prob, th)
        p_tc, p_sp = self.psi.tables(self.prob, [0.0])
        return dict(e_tc=e_tc, e_sp=e_sp, f_tc=f_tc, f_sp=f_sp, psi_tc=p_tc, psi_sp=p_sp)


def manufactured(name: str, prob: Problem, e_terms: list, p: int, q: int, amp: float) -> Workload:
    """Build f = e du/dt - sum_i kappa_i d^{alpha_i} u for u = amp e^{-t} prod phi(x_i).

    e_terms: list of (time_fn, [space_fns]) for e(x,t).
    Interval (L_i, R_i) is mapped to (0,1) affinely; the Riesz derivative
    picks up the factor (R_i - L_i)^{-alpha_i}.
    """
    d = prob.d

    def mapped(i, fn):
        Li, Ri = prob.L[i], prob.R[i]
        return lambda x: fn((np.asarray(x) - Li) / (Ri - Li))

    phis = [mapped(i, bump(p, q)) for i in range(d)]
    f_terms = []
    # e * du/dt = -e u
    for tf, sfs in e_terms:
        f_terms.append((lambda t, tf=tf: -amp * np.exp(-t) * tf(t),
                        [(lambda x, a=sfs[i], b=phis[i]: a(x) * b(x)) for i in range(d)]))
    # - kappa_i d^{alpha_i} u
    for i in range(d):
        Li, Ri = prob.L[i], prob.R[i]
        rz = riesz_bump(p, q, prob.alpha[i], scale=(Ri - Li) ** (-prob.alpha[i]))
        sf = [phis[l] if l != i else mapped(i, rz) for l in range(d)]
        kap = prob.kappa[i]
        f_terms.append((lambda t, kap=kap: -kap * amp * np.exp(-t), sf))
    psi = SeparableField([(_const(amp), phis)])

    def exact(t):
        g = [phis[i](prob.grid(i)[1:-1]) for i in range(d)]
        u = g[0]
        for i in range(1, d):
            u = np.multiply.outer(g[i], u)
        return amp * math.exp(-t) * u.reshape(-1)

    return Workload(name, prob, SeparableField(e_terms), SeparableField(f_terms), psi, exact)


def _sinpi(x):
    return np.sin(np.pi * np.asarray(x))


def _cospi(x):
    return np.cos(np.pi * np.asarray(x))


def c1_1d(n: int = 127, M: int = 32, tol: float = 1e-12) -> Workload:
    """1-D, alpha=1.5, kappa=1, e=1+0.5 sin(pi x)(1+t), u=e^{-t}x^2(1-x)^2."""
    prob = Problem(d=1, n=[n], alpha=[1.5], kappa=[1.0], T=1.0, M=M, tol=tol)
    e_terms = [(_const(1.0), [_one]), (lambda t: 0.5 * (1.0 + t), [_sinpi])]
    return manufactured(f"1d_n{n}_M{M}", prob, e_terms, 2, 2, 1.0)


def c2_2d(n: int = 1023, M: int = 100, tol: float = 1e-12) -> Workload:
    """2-D, alpha=(1.4,1.8), kappa=(1,0.5), e=2+sin(pi x)cos(pi y)(1+t)."""
    prob = Problem(d=2, n=[n, n], alpha=[1.4, 1.8], kappa=[1.0, 0.5], T=1.0, M=M, tol=tol)
    e_terms = [(_const(2.0), [_one, _one]), (lambda t: 1.0 + t, [_sinpi, _cospi])]
    return manufactured(f"2d_n{n}_M{M}", prob, e_terms, 2, 2, 1.0)


def c3_3d(n: int = 255, M: int = 50, tol: float = 1e-12) -> Workload:
    """3-D, alpha=(1.2,1.5,1.9), kappa=(1,1,0.5), e=1.5+0.5 prod sin(pi x_i)(1+t)."""
    prob = Problem(d=3, n=[n, n, n], alpha=[1.2, 1.5, 1.9], kappa=[1.0, 1.0, 0.5], T=1.0, M=M, tol=tol)
    e_terms = [(_const(1.5), [_one, _one, _one]), (lambda t: 0.5 * (1.0 + t), [_sinpi, _sinpi, _sinpi])]
    return manufactured(f"3d_n{n}_M{M}", prob, e_terms, 2, 2, 1.0)


def paper_example(d: int, alpha: Sequence[float], n: int, M: int, tol: float | None = None) -> Workload:
    """Examples 1-3 of §4: u = 100^d e^{-t} prod x_i^4 (1-x_i)^4."""
    kappa = {1: [100.0], 2: [100.0, 100.0], 3: [100.0, 85.0, 103.0]}[d]
    if tol is None:
        tol = 1e-10 if d == 3 else 1e-9
    max_iter = {1: 10, 2: 100, 3: 200}[d]
    prob = Problem(d=d, n=[n] * d, alpha=list(alpha), kappa=kappa, T=1.0, M=M, tol=tol, max_iter=max_iter)
    div = 50.0 if d == 1 else 100.0
    sq = lambda x: np.asarray(x) ** 2
    e_terms = []
    for i in range(d):
        e_terms.append((_const(1.0 / div), [sq if l == i else _one for l in range(d)]))
    e_terms.append((lambda t: np.exp(-t) / div, [_one] * d))
    return manufactured(f"example{d}_a{'-'.join(map(str, alpha))}_n{n}_M{M}", prob, e_terms, 4, 4, 100.0 ** d)


# --------------------------------------------------------------------------
# seeded random workloads (splitmix64, published by Steele/Lea/Flood 2014)
# --------------------------------------------------------------------------
class SplitMix64:
    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def choice(self, seq):
        return seq[self.next_u64() % len(seq)]


def random_2d(rng: SplitMix64, sizes=(63, 127, 255, 511), M: int = 20, tol: float = 1e-12) -> Workload:
    """One instance of the uneven batched mix: n_x, n_y from `sizes`,
    alpha_i ~ U(1.1,1.9), kappa_i ~ U(0.2,1), e = 1 + a sin(pi x) sin(pi y)(1+t)."""
    nx, ny = rng.choice(sizes), rng.choice(sizes)
    a1, a2 = rng.uniform(1.1, 1.9), rng.uniform(1.1, 1.9)
    k1, k2 = rng.uniform(0.2, 1.0), rng.uniform(0.2, 1.0)
    amp = rng.uniform(0.1, 1.0)
    prob = Problem(d=2, n=[nx, ny], alpha=[a1, a2], kappa=[k1, k2], T=1.0, M=M, tol=tol)
    e_terms = [(_const(1.0), [_one, _one]), (lambda t, a=amp: a * (1.0 + t), [_sinpi, _sinpi])]
    return manufactured(f"rand2d_{nx}x{ny}", prob, e_terms, 2, 2, 1.0)


def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded N(0,1)-like FP64 vector for operator-level parity tests."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n)


def random_positive(n: int, seed: int, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n)


def serving_mix(count: int, seed: int = 20240416, M_range=(10, 40), precision_hint: str = "mixed",
                n1_range=(1023, 65535), n2_range=(127, 2047), n3_range=(63, 255)) -> List[Workload]:
    """Request mix of the served form: 40 % 1-D with n uniform on n1_range, 45 % 2-D with n uniform on
    n2_range per axis (uneven), 15 % 3-D with n uniform on n3_range per axis; M uniform in M_range;
    alpha_i ~ U(1.1,1.9), kappa_i ~ U(0.2,1), e = 1 + a prod sin(pi x_i)(1+t), a ~ U(0.1,1).
    Any integer n: lines whose n + 1 is a power of two take the FFT route, the others the chirp
    route (n >= 128) or the dense one; 1-D lines with n >= 4096 the long-line route."""
    rng = SplitMix64(seed)
    out = []
    lo, hi = M_range

    def draw(r):
        return r[0] + int(rng.next_u64() % (r[1] - r[0] + 1))

    for _ in range(count):
        u = rng.uniform()
        M = lo + int(rng.uniform() * (hi - lo + 1))
        if u < 0.40:
            d, n = 1, [draw(n1_range)]
        elif u < 0.85:
            d, n = 2, [draw(n2_range), draw(n2_range)]
        else:
            d, n = 3, [draw(n3_range) for _ in range(3)]
        alpha = [rng.uniform(1.1, 1.9) for _ in range(d)]
        kappa = [rng.uniform(0.2, 1.0) for _ in range(d)]
        amp = rng.uniform(0.1, 1.0)
        prob = Problem(d=d, n=n, alpha=alpha, kappa=kappa, T=1.0, M=M, tol=1e-12)
        e_terms = [(_const(1.0), [_one] * d), (lambda t, a=amp: a * (1.0 + t), [_sinpi] * d)]
        out.append(manufactured(f"req{d}d", prob, e_terms, 2, 2, 1.0))
    return out


def dense_fields(prob: Problem, time_dependent_e: bool = True, with_f: bool = True) -> dict:
    """Fields that are not separable expansions, sampled on the grid (for the device-array field
    form of the boundary): e = 1 + (x_1 x_2 ... x_d) exp(-t x_1) (positive), f = sin(pi x_1 x_2 ...)
    (1 + t) + x_1^2 cos(pi t (x_2 + ... )), psi = prod x_i (1 - x_i) exp(x_1 x_d), each at
    t_{m+1/2}; x_1 fastest.  Returns e_dense (M, n_tot) or (n_tot,), f_dense (M, prod(n_i+2)) or
    None, psi_dense (n_tot,)."""
    d = prob.d
    pad = [prob.grid(i) for i in range(d)]

    def mesh(axes):
        # arrays of shape (n_d, ..., n_1): index i of the list is dimension i + 1
        grids = np.meshgrid(*reversed(axes), indexing="ij")
        return list(reversed(grids))

    xi = mesh([g[1:-1] for g in pad])
    xp = mesh(pad)
    prod_i = np.prod(np.stack(xi), axis=0)
    prod_p = np.prod(np.stack(xp), axis=0)
    rest_p = sum(xp[1:]) if d > 1 else np.zeros_like(xp[0])
    ts = prob.half_times()
    if time_dependent_e:
        e = np.stack([(1.0 + prod_i * np.exp(-t * xi[0])).reshape(-1) for t in ts])
    else:
        e = (1.0 + prod_i * np.exp(-0.5 * xi[0])).reshape(-1)
    f = None
    if with_f:
        f = np.stack([(np.sin(np.pi * prod_p) * (1.0 + t) + xp[0] ** 2 * np.cos(np.pi * t * rest_p)).reshape(-1)
                      for t in ts])
    psi = np.prod(np.stack([x * (1.0 - x) for x in xi]), axis=0) * np.exp(xi[0] * xi[-1])
    return {"e_dense": e, "f_dense": f, "psi_dense": psi.reshape(-1)}
