"""Plain FP64 NumPy oracle (test infrastructure only; see package header).

Array convention: a grid vector is stored with x_1 fastest (lexicographic
order of §2, which the Kronecker order B_{alpha_d} ⊗ ... ⊗ B_{alpha_1} of
Eq. (Salpha) implies).  As a NumPy array it has shape (N_d, ..., N_1), so
dimension i (1-based) is array axis d - i.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

__all__ = [
    "fcd_weights", "fcd_weights_gamma", "tridiag_B", "toeplitz_S", "hankel_H", "tau_of",
    "sine_matrix", "tau_eigs_q", "beta_eigs", "etas", "kron_all", "mode_product",
    "dense_B", "dense_S", "dense_tauS", "dense_A", "dense_M", "dense_P",
    "apply_B", "apply_A", "apply_S", "apply_Minv", "mu_tensor", "ebar_from_tables",
    "eval_field", "eval_field_interior", "rhs_F", "rhs_b", "gmres", "GmresResult",
    "step_direct", "time_march", "l2_error", "OracleSolver", "fcd_apply_line",
    "gmres_paper_form", "theorem_c", "two_sided_gmres", "two_sided_structured", "beta_tensor",
    "apply_sine_diag", "numerical_range_bounds", "spectral_summary", "strang_circulant",
    "circulant_dense", "strang_pc_eigs", "dense_Pc", "apply_Pc_inv", "spgm", "sine_rows",
    "toeplitz_rows", "tau_eigs_q_at",
]


# --------------------------------------------------------------------------
# §2: FCD weights, B_{alpha_i}, S_{alpha_i}
# --------------------------------------------------------------------------
def fcd_weights(alpha: float, n: int) -> np.ndarray:
    """s_0..s_{n-1} by the recurrence of §2 (below Eq. (eq0)):
    s_0 = Gamma(alpha+1)/Gamma(alpha/2+1)^2, s_k = (1 - (alpha+1)/(alpha/2+k)) s_{k-1}."""
    s = np.zeros(n, dtype=np.float64)
    if n == 0:
        return s
    s[0] = math.gamma(alpha + 1.0) / math.gamma(alpha / 2.0 + 1.0) ** 2
    for k in range(1, n):
        s[k] = (1.0 - (alpha + 1.0) / (alpha / 2.0 + k)) * s[k - 1]
    return s


def fcd_weights_gamma(alpha: float, n: int) -> np.ndarray:
    """s_j = (-1)^j Gamma(alpha+1) / (Gamma(alpha/2-j+1) Gamma(alpha/2+j+1)), §2 (FCD formula)."""
    out = np.zeros(n, dtype=np.float64)
    for j in range(n):
        out[j] = (-1.0) ** j * math.gamma(alpha + 1.0) / (
            math.gamma(alpha / 2.0 - j + 1.0) * math.gamma(alpha / 2.0 + j + 1.0))
    return out


def fcd_apply_line(alpha: float, h: float, u_pad: np.ndarray) -> np.ndarray:
    """delta^alpha u at interior nodes, §2 (display below Eq. (2.1)):
    -(1/h^alpha) sum_j s_j u(x - j h) over all grid nodes of the interval.
    u_pad holds u at x_0..x_{N+1}; returns the N interior values."""
    Np2 = len(u_pad)
    N = Np2 - 2
    s = fcd_weights(alpha, Np2)
    out = np.zeros(N)
    for jj in range(1, N + 1):
        acc = 0.0
        for l in range(Np2):
            acc += s[abs(jj - l)] * u_pad[l]
        out[jj - 1] = -acc / h ** alpha
    return out


def tridiag_B(alpha: float, n: int) -> np.ndarray:
    """B_{alpha_i} = I_N + (alpha_i/24) tridiag(1,-2,1), Eq. (Ha)."""
    B = np.eye(n) * (1.0 - alpha / 12.0)
    idx = np.arange(n - 1)
    B[idx, idx + 1] = alpha / 24.0
    B[idx + 1, idx] = alpha / 24.0
    return B


def toeplitz_S(alpha: float, n: int) -> np.ndarray:
    """Symmetric Toeplitz S_{alpha_i} with first column s_0..s_{N-1}, Eq. (eq0)."""
    s = fcd_weights(alpha, n)
    i = np.arange(n)
    return s[np.abs(i[:, None] - i[None, :])]


# --------------------------------------------------------------------------
# §3: tau matrices
# --------------------------------------------------------------------------
def hankel_H(t: np.ndarray) -> np.ndarray:
    """Hankel part H(T) of Eq. (tau): first row (t_2, ..., t_{N-1}, 0, 0),
    persymmetric, last row (0, 0, t_{N-1}, ..., t_2).  With 1-based (i, j):
    H_ij = t_{i+j} for i+j <= N-1 and t_{2N+2-i-j} for i+j >= N+3."""
    n = len(t)
    H = np.zeros((n, n))
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            s = i + j
            if s <= n - 1:
                H[i - 1, j - 1] = t[s]
            elif s >= n + 3:
                H[i - 1, j - 1] = t[2 * n + 2 - s]
    return H


def tau_of(t: np.ndarray) -> np.ndarray:
    """Natural tau approximation tau(T) = T - H(T), Eq. (tau)."""
    n = len(t)
    i = np.arange(n)
    T = t[np.abs(i[:, None] - i[None, :])]
    return T - hankel_H(t)


def sine_matrix(n: int) -> np.ndarray:
    """S = sqrt(2/(N+1)) [sin(pi j k/(N+1))]_{j,k=1..N}, §3 (below Eq. (q)).
    The integer j*k is reduced modulo 2(N+1) before forming the angle (sin has period 2 pi),
    so no entry is evaluated at a large, rounded argument."""
    j = np.arange(1, n + 1, dtype=np.int64)
    jk = np.outer(j, j) % (2 * (n + 1))
    return math.sqrt(2.0 / (n + 1)) * np.sin(np.pi * jk / (n + 1))


def tau_eigs_q(t: np.ndarray) -> np.ndarray:
    """q_i = t_0 + 2 sum_{j=1}^{N-1} t_j cos(pi j (i+1)/(N+1)), i = 0..N-1, Eq. (q)."""
    n = len(t)
    i1 = np.arange(1, n + 1, dtype=np.int64)          # i + 1 for i = 0..N-1
    q = np.full(n, t[0], dtype=np.float64)
    for j in range(1, n):
        # angle pi j (i+1)/(N+1) with j (i+1) reduced modulo 2(N+1) (cos has period 2 pi)
        q += 2.0 * t[j] * np.cos(np.pi * ((j * i1) % (2 * (n + 1))) / (n + 1))
    return q


def sine_rows(n: int, ks: np.ndarray) -> np.ndarray:
    """Rows k (1-based, the entries of ks) of S of §3 (below Eq. (q)), for grids too large for
    the whole matrix; j*k reduced modulo 2(N+1) as in sine_matrix."""
    j = np.arange(1, n + 1, dtype=np.int64)
    jk = np.outer(np.asarray(ks, dtype=np.int64), j) % (2 * (n + 1))
    return math.sqrt(2.0 / (n + 1)) * np.sin(np.pi * jk / (n + 1))


def toeplitz_rows(alpha: float, n: int, ks: np.ndarray) -> np.ndarray:
    """Rows k (0-based, the entries of ks) of the Toeplitz S_{alpha_i} of Eq. (eq0): s_|k-j|."""
    s = fcd_weights(alpha, n)
    j = np.arange(n)
    return s[np.abs(np.asarray(ks, dtype=np.int64)[:, None] - j[None, :])]


def tau_eigs_q_at(t: np.ndarray, ks: np.ndarray) -> np.ndarray:
    """q at the 1-based sine modes ks: q = t_0 + 2 sum_{j=1}^{N-1} t_j cos(pi j k/(N+1)), Eq. (q),
    one mode at a time (O(N) each); j k reduced modulo 2(N+1)."""
    n = len(t)
    j = np.arange(1, n, dtype=np.int64)
    out = np.empty(len(ks), dtype=np.float64)
    for a, k in enumerate(np.asarray(ks, dtype=np.int64)):
        out[a] = t[0] + 2.0 * np.dot(t[1:], np.cos(np.pi * ((j * k) % (2 * (n + 1))) / (n + 1)))
    return out


def beta_eigs(alpha: float, n: int) -> np.ndarray:
    """Eigenvalues of B_{alpha_i} on sine mode k = 1..N: 1 - (alpha/6) sin^2(k pi/(2N+2)), Lemma Heig."""
    k = np.arange(1, n + 1)
    return 1.0 - (alpha / 6.0) * np.sin(k * np.pi / (2 * n + 2)) ** 2


def etas(prob) -> List[float]:
    """eta_i = kappa_i dt / (2 h_i^{alpha_i}), Eq. (Salpha)."""
    return [prob.kappa[i] * prob.dt / (2.0 * prob.h(i) ** prob.alpha[i]) for i in range(prob.d)]


# --------------------------------------------------------------------------
# dense tier (explicit Kronecker assembly, Eqs. (tls), (Salpha), (tauSalpha), (Pa))
# --------------------------------------------------------------------------
def kron_all(mats_d_to_1: List[np.ndarray]) -> np.ndarray:
    """mats given in the order (dim d, ..., dim 1); returns their Kronecker product."""
    out = mats_d_to_1[0]
    for m in mats_d_to_1[1:]:
        out = np.kron(out, m)
    return out


def _per_dim(prob, fn):
    return [fn(prob.alpha[i], prob.n[i]) for i in range(prob.d)]


def dense_B(prob) -> np.ndarray:
    Bs = _per_dim(prob, tridiag_B)
    return kron_all(Bs[::-1])


def _dense_sum(prob, inner: List[np.ndarray]) -> np.ndarray:
    """sum_i eta_i (B_d ⊗ ... ⊗ inner_i ⊗ ... ⊗ B_1)."""
    Bs = _per_dim(prob, tridiag_B)
    eta = etas(prob)
    out = 0.0
    for i in range(prob.d):
        mats = [inner[i] if l == i else Bs[l] for l in range(prob.d)]
        out = out + eta[i] * kron_all(mats[::-1])
    return out


def dense_S(prob) -> np.ndarray:
    """S_alpha, Eq. (Salpha)."""
    return _dense_sum(prob, _per_dim(prob, toeplitz_S))


def dense_tauS(prob) -> np.ndarray:
    """tau(S_alpha), Eq. (tauSalpha)."""
    return _dense_sum(prob, [tau_of(fcd_weights(prob.alpha[i], prob.n[i])) for i in range(prob.d)])


def dense_A(prob, e_vec: np.ndarray) -> np.ndarray:
    """A^{(m)} = B_alpha E^{(m+1/2)} + S_alpha, Eq. (tls)."""
    return dense_B(prob) @ np.diag(e_vec) + dense_S(prob)


def dense_P(prob, ebar: float) -> np.ndarray:
    """P_alpha = ebar I + B^{-1/2} tau(S) B^{-1/2} = ebar I + B^{-1} tau(S) (Eq. (Pa) and the
    commutativity remark of §3)."""
    B = dense_B(prob)
    return ebar * np.eye(B.shape[0]) + np.linalg.solve(B, dense_tauS(prob))


def dense_M(prob, ebar: float) -> np.ndarray:
    """M = B_alpha P_alpha = ebar B_alpha + tau(S_alpha): the preconditioner of the
    algebraically identical A-form  M^{-1} A u = M^{-1} b  of Eq. (one-sided)."""
    return ebar * dense_B(prob) + dense_tauS(prob)


# --------------------------------------------------------------------------
# structured tier: per-dimension mode products with explicit N_i x N_i matrices
# --------------------------------------------------------------------------
def mode_product(X: np.ndarray, K: np.ndarray, axis: int) -> np.ndarray:
    """Y[..., j, ...] = sum_l K[j, l] X[..., l, ...] along `axis`."""
    Y = np.tensordot(K, X, axes=([1], [axis]))
    return np.moveaxis(Y, 0, axis)


def _shape(prob):
    return tuple(prob.n[i] for i in range(prob.d - 1, -1, -1))


def _axis(prob, i):
    return prob.d - 1 - i


def apply_B_line(X: np.ndarray, alpha: float, axis: int) -> np.ndarray:
    """B_{alpha_i} along one axis as the 3-point stencil of 𝓗_{alpha} (Eq. (2.2)), zero boundary."""
    Y = (1.0 - alpha / 12.0) * X
    Xm = np.moveaxis(X, axis, 0)
    Ym = np.moveaxis(Y, axis, 0)
    Ym[1:] += (alpha / 24.0) * Xm[:-1]
    Ym[:-1] += (alpha / 24.0) * Xm[1:]
    return Y


def apply_B(prob, x: np.ndarray) -> np.ndarray:
    """B_alpha x."""
    X = x.reshape(_shape(prob))
    for i in range(prob.d):
        X = apply_B_line(X, prob.alpha[i], _axis(prob, i))
    return X.reshape(-1)


def apply_S(prob, x: np.ndarray, toeps: Optional[List[np.ndarray]] = None) -> np.ndarray:
    """S_alpha x = sum_i eta_i (B ⊗ .. ⊗ S_{alpha_i} ⊗ .. ⊗ B) x, Eq. (Salpha)."""
    if toeps is None:
        toeps = _per_dim(prob, toeplitz_S)
    eta = etas(prob)
    X = x.reshape(_shape(prob))
    out = np.zeros_like(X)
    for i in range(prob.d):
        Y = mode_product(X, toeps[i], _axis(prob, i))
        for l in range(prob.d):
            if l != i:
                Y = apply_B_line(Y, prob.alpha[l], _axis(prob, l))
        out += eta[i] * Y
    return out.reshape(-1)


def apply_A(prob, e_vec: np.ndarray, x: np.ndarray, toeps=None) -> np.ndarray:
    """A x = B_alpha (e ∘ x) + S_alpha x, Eq. (tls)."""
    return apply_B(prob, e_vec * x) + apply_S(prob, x, toeps)


def mu_tensor(prob, ebar: float) -> np.ndarray:
    """Eigenvalues of M = ebar B + tau(S) on the d-dimensional sine basis
    (Lemma le:eig applied to Eqs. (Ha), (q), (tauSalpha)):
    mu_k = ebar prod_i beta^{(i)}_{k_i} + sum_i eta_i q^{(i)}_{k_i} prod_{l!=i} beta^{(l)}_{k_l}."""
    d = prob.d
    betas = [beta_eigs(prob.alpha[i], prob.n[i]) for i in range(d)]
    qs = [tau_eigs_q(fcd_weights(prob.alpha[i], prob.n[i])) for i in range(d)]
    eta = etas(prob)

    def outer(vs):  # vs in dim order 1..d -> array shape (N_d..N_1)
        out = vs[0]
        for v in vs[1:]:
            out = np.multiply.outer(v, out)
        return out

    mu = ebar * outer(betas)
    for i in range(d):
        vs = [qs[l] * eta[i] if l == i else betas[l] for l in range(d)]
        mu = mu + outer(vs)
    return mu.reshape(-1)


def apply_Minv(prob, ebar: float, r: np.ndarray, mu: Optional[np.ndarray] = None) -> np.ndarray:
    """M^{-1} r = S_d diag(1/mu) S_d r with S_d = S ⊗ ... ⊗ S (Eq. (diag); S^2 = I)."""
    if mu is None:
        mu = mu_tensor(prob, ebar)
    X = r.reshape(_shape(prob))
    Ss = [sine_matrix(prob.n[i]) for i in range(prob.d)]
    for i in range(prob.d):
        X = mode_product(X, Ss[i], _axis(prob, i))
    X = X / mu.reshape(_shape(prob))
    for i in range(prob.d):
        X = mode_product(X, Ss[i], _axis(prob, i))
    return X.reshape(-1)


def beta_tensor(prob) -> np.ndarray:
    """Eigenvalues of B_alpha = B_{alpha_d} ⊗ ... ⊗ B_{alpha_1} on the d-dimensional sine basis
    (Lemma le:eig with Lemma Heig): prod_i beta^{(i)}_{k_i}."""
    betas = [beta_eigs(prob.alpha[i], prob.n[i]) for i in range(prob.d)]
    out = betas[0]
    for v in betas[1:]:
        out = np.multiply.outer(v, out)
    return out.reshape(-1)


def apply_sine_diag(prob, r: np.ndarray, dvec: np.ndarray) -> np.ndarray:
    """S_d diag(dvec) S_d r with the orthonormal d-dimensional DST-I S_d (Eq. (diag))."""
    X = r.reshape(_shape(prob))
    Ss = [sine_matrix(prob.n[i]) for i in range(prob.d)]
    for i in range(prob.d):
        X = mode_product(X, Ss[i], _axis(prob, i))
    X = X * dvec.reshape(_shape(prob))
    for i in range(prob.d):
        X = mode_product(X, Ss[i], _axis(prob, i))
    return X.reshape(-1)


def two_sided_structured(prob, e_vec: np.ndarray, b: np.ndarray, ebar: float, tol: float, max_iter: int,
                         u0: Optional[np.ndarray] = None, toeps=None) -> GmresResult:
    """Two-sided τ-preconditioned GMRES (TPGM), Eq. (Pls), with the structured operators.

    P_alpha = ebar I + B^{-1} tau(S) (Eq. (Pa)) is a τ-matrix: on the sine basis its eigenvalues
    are ebar + tau_k / beta_k = mu_k / beta_k (mu_tensor, beta_tensor), so
    P^{-1/2} = S_d diag((beta/mu)^{1/2}) S_d and P^{-1/2} B^{-1} = S_d diag((beta mu)^{-1/2}) S_d.
    GMRES runs on P^{-1/2} Ã P^{-1/2} ũ = P^{-1/2} b̃ with Ã = B^{-1} A, b̃ = B^{-1} b (Eq. (equi)),
    from ũ_0 = P^{1/2} u0 (zero without u0); the returned x is u = P^{-1/2} ũ."""
    mu = mu_tensor(prob, ebar)
    beta = beta_tensor(prob)
    d_pmh = np.sqrt(beta / mu)
    d_pmhb = 1.0 / np.sqrt(beta * mu)
    op = lambda v: apply_sine_diag(prob, apply_A(prob, e_vec, apply_sine_diag(prob, v, d_pmh), toeps), d_pmhb)
    rhs = apply_sine_diag(prob, b, d_pmhb)
    x0 = np.zeros_like(b) if u0 is None else apply_sine_diag(prob, u0, 1.0 / d_pmh)
    res = gmres(op, rhs, x0, tol, max_iter)
    res.x = apply_sine_diag(prob, res.x, d_pmh)
    return res


# --------------------------------------------------------------------------
# fields and right-hand side (Eq. (tls), Appendix A)
# --------------------------------------------------------------------------
def eval_field(prob, tc_row: np.ndarray, space: List[np.ndarray]) -> np.ndarray:
    """g on the padded grid (N_d+2, ..., N_1+2) from separable tables."""
    d = prob.d
    out = 0.0
    for r in range(len(tc_row)):
        term = space[0][r]
        for i in range(1, d):
            term = np.multiply.outer(space[i][r], term)
        out = out + tc_row[r] * term
    return np.asarray(out, dtype=np.float64)


def eval_field_interior(prob, tc_row, space) -> np.ndarray:
    g = eval_field(prob, tc_row, space)
    sl = tuple(slice(1, -1) for _ in range(prob.d))
    return g[sl].reshape(-1)


def rhs_F(prob, f_pad: np.ndarray) -> np.ndarray:
    """F = interior restriction of (𝓗_{alpha_1} ... 𝓗_{alpha_d}) f on the padded grid
    (Eq. (2.2) applied to f; reproduces the 1-D and 2-D forms of Appendix A)."""
    G = f_pad.copy()
    for i in range(prob.d):
        ax = _axis(prob, i)
        a = prob.alpha[i]
        Gm = np.moveaxis(G, ax, 0)
        H = Gm.copy()
        H[1:-1] = (a / 24.0) * Gm[:-2] + (1.0 - a / 12.0) * Gm[1:-1] + (a / 24.0) * Gm[2:]
        G = np.moveaxis(H, 0, ax)
    sl = tuple(slice(1, -1) for _ in range(prob.d))
    return G[sl].reshape(-1)


def rhs_b(prob, e_vec, u, F, toeps=None) -> np.ndarray:
    """b^{(m)} = (B E - S) u^{(m)} + dt F^{(m+1/2)}, Eq. (tls)."""
    return apply_B(prob, e_vec * u) - apply_S(prob, u, toeps) + prob.dt * F


def ebar_from_tables(prob, e_tc: np.ndarray, e_sp) -> tuple:
    """(ebar, ehat, echeck) over the interior grid and all t_{m+1/2}, Eqs. (bard), (dhat)."""
    hi, lo = -np.inf, np.inf
    for m in range(e_tc.shape[0]):
        ev = eval_field_interior(prob, e_tc[m], e_sp)
        hi = max(hi, ev.max())
        lo = min(lo, ev.min())
    return 0.5 * (hi + lo), hi, lo


# --------------------------------------------------------------------------
# GMRES (Lemma Krylov; stopping rule ||r_k|| <= tol ||r_0|| of §4)
# --------------------------------------------------------------------------
@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    res: List[float]           # |g_{j}| estimates, j = 0..iters (preconditioned residual norms)
    hessenberg: np.ndarray = field(default=None)
    basis: np.ndarray = field(default=None)


def gmres(apply_op: Callable, b: np.ndarray, x0: np.ndarray, tol: float, max_iter: int,
          apply_prec: Callable = lambda v: v) -> GmresResult:
    """Left-preconditioned GMRES (Arnoldi with modified Gram-Schmidt, Givens rotations).

    Minimises ||M^{-1}(b - A x)|| over x0 + K_j(M^{-1}A, r_0) (Lemma Krylov) and stops
    at the first j with ||r_j|| <= tol ||r_0|| (§4), or at max_iter.
    """
    n = b.shape[0]
    r0 = apply_prec(b - apply_op(x0))
    beta = float(np.linalg.norm(r0))
    if beta == 0.0:
        return GmresResult(x0.copy(), 0, [0.0])
    V = np.zeros((max_iter + 1, n))
    H = np.zeros((max_iter + 1, max_iter))
    cs = np.zeros(max_iter)
    sn = np.zeros(max_iter)
    g = np.zeros(max_iter + 1)
    g[0] = beta
    V[0] = r0 / beta
    res = [beta]
    k = max_iter
    for j in range(max_iter):
        w = apply_prec(apply_op(V[j]))
        for i in range(j + 1):
            H[i, j] = float(np.dot(w, V[i]))
            w = w - H[i, j] * V[i]
        H[j + 1, j] = float(np.linalg.norm(w))
        # apply the previous rotations to column j
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        rr = math.hypot(H[j, j], H[j + 1, j])
        cs[j] = H[j, j] / rr
        sn[j] = H[j + 1, j] / rr
        H[j, j] = rr
        hj1 = H[j + 1, j]
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        res.append(abs(g[j + 1]))
        if abs(g[j + 1]) <= tol * beta or hj1 == 0.0:
            k = j + 1
            break
        V[j + 1] = w / hj1
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
    x = x0 + V[:k].T @ y
    return GmresResult(x, k, res, H[: k + 1, :k], V[: k + 1])


def gmres_paper_form(prob, e_vec, b, x0, ebar, tol, max_iter) -> GmresResult:
    """GMRES on P^{-1} Ã u = P^{-1} b̃ with Ã = E + B^{-1} S, b̃ = B^{-1} b (Eqs. (equi), (one-sided)),
    dense tier."""
    B = dense_B(prob)
    At = np.diag(e_vec) + np.linalg.solve(B, dense_S(prob))
    bt = np.linalg.solve(B, b)
    P = dense_P(prob, ebar)
    return gmres(lambda v: At @ v, bt, x0, tol, max_iter, lambda v: np.linalg.solve(P, v))


def two_sided_gmres(prob, e_vec, b, ebar, tol, max_iter, u0_tilde=None) -> GmresResult:
    """GMRES on P^{-1/2} Ã P^{-1/2} ũ = P^{-1/2} b̃, Eq. (Pls) (dense tier; P^{-1/2} by eigvalsh).
    Returns the iterate in ũ coordinates."""
    B = dense_B(prob)
    At = np.diag(e_vec) + np.linalg.solve(B, dense_S(prob))
    bt = np.linalg.solve(B, b)
    P = dense_P(prob, ebar)
    Ps = 0.5 * (P + P.T)
    w, Q = np.linalg.eigh(Ps)
    Pmh = (Q * w ** -0.5) @ Q.T
    Abr = Pmh @ At @ Pmh
    x0 = np.zeros_like(b) if u0_tilde is None else u0_tilde
    return gmres(lambda v: Abr @ v, Pmh @ bt, x0, tol, max_iter)


def strang_circulant(t: np.ndarray) -> np.ndarray:
    """First column of the Strang circulant s(T) of the symmetric Toeplitz T with first column t
    (§4, Eq. (Pcir)): the central diagonals of T kept, wrapped around: c_k = t_k for k <= N/2,
    c_k = t_{N-k} otherwise."""
    N = t.shape[0]
    c = np.array(t, dtype=np.float64)
    for k in range(N // 2 + 1, N):
        c[k] = t[N - k]
    return c


def circulant_dense(c: np.ndarray) -> np.ndarray:
    """Dense circulant with first column c: C_{jk} = c_{(j-k) mod N}."""
    N = c.shape[0]
    j = np.arange(N)
    return c[(j[:, None] - j[None, :]) % N]


def _strang_eigs(prob):
    """Per-dimension DFT eigenvalues of s(B_{alpha_i}) and s(S_{alpha_i}) (real: symmetric circulants)."""
    bs, ss = [], []
    for i in range(prob.d):
        n, a = prob.n[i], prob.alpha[i]
        tb = np.zeros(n)
        tb[0] = 1.0 - a / 12.0
        if n > 1:
            tb[1] = a / 24.0
        bs.append(np.fft.fft(strang_circulant(tb)).real)
        ss.append(np.fft.fft(strang_circulant(fcd_weights(a, n))).real)
    return bs, ss


def strang_pc_eigs(prob, ebar: float) -> np.ndarray:
    """Eigenvalues of P_c = ebar I + c(B)^{-1} c(S) (Eq. (Pcir); circulants commute) on the
    d-dimensional Fourier basis, as an array of shape (N_d, ..., N_1)."""
    bs, ss = _strang_eigs(prob)
    eta = etas(prob)

    def outer(vs):
        out = vs[0]
        for v in vs[1:]:
            out = np.multiply.outer(v, out)
        return out

    cb = outer(bs)
    cs = 0.0
    for i in range(prob.d):
        cs = cs + eta[i] * outer([ss[l] if l == i else bs[l] for l in range(prob.d)])
    return ebar + cs / cb


def dense_Pc(prob, ebar: float) -> np.ndarray:
    """P_c = ebar I + c(B)^{-1/2} c(S) c(B)^{-1/2} = ebar I + c(B)^{-1} c(S), assembled densely from
    the Strang circulants of every factor (Eq. (Pcir))."""
    d = prob.d
    sB = [circulant_dense(strang_circulant(np.r_[1.0 - prob.alpha[i] / 12.0, prob.alpha[i] / 24.0,
                                                 np.zeros(max(prob.n[i] - 2, 0))][: prob.n[i]]))
          for i in range(d)]
    sS = [circulant_dense(strang_circulant(fcd_weights(prob.alpha[i], prob.n[i]))) for i in range(d)]
    eta = etas(prob)
    cB = kron_all([sB[i] for i in reversed(range(d))])
    cS = 0.0
    for i in range(d):
        cS = cS + eta[i] * kron_all([sS[l] if l == i else sB[l] for l in reversed(range(d))])
    return ebar * np.eye(cB.shape[0]) + np.linalg.solve(cB, cS)


def apply_Pc_inv(prob, ebar: float, r: np.ndarray, pc: Optional[np.ndarray] = None) -> np.ndarray:
    """P_c^{-1} r by the d-dimensional DFT (numpy FFT as the transform step)."""
    if pc is None:
        pc = strang_pc_eigs(prob, ebar)
    X = np.fft.fftn(r.reshape(_shape(prob)))
    return np.fft.ifftn(X / pc).real.reshape(-1)


def spgm(prob, e_vec: np.ndarray, b: np.ndarray, ebar: float, tol: float, max_iter: int,
         x0: Optional[np.ndarray] = None, toeps=None) -> GmresResult:
    """SPGM (Table 1): GMRES on P_c^{-1} Ã u = P_c^{-1} b̃ with Ã = B^{-1} A, b̃ = B^{-1} b (Eq. (equi)),
    i.e. the one-sided method with the τ preconditioner replaced by the Strang circulant one (the
    reading of "one-sided Strang PGMRES"; B^{-1} by the DST, P_c^{-1} by the DFT)."""
    binv = 1.0 / beta_tensor(prob)
    pc = strang_pc_eigs(prob, ebar)
    op = lambda v: apply_sine_diag(prob, apply_A(prob, e_vec, v, toeps), binv)
    x0 = np.zeros_like(b) if x0 is None else x0
    return gmres(op, apply_sine_diag(prob, b, binv), x0, tol, max_iter, lambda v: apply_Pc_inv(prob, ebar, v, pc))


def numerical_range_bounds(A: np.ndarray, n_angles: int = 720):
    """(v, r) of Eq. (numrag): the distance of the numerical range W(A) from the origin and the
    numerical radius.  W(A) is convex; its support function in the direction e^{-i phi} is the largest
    eigenvalue of the Hermitian part of e^{i phi} A, so r = max_phi lambda_max(H(e^{i phi} A)) and,
    when 0 is not in W(A), v = max_phi lambda_min(H(e^{i phi} A)) (sampled on n_angles angles)."""
    vmax, rmax = -np.inf, 0.0
    for phi in np.linspace(0.0, 2 * np.pi, n_angles, endpoint=False):
        R = np.exp(1j * phi) * A
        w = np.linalg.eigvalsh(0.5 * (R + R.conj().T))
        vmax = max(vmax, float(w[0]))
        rmax = max(rmax, float(w[-1]))
    return vmax, rmax


def spectral_summary(prob, e_vec: np.ndarray, ebar: float) -> dict:
    """Spectral diagnostics of §3 at small N (Figs. 1–3, Theorem GMRES), dense tier: the spread
    max|lambda| / min|lambda| of Ã = E + B^{-1} S and of P^{-1} Ã (Eqs. (equi), (Pa)), and the
    numerical-range angle of Ă = P^{-1/2} Ã P^{-1/2} (Eq. (Pls)): cos(theta) = v / r."""
    B = dense_B(prob)
    At = np.diag(e_vec) + np.linalg.solve(B, dense_S(prob))
    P = dense_P(prob, ebar)
    lam_a = np.linalg.eigvals(At)
    lam_p = np.linalg.eigvals(np.linalg.solve(P, At))
    w, Q = np.linalg.eigh(0.5 * (P + P.T))
    Pmh = (Q * w ** -0.5) @ Q.T
    v, r = numerical_range_bounds(Pmh @ At @ Pmh)
    cos_t = v / r
    return {"spread_A": float(np.abs(lam_a).max() / np.abs(lam_a).min()),
            "spread_PA": float(np.abs(lam_p).max() / np.abs(lam_p).min()),
            "re_PA_min": float(lam_p.real.min()), "re_PA_max": float(lam_p.real.max()),
            "im_PA_absmax": float(np.abs(lam_p.imag).max()),
            "v": v, "r": r, "sin_theta": float(math.sqrt(max(0.0, 1.0 - cos_t * cos_t)))}


def theorem_c(ehat: float, echeck: float) -> float:
    """Rate constant c of Theorem GMRES (§3)."""
    s6 = math.sqrt(6.0)
    e1, e0 = ehat, echeck
    return max(math.sqrt(1 - e0 ** 2 / e1 ** 2),
               math.sqrt(16 * s6 / (4 + s6) ** 2),
               math.sqrt(1 - (e1 + e0) ** 2 * (11 - 4 * s6) / (32 * e1 ** 2)),
               math.sqrt(1 - 32 * e0 ** 2 / ((11 + 4 * s6) * (e1 + e0) ** 2)))


# --------------------------------------------------------------------------
# time marching (Eq. (tls) for m = 0..M-1)
# --------------------------------------------------------------------------
def step_direct(prob, e_vec, b) -> np.ndarray:
    """u^{(m+1)} = A^{-1} b by dense LU: the definition GMRES converges to."""
    return np.linalg.solve(dense_A(prob, e_vec), b)


def l2_error(prob, u, u_exact) -> float:
    """Discrete L2 norm (prod h_i sum_J (u*-u)^2)^{1/2}."""
    hprod = float(np.prod([prob.h(i) for i in range(prob.d)]))
    return math.sqrt(hprod * float(np.sum((u_exact - u) ** 2)))


class OracleSolver:
    """Whole time-march with τ-preconditioned GMRES, structured tier: one-sided in the A-form
    (M = ebar B + tau(S)) or two-sided (Eq. (Pls))."""

    def __init__(self, prob, tables: dict, ebar: Optional[float] = None, sided: int = 1):
        """sided 1: one-sided (OPGM, Eq. (one-sided)); 2: two-sided (TPGM, Eq. (Pls));
        3: the Strang circulant comparison method (SPGM, Table 1).

        tables: separable tables (e_tc, e_sp, f_tc, f_sp, psi_tc, psi_sp), or the fields as grid
        arrays of any form (§1 allows any positive e and any f): "e_dense" of shape (M, n_tot) or
        (n_tot,) for an e that does not depend on t, "f_dense" of shape (M, prod(n_i + 2)) or
        (prod(n_i + 2),) on the padded grid (x_1 fastest) or None for f = 0, and "psi_dense" of
        shape (n_tot,) or None for psi = 0; every value taken at t_{m+1/2} (reading R5)."""
        self.prob = prob
        self.sided = sided
        self.t = tables
        self.dense = "e_dense" in tables
        if ebar is None:
            if self.dense:
                ev = np.asarray(tables["e_dense"])
                ebar = 0.5 * (float(ev.max()) + float(ev.min()))   # Eqs. (bard), (dhat) over all values
            else:
                ebar = ebar_from_tables(prob, tables["e_tc"], tables["e_sp"])[0]
        self.ebar = ebar
        self.toeps = _per_dim(prob, toeplitz_S)
        self.mu = mu_tensor(prob, ebar)
        if self.dense:
            psi = tables.get("psi_dense")
            self.u = np.zeros(prob.n_tot) if psi is None else np.array(psi, dtype=np.float64)
        else:
            self.u = eval_field_interior(prob, tables["psi_tc"][0], tables["psi_sp"])
        self.m = 0
        self.iters: List[int] = []

    def e_at(self, m):
        if self.dense:
            ev = np.asarray(self.t["e_dense"], dtype=np.float64)
            return ev[m] if ev.ndim == 2 else ev
        return eval_field_interior(self.prob, self.t["e_tc"][m], self.t["e_sp"])

    def F_at(self, m):
        if self.dense:
            fv = self.t.get("f_dense")
            if fv is None:
                return np.zeros(self.prob.n_tot)
            fv = np.asarray(fv, dtype=np.float64)
            fm = fv[m] if fv.ndim == 2 else fv
            shape = tuple(self.prob.n[i] + 2 for i in reversed(range(self.prob.d)))
            return rhs_F(self.prob, fm.reshape(shape))
        return rhs_F(self.prob, eval_field(self.prob, self.t["f_tc"][m], self.t["f_sp"]))

    def step(self, direct: bool = False) -> GmresResult | None:
        p = self.prob
        m = self.m
        e = self.e_at(m)
        b = rhs_b(p, e, self.u, self.F_at(m), self.toeps)
        if direct:
            self.u = step_direct(p, e, b)
            self.m += 1
            return None
        x0 = np.zeros_like(b) if p.x0_mode == 0 else self.u.copy()
        if self.sided == 2:
            res = two_sided_structured(p, e, b, self.ebar, p.tol, p.max_iter,
                                       None if p.x0_mode == 0 else x0, self.toeps)
        elif self.sided == 3:
            res = spgm(p, e, b, self.ebar, p.tol, p.max_iter, x0, self.toeps)
        else:
            res = gmres(lambda v: apply_A(p, e, v, self.toeps), b, x0, p.tol, p.max_iter,
                        lambda v: apply_Minv(p, self.ebar, v, self.mu))
        self.u = res.x
        self.iters.append(res.iters)
        self.m += 1
        return res

    def run(self, steps: Optional[int] = None, direct: bool = False):
        steps = self.prob.M - self.m if steps is None else steps
        for _ in range(steps):
            self.step(direct)
        return self.u


def time_march(prob, tables, direct=False, steps=None):
    s = OracleSolver(prob, tables)
    s.run(steps, direct)
    return s
