"""Float64 CPU oracle: log-domain Sinkhorn, SK-NR(l), spectral modes, evaluator.

TEST INFRASTRUCTURE ONLY (see the package docstring): the library never imports
this module.

Paper: "Faster Computation of Entropic Optimal Transport via Stable Low
Frequency Modes" (Chhaibi, Gratton, Vaiter).  Notation follows the paper:
alpha = a (n,), beta = b (m,), cost C (n x m), potentials f (n,), g (m,),
regularisation eps.  Everything is float64; inputs given as float32 are
promoted exactly.

Pins (what fixes each function independently of this file; the tests live in
``tests/test_oracle_*.py``):

* ``sq_euclidean_cost``       brute-force per-entry loop; translation invariance.
* ``sq_euclidean_cost_gram``  the per-entry loop, to float64 cancellation.
* ``c_transform_f`` / ``_g``  separable cost closed form, m = 1 closed form,
                              eps -> infinity limit, permutation equivariance,
                              log-sum-exp against direct summation at safe scales.
* ``sinkhorn`` / ``sknr``     2 x 2 closed form (coupling and SK contraction
                              rate rho_1^2, Lemma 3.2), brute-force OT as
                              eps -> 0, dense direct Newton at tiny n, monotone
                              ascent of the semi-dual (Thm 4.2, step 1).
* ``grad_semi`` / ``hess_semi`` central finite differences of ``q_semi``;
                              H 1 = 0.
* ``newton_cg``               numpy.linalg.solve on SPD systems (exact in k
                              steps up to rounding); breakdown on indefinite
                              ones; SK-NR with it repeats the direct solve.
* ``operator_K`` / ``spectral_modes_*``  Thm 3.1 invariants (spectrum in
                              [-1, 1], symmetric, rho_0 = 1 with eigenvector
                              1 + 1), Hermitization (singular values of R),
                              the semi-dual Hessian identity of App. A.4,
                              subspace iteration (plain and Chebyshev-filtered)
                              against ``numpy.linalg.eigh``.
* ``duality_gap`` / ``evaluate``  a hand-worked 2 x 2 value away from the
                              optimum; primal_value(pi(f,g)) - q_dual(f,g) at
                              random (f, g); zero at the fixed point.

Readings of the paper that this file adopts (each is also recorded in the
design notes of the repository):

* the stopping test uses the L1 norm: ||pi 1 - a||_1 + ||pi^T 1 - b||_1;
* V_l excludes the trivial eigenvector rho_0 = 1 and is orthonormal in L2(alpha);
* the Newton Hessian on V_l is the semi-dual Hessian of Eq. (d2Q_semi); the
  cheaper variant that replaces D_r by D_alpha is selectable (``hessian=``);
* the accept test is strict: Q_semi(f') > Q_semi(f_k); a Hessian that is not
  negative definite on V_l rejects the step;
* the "power method" of Sec. 4 is block subspace iteration with Rayleigh-Ritz,
  deflating the constant mode, started from a SplitMix64 block.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "sq_euclidean_cost", "sq_euclidean_cost_gram", "cost_entries",
    "lse", "c_transform_f", "c_transform_g",
    "plan", "marginals", "marginal_errors",
    "q_dual", "q_semi", "primal_value", "duality_gap", "evaluate", "gauge_normalize",
    "grad_semi", "hess_semi", "hess_dual",
    "op_pi", "op_pi_T", "operator_K", "R_matrix", "semidual_operator_M",
    "splitmix64_uniform", "spectral_modes_dense", "spectral_modes_subspace",
    "spectral_modes_chebyshev", "newton_cg", "newton_step",
    "SolveResult", "sinkhorn", "sknr", "eps_schedule", "continuation",
    "bruteforce_ot", "dense_newton",
]


def _f64(x):
    return np.asarray(x, dtype=np.float64)


# ---------------------------------------------------------------------------
# Cost (Sec. 2: the cost is a matrix C in R_+^{n x m}; Sec. 5 uses the squared
# Euclidean distance between the samples).
# ---------------------------------------------------------------------------

def sq_euclidean_cost(X, Y, normalize: bool = False) -> np.ndarray:
    """C_ij = ||x_i - y_j||^2 in float64, optionally divided by max_ij C_ij."""
    X = _f64(X)
    Y = _f64(Y)
    C = np.zeros((X.shape[0], Y.shape[0]))
    for k in range(X.shape[1]):
        diff = X[:, k][:, None] - Y[:, k][None, :]
        C += diff * diff
    if normalize:
        cmax = C.max()
        if cmax > 0:
            C = C / cmax
    return C


def sq_euclidean_cost_gram(X, Y) -> np.ndarray:
    """C_ij = |x_i|^2 + |y_j|^2 - 2 x_i . y_j in float64, the same cost with
    the cross term as one matrix product (a library routine); for large clouds
    where the per-coordinate loop of ``sq_euclidean_cost`` is slow.  The
    cancellation loses at most a few float64 ulps of |x_i|^2 + |y_j|^2."""
    X = _f64(X)
    Y = _f64(Y)
    return (X * X).sum(axis=1)[:, None] + (Y * Y).sum(axis=1)[None, :] - 2.0 * (X @ Y.T)


def cost_entries(X, Y, rows, cols, scale: float = 1.0) -> np.ndarray:
    """Selected entries ||x_i - y_j||^2 / scale (float64), one by one."""
    X = _f64(X)
    Y = _f64(Y)
    out = np.empty(len(rows))
    for t, (i, j) in enumerate(zip(rows, cols)):
        d = X[i] - Y[j]
        out[t] = float(d @ d) / scale
    return out


# ---------------------------------------------------------------------------
# (C, eps)-transforms, Eq. (foc_f) and Eq. (foc_g).
# ---------------------------------------------------------------------------

def lse(M: np.ndarray, axis: int) -> np.ndarray:
    """log sum exp along ``axis``, shifted by the maximum (exact in real arithmetic)."""
    mx = np.max(M, axis=axis, keepdims=True)
    mx = np.where(np.isfinite(mx), mx, 0.0)
    s = np.sum(np.exp(M - mx), axis=axis, keepdims=True)
    return np.squeeze(mx + np.log(s), axis=axis)


def c_transform_f(f, C, a, eps) -> np.ndarray:
    """f^{C,eps}(y_j) = -eps log sum_i a_i exp((f_i - C_ij)/eps)   (Eq. foc_g)."""
    f, C, a = _f64(f), _f64(C), _f64(a)
    return -eps * lse(np.log(a)[:, None] + (f[:, None] - C) / eps, axis=0)


def c_transform_g(g, C, b, eps) -> np.ndarray:
    """g^{C,eps}(x_i) = -eps log sum_j b_j exp((g_j - C_ij)/eps)   (Eq. foc_f)."""
    g, C, b = _f64(g), _f64(C), _f64(b)
    return -eps * lse(np.log(b)[None, :] + (g[None, :] - C) / eps, axis=1)


# ---------------------------------------------------------------------------
# Coupling, objectives, evaluator (Eq. Optimal_P_epsilon, def_Q, def_Q_semi,
# primal_EOT).
# ---------------------------------------------------------------------------

def plan(f, g, C, a, b, eps) -> np.ndarray:
    """pi_ij = a_i b_j exp((f_i + g_j - C_ij)/eps)   (Eq. Optimal_P_epsilon)."""
    f, g, C, a, b = map(_f64, (f, g, C, a, b))
    return a[:, None] * b[None, :] * np.exp((f[:, None] + g[None, :] - C) / eps)


def marginals(f, g, C, a, b, eps):
    P = plan(f, g, C, a, b, eps)
    return P.sum(axis=1), P.sum(axis=0)


def marginal_errors(f, g, C, a, b, eps):
    """(||pi 1 - a||_1, ||pi^T 1 - b||_1) for pi = pi(f, g)   (Alg. 4.1 stopping test)."""
    r, c = marginals(f, g, C, a, b, eps)
    return float(np.abs(r - _f64(a)).sum()), float(np.abs(c - _f64(b)).sum())


def q_dual(f, g, C, a, b, eps) -> float:
    """Q_eps(f, g) = <f,a> + <g,b> - eps (sum_ij pi_ij - 1)   (Eq. def_Q)."""
    P = plan(f, g, C, a, b, eps)
    return float(_f64(f) @ _f64(a) + _f64(g) @ _f64(b) - eps * (P.sum() - 1.0))


def q_semi(f, C, a, b, eps) -> float:
    """Q_semi(f) = <f,a> + <f^{C,eps}, b>   (Eq. def_Q_semi)."""
    h = c_transform_f(f, C, a, eps)
    return float(_f64(f) @ _f64(a) + h @ _f64(b))


def primal_value(P, C, a, b, eps) -> float:
    """<pi, C> + eps KL(pi || a x b)   (Eq. primal_EOT), for a positive pi."""
    P, C, a, b = map(_f64, (P, C, a, b))
    ref = a[:, None] * b[None, :]
    return float((P * C).sum() + eps * (P * np.log(P / ref)).sum())


def duality_gap(f, g, C, a, b, eps) -> float:
    """<pi 1 - a, f> + <pi^T 1 - b, g> + eps (sum pi - 1), pi = pi(f, g).

    This equals primal_value(pi(f,g)) - q_dual(f,g): with log(pi/(a b)) =
    (f + g - C)/eps, the entropy term cancels <pi, C>.
    """
    r, c = marginals(f, g, C, a, b, eps)
    f, g, a, b = map(_f64, (f, g, a, b))
    return float((r - a) @ f + (c - b) @ g + eps * (r.sum() - 1.0))


def gauge_normalize(f, g, a, b):
    """Shift (f, g) by c (1, -1) (Sec. 2: the dual is invariant) so that <f,a> = <g,b>."""
    f, g = _f64(f).copy(), _f64(g).copy()
    c = 0.5 * (g @ _f64(b) - f @ _f64(a))
    return f + c, g - c


def evaluate(f, g, C, a, b, eps) -> dict:
    """Float64 scores of a pair of potentials: marginal errors, objectives, gap."""
    rl1, cl1 = marginal_errors(f, g, C, a, b, eps)
    return {
        "row_l1": rl1,
        "col_l1": cl1,
        "l1": rl1 + cl1,
        "q_dual": q_dual(f, g, C, a, b, eps),
        "q_semi": q_semi(f, C, a, b, eps),
        "gap": duality_gap(f, g, C, a, b, eps),
    }


# ---------------------------------------------------------------------------
# Derivatives (App. A.1: Eq. dQ, d2Q, dQ_semi, d2Q_semi), Euclidean coordinates.
# ---------------------------------------------------------------------------

def grad_semi(f, C, a, b, eps) -> np.ndarray:
    """dQ_semi(f)/df_i = a_i - sum_j pi_ij with pi = pi(f, f^{C,eps})   (Eq. dQ_semi)."""
    h = c_transform_f(f, C, a, eps)
    P = plan(f, h, C, a, b, eps)
    return _f64(a) - P.sum(axis=1)


def hess_semi(f, C, a, b, eps) -> np.ndarray:
    """Matrix of the quadratic form of Eq. (d2Q_semi):
    -(1/eps) [ diag(pi 1) - pi diag(1/b) pi^T ],  pi = pi(f, f^{C,eps})."""
    h = c_transform_f(f, C, a, eps)
    P = plan(f, h, C, a, b, eps)
    return -(1.0 / eps) * (np.diag(P.sum(axis=1)) - (P / _f64(b)[None, :]) @ P.T)


def hess_dual(f, g, C, a, b, eps) -> np.ndarray:
    """Matrix of Eq. (d2Q) on (f1, g1):  -(1/eps) [[diag(pi 1), pi], [pi^T, diag(pi^T 1)]]."""
    P = plan(f, g, C, a, b, eps)
    n, m = P.shape
    H = np.zeros((n + m, n + m))
    H[:n, :n] = np.diag(P.sum(axis=1))
    H[n:, n:] = np.diag(P.sum(axis=0))
    H[:n, n:] = P
    H[n:, :n] = P.T
    return -(1.0 / eps) * H


# ---------------------------------------------------------------------------
# The operator K_eps (Eq. def_operator_K, def_Op_pi, def_Op_pi_T) and the
# semi-dual Hessian relation (App. A.4, Eq. semidual_Hessian).
# ---------------------------------------------------------------------------

def op_pi(g1, f, g, C, a, b, eps) -> np.ndarray:
    """Op(pi)(g1)(x_i) = sum_j exp((f_i + g_j - C_ij)/eps) g1_j b_j   (Eq. def_Op_pi)."""
    f, g, C, b = map(_f64, (f, g, C, b))
    E = np.exp((f[:, None] + g[None, :] - C) / eps)
    return E @ (_f64(g1) * b[:, None] if np.ndim(g1) == 2 else _f64(g1) * b)


def op_pi_T(f1, f, g, C, a, b, eps) -> np.ndarray:
    """Op(pi)^T(f1)(y_j) = sum_i exp((f_i + g_j - C_ij)/eps) f1_i a_i   (Eq. def_Op_pi_T)."""
    f, g, C, a = map(_f64, (f, g, C, a))
    E = np.exp((f[:, None] + g[None, :] - C) / eps)
    return E.T @ (_f64(f1) * a[:, None] if np.ndim(f1) == 2 else _f64(f1) * a)


def operator_K(f, g, C, a, b, eps) -> np.ndarray:
    """Matrix of K_eps acting on f1 (+) g1 in the Dirac basis (Eq. def_operator_K)."""
    f, g, C, a, b = map(_f64, (f, g, C, a, b))
    E = np.exp((f[:, None] + g[None, :] - C) / eps)
    n, m = E.shape
    K = np.zeros((n + m, n + m))
    K[:n, n:] = E * b[None, :]
    K[n:, :n] = E.T * a[None, :]
    return K


def R_matrix(f, g, C, a, b, eps) -> np.ndarray:
    """R of Eq. (K_form): Op(pi) in orthonormal bases of L2(a) and L2(b),
    R = D_a^{-1/2} pi D_b^{-1/2}."""
    P = plan(f, g, C, a, b, eps)
    return P / np.sqrt(_f64(a))[:, None] / np.sqrt(_f64(b))[None, :]


def semidual_operator_M(f, g, C, a, b, eps) -> np.ndarray:
    """Op(pi) o Op(pi)^T = D_a^{-1} pi D_b^{-1} pi^T (n x n), self-adjoint in L2(a)."""
    P = plan(f, g, C, a, b, eps)
    return (P / _f64(a)[:, None]) @ (P.T / _f64(b)[:, None])


# ---------------------------------------------------------------------------
# Low-frequency modes V_l (Sec. 4: partial eigendecomposition by a power
# method; Eq. semidual_Hessian).
# ---------------------------------------------------------------------------

_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB
_U64 = (1 << 64) - 1


def _splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014)."""
    z = x & _U64
    z = ((z ^ (z >> 30)) * _SM_M1) & _U64
    z = ((z ^ (z >> 27)) * _SM_M2) & _U64
    return z ^ (z >> 31)


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """u_k in [-1, 1): k-th SplitMix64 output of the counter seed + (k+1)*gamma,
    top 53 bits scaled to [0, 1), then mapped to [-1, 1)."""
    out = np.empty(count)
    for k in range(count):
        z = _splitmix64((seed + (k + 1) * _SM_GAMMA) & _U64)
        out[k] = 2.0 * ((z >> 11) * (1.0 / 9007199254740992.0)) - 1.0
    return out


def spectral_modes_dense(f, g, C, a, b, eps, ell: int):
    """Top-l non-trivial eigenpairs of Op(pi) o Op(pi)^T (Eq. semidual_Hessian).

    The symmetric form S = R R^T (R = D_a^{-1/2} pi D_b^{-1/2}) is diagonalised
    by ``numpy.linalg.eigh``; its leading eigenvector sqrt(a) (rho_0 = 1, the
    constant mode of Thm 3.1) is dropped.  Returns (V, rho2) with V = D_a^{-1/2} U
    (n x l, orthonormal in L2(a)) and rho2 = (rho_1^2, ..., rho_l^2).
    """
    R = R_matrix(f, g, C, a, b, eps)
    S = R @ R.T
    w, U = np.linalg.eigh(0.5 * (S + S.T))
    order = np.argsort(w)[::-1]
    w, U = w[order], U[:, order]
    U = U[:, 1:ell + 1]
    V = U / np.sqrt(_f64(a))[:, None]
    return V, w[1:ell + 1].copy()


def _alpha_orthonormalize(Z, a):
    """CholQR2 in L2(a): Z <- Z L^{-T} with L L^T = Z^T D_a Z, applied twice."""
    for _ in range(2):
        G = Z.T @ (a[:, None] * Z)
        L = np.linalg.cholesky(0.5 * (G + G.T))
        Z = np.linalg.solve(L, Z.T).T
    return Z


def spectral_modes_subspace(f, g, C, a, b, eps, ell: int, oversample: int = 10,
                            tol: float = 1e-6, max_iter: int = 200, seed: int = 0,
                            V0: Optional[np.ndarray] = None):
    """Block subspace iteration for the top-l non-trivial modes of
    M = Op(pi) o Op(pi)^T (Eq. semidual_Hessian), in L2(a).

    Each step: deflate the constant mode (a-orthogonal projection), CholQR2 in
    L2(a), apply M = D_a^{-1} pi D_b^{-1} pi^T, Rayleigh-Ritz on Z^T D_a M Z, and
    stop once every one of the first l Ritz pairs has residual
    ||M z - theta z||_a <= tol.  The start block is V0 (if given) completed by
    SplitMix64 columns.  Returns (V, rho2, iterations, max_residual).
    """
    f, g, C, a, b = map(_f64, (f, g, C, a, b))
    n = f.shape[0]
    p = ell + oversample
    Z = splitmix64_uniform(seed, n * p).reshape(n, p)
    if V0 is not None:
        k = min(V0.shape[1], p)
        Z[:, :k] = V0[:, :k]
    P = plan(f, g, C, a, b, eps)
    Pa = P / a[:, None]
    PbT = P.T / b[:, None]
    theta = np.zeros(ell)
    res = np.inf
    it = 0
    Zr = Z[:, :ell]
    for it in range(1, max_iter + 1):
        Z = Z - np.ones((n, 1)) * (a @ Z)[None, :]
        Z = _alpha_orthonormalize(Z, a)
        MZ = Pa @ (PbT @ Z)
        T = Z.T @ (a[:, None] * MZ)
        w, Q = np.linalg.eigh(0.5 * (T + T.T))
        order = np.argsort(w)[::-1]
        w, Q = w[order], Q[:, order]
        Zr, MZr = Z @ Q, MZ @ Q
        R = MZr[:, :ell] - Zr[:, :ell] * w[None, :ell]
        res = float(np.sqrt((a[:, None] * R * R).sum(axis=0)).max())
        theta = w[:ell]
        if res <= tol:
            break
        Z = MZr
    return Zr[:, :ell].copy(), theta.copy(), it, res


def spectral_modes_chebyshev(f, g, C, a, b, eps, ell: int, oversample: int = 10,
                             degree: int = 4, tol: float = 1e-6, max_iter: int = 200,
                             seed: int = 0, V0: Optional[np.ndarray] = None):
    """Chebyshev-filtered block subspace iteration (a faster spectral step for
    eigenvalues rho^2 clustered near 1, Sec. 3): the same deflation, L2(a)
    orthonormalisation, Rayleigh-Ritz and stopping rule as
    ``spectral_modes_subspace``, but between two Rayleigh-Ritz steps the block
    is multiplied by T_d((M - c)/e), the Chebyshev polynomial of the first
    kind of degree d (three-term recurrence T_{k+1} = 2 x T_k - T_{k-1}),
    where [c - e, c + e] = [0, theta_p] covers the spectrum below the block's
    smallest Ritz value theta_p (M is positive semidefinite): that part stays
    bounded by 1 while the wanted eigenvalues above theta_p grow like
    cosh(d arccosh x).  One step costs d applications of M.  Returns (V, rho2,
    steps, max_residual, applications of M)."""
    f, g, C, a, b = map(_f64, (f, g, C, a, b))
    n = f.shape[0]
    p = ell + oversample
    Z = splitmix64_uniform(seed, n * p).reshape(n, p)
    if V0 is not None:
        k = min(V0.shape[1], p)
        Z[:, :k] = V0[:, :k]
    P = plan(f, g, C, a, b, eps)
    Pa = P / a[:, None]
    PbT = P.T / b[:, None]
    ones = np.ones((n, 1))

    def apply_M(Y):
        Y = Y - ones * (a @ Y)[None, :]     # stay orthogonal to the constant mode
        return Pa @ (PbT @ Y)

    applications = 0
    theta = np.zeros(ell)
    res = np.inf
    it = 0
    Zr = Z[:, :ell]
    sa = np.sqrt(a)[:, None]
    for it in range(1, max_iter + 1):
        Z = Z - ones * (a @ Z)[None, :]
        # Householder QR in L2(a): the filtered columns differ in scale by the
        # filter's gain, beyond what a Cholesky-based QR tolerates
        Qh, _ = np.linalg.qr(sa * Z)
        Z = Qh / sa
        MZ = apply_M(Z)
        applications += 1
        T = Z.T @ (a[:, None] * MZ)
        w, Q = np.linalg.eigh(0.5 * (T + T.T))
        order = np.argsort(w)[::-1]
        w, Q = w[order], Q[:, order]
        Zr, MZr = Z @ Q, MZ @ Q
        R = MZr[:, :ell] - Zr[:, :ell] * w[None, :ell]
        res = float(np.sqrt((a[:, None] * R * R).sum(axis=0)).max())
        theta = w[:ell]
        if res <= tol:
            break
        cut = max(float(w[p - 1]), 0.0)
        c = e = 0.5 * cut
        if not e > 0.0:
            Z = MZr
            continue
        # T_1 = (M - c) Z / e from the product already formed, then the recurrence
        Yprev, Y = Zr, (MZr - c * Zr) / e
        for _ in range(degree - 1):
            Ynext = 2.0 * (apply_M(Y) - c * Y) / e - Yprev
            applications += 1
            Yprev, Y = Y, Ynext
        Z = Y
    return Zr[:, :ell].copy(), theta.copy(), it, res, applications


# ---------------------------------------------------------------------------
# Sinkhorn (Eq. SK_iterations) and SK-NR(l) (Algorithm 4.1).
# ---------------------------------------------------------------------------

@dataclass
class SolveResult:
    f: np.ndarray
    g: np.ndarray
    iters: int
    converged: bool
    err_history: list = field(default_factory=list)
    qsemi_history: list = field(default_factory=list)
    nr_accepted: int = 0
    nr_rejected: int = 0


def newton_cg(A, rhs, tol: float = 1e-14, max_iter: Optional[int] = None):
    """Conjugate gradients (Hestenes-Stiefel) for A x = rhs, A symmetric
    (Sec. 4, remarks on the design: the Newton system of the NR step solved
    iteratively, the form that parallelises over many problems).  Stops at a
    relative residual ``tol`` or after ``max_iter`` steps (default 10 k: in
    floating point CG needs more than the k steps of exact arithmetic on an
    ill-conditioned system).  Returns (x, ok): ok is False when a search
    direction has non-positive curvature p^T A p <= 0 (A is not positive
    definite along it), in which case the step is rejected like a failed
    Cholesky factorisation."""
    A, rhs = _f64(A), _f64(rhs)
    k = rhs.shape[0]
    x = np.zeros(k)
    r = rhs.copy()
    p = r.copy()
    rr = float(r @ r)
    stop = tol * tol * max(rr, 1e-300)
    for _ in range(10 * k if max_iter is None else max_iter):
        if rr <= stop:
            break
        Ap = A @ p
        curv = float(p @ Ap)
        if not curv > 0.0:
            return x, False
        alpha = rr / curv
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, True


def newton_step(f, C, a, b, eps, V, hessian: str = "exact", newton: str = "direct") -> dict:
    """The Newton part of one iteration of Algorithm 4.1 at f = f_k (after the
    row half-step), with every intermediate returned:

      h = f_k^{C,eps} (Eq. foc_g) and Q_semi(f_k) = <f_k, a> + <h, b>;
      pi = pi(f_k, h), r = pi 1, W = pi^T V;
      grad = V^T (a - r)                              (Eq. dQ_semi on V);
      GV = V^T D V with D = D_r (exact) or D_a (``diag_alpha``), WtDW = W^T D_b^-1 W,
      H = -(1/eps) [GV - WtDW]                        (Eq. d2Q_semi on V);
      ok = -H positive definite (Cholesky), Delta = (-H)^-1 grad;
      f' = f_k + V Delta, h' = f'^{C,eps}, Q_semi(f') = <f', a> + <h', b>;
      accepted = Q_semi(f') > Q_semi(f_k) (strict), dq = Q_semi(f') - Q_semi(f_k),
      dq_diff = <V Delta, a> + <h' - h, b> (the same difference, summed as one).
    With ``newton="cg"`` Delta comes from ``newton_cg``; ok is then its
    curvature test.  When ok is False the trial entries are None.
    """
    f, C, a, b, V = map(_f64, (f, C, a, b, V))
    h = c_transform_f(f, C, a, eps)
    q_k = float(f @ a + h @ b)
    P = plan(f, h, C, a, b, eps)
    r = P.sum(axis=1)
    grad = V.T @ (a - r)
    W = P.T @ V
    d = r if hessian == "exact" else a
    GV = V.T @ (d[:, None] * V)
    WtDW = W.T @ (W / b[:, None])
    H = -(1.0 / eps) * (GV - WtDW)
    negH = 0.5 * (-H - H.T)
    out = {"h": h, "q_semi": q_k, "r": r, "W": W, "grad": grad, "GV": GV, "WtDW": WtDW,
           "H": H, "ok": True, "delta": None, "f_trial": None, "h_trial": None,
           "q_trial": None, "dq": None, "dq_diff": None, "accepted": False}
    if newton == "cg":
        delta, ok = newton_cg(negH, grad)
        if not ok:
            out["ok"] = False
            return out
    else:
        try:
            np.linalg.cholesky(negH)
        except np.linalg.LinAlgError:
            out["ok"] = False
            return out
        delta = np.linalg.solve(negH, grad)
    step = V @ delta
    f_new = f + step
    h_new = c_transform_f(f_new, C, a, eps)
    q_new = float(f_new @ a + h_new @ b)
    out.update(delta=delta, f_trial=f_new, h_trial=h_new, q_trial=q_new, dq=q_new - q_k,
               dq_diff=float(step @ a + (h_new - h) @ b), accepted=q_new > q_k)
    return out


def sknr(C, a, b, eps, V=None, tol: float = 1e-6, max_iter: int = 10000, f0=None,
         hessian: str = "exact", record: bool = False, newton: str = "direct") -> SolveResult:
    """Algorithm 4.1, SK-NR(l).  With V None (or l = 0) it is log-domain Sinkhorn.

    Iteration k (the algorithm's order):
      g_k = f_{k-1}^{C,eps}; f_k = g_k^{C,eps}        (Eq. SK_iterations)
      stop if ||pi 1 - a||_1 + ||pi^T 1 - b||_1 < tol, pi = pi(f_k, g_k)
      if l > 0: value Q_semi(f_k); gradient and Hessian on V (Eq. dQ_semi,
      d2Q_semi at f_k with g = f_k^{C,eps}); Newton step
      Delta = -(H_V)^{-1} grad_V; f' = f_k + V Delta; keep f' iff
      Q_semi(f') > Q_semi(f_k).
    ``hessian="exact"`` uses D_r with r = pi(f_k, f_k^{C,eps}) 1 (Eq. d2Q_semi);
    ``hessian="diag_alpha"`` replaces D_r by D_a (equal at the optimum).
    ``newton="direct"`` solves for Delta by Cholesky; ``newton="cg"`` by
    conjugate gradients (``newton_cg``), rejecting on non-positive curvature.
    Returns (f_k, g_k) of the stopping iteration.
    """
    C, a, b = _f64(C), _f64(a), _f64(b)
    n, m = C.shape
    f = np.zeros(n) if f0 is None else _f64(f0).copy()
    g = np.zeros(m)
    ell = 0 if V is None else int(V.shape[1])
    V = None if ell == 0 else _f64(V)
    res = SolveResult(f=f, g=g, iters=0, converged=False)
    for k in range(1, max_iter + 1):
        g = c_transform_f(f, C, a, eps)
        f = c_transform_g(g, C, b, eps)
        rl1, cl1 = marginal_errors(f, g, C, a, b, eps)
        err = rl1 + cl1
        res.iters = k
        if record:
            res.err_history.append(err)
        if err < tol:
            res.converged = True
            break
        if ell > 0:
            step = newton_step(f, C, a, b, eps, V, hessian=hessian, newton=newton)
            if not step["ok"]:
                res.nr_rejected += 1
                continue
            if step["accepted"]:
                f = step["f_trial"]
                res.nr_accepted += 1
            else:
                res.nr_rejected += 1
            if record:
                res.qsemi_history.append(q_semi(f, C, a, b, eps))
    res.f, res.g = f, g
    return res


def sinkhorn(C, a, b, eps, tol: float = 1e-6, max_iter: int = 10000, f0=None,
             record: bool = False) -> SolveResult:
    """Log-domain Sinkhorn (Eq. SK_iterations): Algorithm 4.1 with l = 0."""
    return sknr(C, a, b, eps, None, tol=tol, max_iter=max_iter, f0=f0, record=record)


def eps_schedule(eps_start: float, eps: float, factor: float) -> list:
    """Decreasing levels eps_start, eps_start*factor, ... (> eps), then eps itself."""
    if eps_start <= eps or factor <= 0.0 or factor >= 1.0:
        return [float(eps)]
    levels = []
    e = float(eps_start)
    while e > eps * (1.0 + 1e-9):
        levels.append(e)
        e *= factor
    levels.append(float(eps))
    return levels


def continuation(C, a, b, eps, tol: float = 1e-6, eps_start: float = 1e-1,
                 eps_factor: float = 0.5, ell: int = 0, sequential: bool = True,
                 max_iter: int = 100000, level_tol: Optional[float] = None,
                 hessian: str = "exact", modes: str = "dense", oversample: int = 10,
                 eig_tol: float = 1e-6, eig_max_iter: int = 200, seed: int = 0,
                 return_levels: bool = False, newton: str = "direct"):
    """eps-continuation with spectral warm start (Sec. 4 and Sec. 5, Fig. 5.1/5.2).

    Levels come from ``eps_schedule``.  Potentials are carried from level to
    level.  With l > 0 the modes V_l(eps') are computed at the converged
    potentials of a level and used at the next one: refreshed at every level
    (``sequential``) or computed once at the first level (static warm start).
    ``newton`` selects the Newton system's solve in ``sknr`` ("direct" or "cg").
    """
    levels = eps_schedule(eps_start, eps, eps_factor)
    n = np.shape(C)[0]
    f = np.zeros(n)
    V = None
    history = []
    out = None
    for t, e in enumerate(levels):
        last = t == len(levels) - 1
        tl = tol if (last or level_tol is None) else level_tol
        out = sknr(C, a, b, e, V if ell > 0 else None, tol=tl, max_iter=max_iter, f0=f,
                   hessian=hessian, newton=newton)
        history.append({"eps": e, "iters": out.iters, "converged": out.converged,
                        "nr_accepted": out.nr_accepted, "nr_rejected": out.nr_rejected})
        f = out.f
        if ell > 0 and not last and (sequential or V is None):
            if modes == "dense":
                V, _ = spectral_modes_dense(out.f, out.g, C, a, b, e, ell)
            else:
                V, _, _, _ = spectral_modes_subspace(out.f, out.g, C, a, b, e, ell,
                                                     oversample=oversample, tol=eig_tol,
                                                     max_iter=eig_max_iter, seed=seed, V0=V)
    if return_levels:
        return out, history
    return out


# ---------------------------------------------------------------------------
# Independent references used only by the pins.
# ---------------------------------------------------------------------------

def bruteforce_ot(C) -> tuple:
    """Exact OT between two uniform measures of equal size n <= 8 by enumerating
    permutations (Birkhoff: an optimal coupling is a permutation / n)."""
    C = _f64(C)
    n = C.shape[0]
    best, best_perm = math.inf, None
    for perm in itertools.permutations(range(n)):
        v = sum(C[i, perm[i]] for i in range(n)) / n
        if v < best:
            best, best_perm = v, perm
    return best, best_perm


def dense_newton(C, a, b, eps, f0=None, iters: int = 50, tol: float = 1e-13):
    """Full Newton-Raphson on Q_semi (Eq. dQ_semi, d2Q_semi), gauge fixed by
    working on the a-orthogonal complement of the constants, with a
    backtracking ascent guard.  Returns the final f."""
    C, a, b = _f64(C), _f64(a), _f64(b)
    n = C.shape[0]
    f = np.zeros(n) if f0 is None else _f64(f0).copy()
    # basis of {v : <v, a> = 0}
    Bq, _ = np.linalg.qr(np.column_stack([np.ones(n), np.eye(n)[:, :n - 1]]))
    B = Bq[:, 1:]
    B = B - np.ones((n, 1)) * (a @ B)[None, :]
    for _ in range(iters):
        gr = B.T @ grad_semi(f, C, a, b, eps)
        if np.abs(gr).max() < tol:
            break
        H = B.T @ hess_semi(f, C, a, b, eps) @ B
        step = B @ np.linalg.solve(-H, gr)
        q0 = q_semi(f, C, a, b, eps)
        t = 1.0
        while t > 1e-8 and q_semi(f + t * step, C, a, b, eps) < q0:
            t *= 0.5
        f = f + t * step
    return f
