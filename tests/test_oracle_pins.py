"""Pins of the float64 oracle against facts that do not come from the oracle itself:
closed forms, brute force, library routines (numpy eigh / svd), finite
differences and the paper's theorems.  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


def _simplex(rng, k):
    w = rng.random(k) + 0.1
    return w / w.sum()


# --------------------------------------------------------------------------- cost

def test_cost_matches_entrywise_loop():
    rng = _rng(0)
    X = rng.standard_normal((5, 3)).astype(np.float32)
    Y = rng.standard_normal((7, 3)).astype(np.float32)
    C = O.sq_euclidean_cost(X, Y)
    for i in range(5):
        for j in range(7):
            ref = sum((float(X[i, k]) - float(Y[j, k])) ** 2 for k in range(3))
            assert C[i, j] == pytest.approx(ref, rel=1e-14, abs=1e-15)
    Cn = O.sq_euclidean_cost(X, Y, normalize=True)
    assert Cn.max() == pytest.approx(1.0, rel=1e-15)
    assert np.allclose(Cn * C.max(), C, rtol=1e-14)
    t = np.array([0.5, -2.0, 3.0], dtype=np.float32)
    assert np.allclose(O.sq_euclidean_cost(X.astype(np.float64) + t, Y.astype(np.float64) + t), C,
                       rtol=1e-12, atol=1e-12)
    e = O.cost_entries(X, Y, [1, 4], [6, 0])
    assert e[0] == pytest.approx(C[1, 6], rel=1e-14) and e[1] == pytest.approx(C[4, 0], rel=1e-14)


# ------------------------------------------------------------------ c-transforms

def test_c_transform_direct_summation():
    """Eq. (foc_g)/(foc_f) written out with math.exp/math.log at a safe scale."""
    rng = _rng(1)
    n, m, eps = 5, 7, 0.7
    C = rng.random((n, m))
    a, b = _simplex(rng, n), _simplex(rng, m)
    f, g = rng.standard_normal(n), rng.standard_normal(m)
    gt = O.c_transform_f(f, C, a, eps)
    ft = O.c_transform_g(g, C, b, eps)
    for j in range(m):
        s = sum(a[i] * math.exp((f[i] - C[i, j]) / eps) for i in range(n))
        assert gt[j] == pytest.approx(-eps * math.log(s), rel=1e-13, abs=1e-14)
    for i in range(n):
        s = sum(b[j] * math.exp((g[j] - C[i, j]) / eps) for j in range(m))
        assert ft[i] == pytest.approx(-eps * math.log(s), rel=1e-13, abs=1e-14)


def test_c_transform_separable_cost_closed_form():
    """C_ij = u_i + v_j, f = u + c  =>  f^{C,eps} = v - c exactly and pi = a b^T."""
    rng = _rng(2)
    n, m = 9, 13
    u, v = rng.random(n), rng.random(m)
    C = u[:, None] + v[None, :]
    a, b = _simplex(rng, n), _simplex(rng, m)
    for eps in (1e-3, 1e-1, 10.0):
        c = 0.37
        g = O.c_transform_f(u + c, C, a, eps)
        assert np.allclose(g, v - c, rtol=0, atol=1e-12)
        res = O.sinkhorn(C, a, b, eps, tol=1e-12, max_iter=5)
        assert res.iters == 1
        P = O.plan(res.f, res.g, C, a, b, eps)
        assert np.allclose(P, a[:, None] * b[None, :], rtol=1e-10, atol=0)


def test_single_column_closed_form():
    """m = 1: f_i = C_i1 - g, pi_i1 = a_i after one iteration."""
    rng = _rng(3)
    n = 11
    C = rng.random((n, 1))
    a, b = _simplex(rng, n), np.ones(1)
    res = O.sinkhorn(C, a, b, 1e-2, tol=1e-13, max_iter=3)
    assert res.iters == 1
    assert np.allclose(res.f + res.g[0], C[:, 0], atol=1e-13)
    P = O.plan(res.f, res.g, C, a, b, 1e-2)
    assert np.allclose(P[:, 0], a, rtol=1e-12)


def test_large_eps_limit_is_product_coupling():
    """eps -> infinity: the optimal coupling tends to a b^T (error O(1/eps))."""
    rng = _rng(4)
    n, m = 17, 23
    C = rng.random((n, m))
    a, b = _simplex(rng, n), _simplex(rng, m)
    res = O.sinkhorn(C, a, b, 1e6, tol=1e-14, max_iter=50)
    P = O.plan(res.f, res.g, C, a, b, 1e6)
    ab = a[:, None] * b[None, :]
    assert np.abs(P / ab - 1).max() < 5e-6


def test_permutation_equivariance():
    rng = _rng(5)
    n, m, eps = 8, 6, 0.05
    C = rng.random((n, m))
    a, b = _simplex(rng, n), _simplex(rng, m)
    f = rng.standard_normal(n) * 0.1
    p, q = rng.permutation(n), rng.permutation(m)
    g1 = O.c_transform_f(f, C, a, eps)
    g2 = O.c_transform_f(f[p], C[p][:, q], a[p], eps)
    assert np.allclose(g2, g1[q], rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------- 2x2 case

def test_two_by_two_closed_form_and_sk_rate():
    """a = b = (1/2, 1/2): pi = [[p, 1/2-p], [1/2-p, p]] with
    p / (1/2 - p) = exp(-(C11 + C22 - C12 - C21) / (2 eps)); rho_1 = |1 - 4p| is the
    second singular value of R (Hermitization, proof of Thm 3.1) and Lemma 3.2
    gives the SK contraction factor rho_1^2."""
    C = np.array([[0.1, 0.7], [0.5, 0.2]])
    a = b = np.array([0.5, 0.5])
    eps = 0.3
    t = math.exp(-(C[0, 0] + C[1, 1] - C[0, 1] - C[1, 0]) / (2 * eps))
    p = t / (2 * (1 + t))
    res = O.sinkhorn(C, a, b, eps, tol=1e-15, max_iter=1000)
    P = O.plan(res.f, res.g, C, a, b, eps)
    assert np.allclose(P, [[p, 0.5 - p], [0.5 - p, p]], atol=1e-14)
    rho1 = abs(1 - 4 * p)
    _, rho2 = O.spectral_modes_dense(res.f, res.g, C, a, b, eps, 1)
    assert rho2[0] == pytest.approx(rho1 ** 2, rel=1e-10)
    # contraction factor of the SK map on f (modulo constants)
    f = np.array([0.4, -0.3])
    errs = []
    for _ in range(12):
        g = O.c_transform_f(f, C, a, eps)
        f = O.c_transform_g(g, C, b, eps)
        errs.append(abs((f[0] - f[1]) - (res.f[0] - res.f[1])))
    ratios = [errs[k + 1] / errs[k] for k in range(len(errs) - 1) if errs[k + 1] > 1e-12]
    assert ratios[-1] == pytest.approx(rho1 ** 2, rel=1e-3)


# --------------------------------------------------------------- eps -> 0 limit

def test_bruteforce_ot_small_eps():
    """n = m = 6 uniform: W0 (permutation enumeration) <= <pi_eps, C> and
    W0 <= W_eps <= W0 + eps log n; pi_eps -> the optimal permutation / n."""
    rng = _rng(7)
    n = 6
    X, Y = rng.random((n, 2)), rng.random((n, 2))
    C = O.sq_euclidean_cost(X, Y)
    a = b = np.full(n, 1.0 / n)
    w0, perm = O.bruteforce_ot(C)
    # independent check of the enumeration itself
    assert w0 == pytest.approx(min(sum(C[i, s[i]] for i in range(n)) / n
                                   for s in itertools.permutations(range(n))), rel=1e-15)
    Pperm = np.zeros((n, n))
    Pperm[np.arange(n), perm] = 1.0 / n
    prev = None
    # SK-NR with the full a-complement basis (a Newton method) reaches tight
    # marginals at small eps where plain Sinkhorn stalls.
    B = np.eye(n)[:, 1:] - np.ones((n, 1)) * a[1:][None, :]
    for eps in (1e-1, 3e-2, 1e-2, 3e-3, 1e-3):
        res = O.sknr(C, a, b, eps, B, tol=1e-10, max_iter=2000, record=True)
        assert res.err_history[-1] < 1e-9
        P = O.plan(res.f, res.g, C, a, b, eps)
        w_eps = O.primal_value(P, C, a, b, eps)
        assert w0 <= (P * C).sum() + 1e-9
        assert w0 - 1e-9 <= w_eps <= w0 + eps * math.log(n) + 1e-9
        dist = np.abs(P - Pperm).sum()
        if prev is not None:
            assert dist <= prev + 1e-12
        prev = dist
    assert prev < 1e-6


# ------------------------------------------------------------ derivatives / FD

def test_semidual_gradient_and_hessian_finite_differences():
    rng = _rng(8)
    n, m, eps = 7, 9, 0.2
    C = rng.random((n, m))
    a, b = _simplex(rng, n), _simplex(rng, m)
    f = rng.standard_normal(n) * 0.1
    gr = O.grad_semi(f, C, a, b, eps)
    H = O.hess_semi(f, C, a, b, eps)
    h = 1e-5
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd = (O.q_semi(f + e, C, a, b, eps) - O.q_semi(f - e, C, a, b, eps)) / (2 * h)
        assert gr[i] == pytest.approx(fd, abs=1e-8)
        fdg = (O.grad_semi(f + e, C, a, b, eps) - O.grad_semi(f - e, C, a, b, eps)) / (2 * h)
        assert np.allclose(H[:, i], fdg, atol=1e-6)
    assert np.allclose(H @ np.ones(n), 0, atol=1e-12)
    assert abs(gr.sum()) < 1e-13
    assert np.allclose(H, H.T, atol=1e-13)
    assert np.linalg.eigvalsh(H).max() < 1e-12


def test_dual_gradient_finite_differences():
    """Eq. (dQ): the directional derivative of Q_eps, against finite differences."""
    rng = _rng(9)
    n, m, eps = 5, 6, 0.3
    C = rng.random((n, m))
    a, b = _simplex(rng, n), _simplex(rng, m)
    f, g = rng.standard_normal(n) * 0.1, rng.standard_normal(m) * 0.1
    f1, g1 = rng.standard_normal(n), rng.standard_normal(m)
    P = O.plan(f, g, C, a, b, eps)
    dq = f1 @ a + g1 @ b - (P * (f1[:, None] + g1[None, :])).sum()
    h = 1e-6
    fd = (O.q_dual(f + h * f1, g + h * g1, C, a, b, eps)
          - O.q_dual(f - h * f1, g - h * g1, C, a, b, eps)) / (2 * h)
    assert dq == pytest.approx(fd, abs=1e-8)
    Hd = O.hess_dual(f, g, C, a, b, eps)
    x = np.concatenate([f1, g1])
    d2 = -(1 / eps) * (P * (f1[:, None] + g1[None, :]) ** 2).sum()
    assert x @ Hd @ x == pytest.approx(d2, rel=1e-12)


# ---------------------------------------------------------- spectral structure

def _solved(n=30, m=40, eps=0.03, seed=10):
    rng = _rng(seed)
    X, Y = rng.random((n, 2)), rng.random((m, 2))
    C = O.sq_euclidean_cost(X, Y, normalize=True)
    a, b = _simplex(rng, n), _simplex(rng, m)
    res = O.sinkhorn(C, a, b, eps, tol=1e-14, max_iter=200000)
    assert res.converged
    return C, a, b, eps, res.f, res.g


def test_structure_theorem_invariants():
    """Thm 3.1: spectrum of K in [-1, 1], symmetric, rho_0 = 1 with eigenvector
    1 (+) 1; eigenvalues = +- singular values of R (numpy svd); the dual Hessian
    in L2 coordinates is -(1/eps)(Id + K)."""
    C, a, b, eps, f, g = _solved()
    n, m = C.shape
    K = O.operator_K(f, g, C, a, b, eps)
    one = np.ones(n + m)
    assert np.allclose(K @ one, one, atol=1e-11)
    lam = np.sort(np.linalg.eigvals(K).real)
    assert lam.max() == pytest.approx(1.0, abs=1e-10)
    assert lam.min() >= -1 - 1e-10
    k = min(n, m)
    assert np.allclose(lam[:k], -lam[::-1][:k], atol=1e-9)
    s = np.linalg.svd(O.R_matrix(f, g, C, a, b, eps), compute_uv=False)
    assert np.allclose(lam[::-1][:k], s, atol=1e-9)
    D = np.sqrt(np.concatenate([a, b]))
    Hl2 = O.hess_dual(f, g, C, a, b, eps) / D[:, None] / D[None, :]
    Ksym = np.zeros((n + m, n + m))
    R = O.R_matrix(f, g, C, a, b, eps)
    Ksym[:n, n:] = R
    Ksym[n:, :n] = R.T
    assert np.allclose(Hl2, -(1 / eps) * (np.eye(n + m) + Ksym), atol=1e-7)


def test_semidual_hessian_identity():
    """App. A.4 (Eq. semidual_Hessian): at the optimum the semi-dual Hessian is
    -(1/eps)(Id - Op(pi) o Op(pi)^T) in L2(a)."""
    C, a, b, eps, f, g = _solved()
    H = O.hess_semi(f, C, a, b, eps)
    M = O.semidual_operator_M(f, g, C, a, b, eps)
    assert np.allclose(H, -(1 / eps) * (np.diag(a) - a[:, None] * M), atol=1e-8)
    # Op(pi) and Op(pi)^T against the dense operator
    rng = _rng(11)
    g1, f1 = rng.standard_normal(C.shape[1]), rng.standard_normal(C.shape[0])
    Kd = O.operator_K(f, g, C, a, b, eps)
    n = C.shape[0]
    out = Kd @ np.concatenate([f1, g1])
    assert np.allclose(out[:n], O.op_pi(g1, f, g, C, a, b, eps))
    assert np.allclose(out[n:], O.op_pi_T(f1, f, g, C, a, b, eps))


def test_subspace_iteration_matches_eigh():
    C, a, b, eps, f, g = _solved(n=60, m=70, eps=0.05, seed=12)
    ell = 5
    Vd, rd = O.spectral_modes_dense(f, g, C, a, b, eps, ell)
    Vs, rs, it, res = O.spectral_modes_subspace(f, g, C, a, b, eps, ell, oversample=8,
                                                tol=1e-10, max_iter=2000)
    assert res <= 1e-10
    assert np.allclose(rs, rd, atol=1e-9)
    # a-orthonormal, orthogonal to constants, same subspace
    G = Vs.T @ (a[:, None] * Vs)
    assert np.allclose(G, np.eye(ell), atol=1e-10)
    assert np.abs(a @ Vs).max() < 1e-10
    Pd = Vd @ Vd.T @ np.diag(a)
    assert np.allclose(Pd @ Vs, Vs, atol=1e-6)
    assert 0 < rd[-1] <= rd[0] < 1


def test_splitmix64_reference_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as fh:
        vals = [int(line, 16) for line in fh.read().splitlines()
                if line.strip() and not line.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    for k, v in enumerate(vals):
        assert O.eot_oracle._splitmix64(((k + 1) * gamma) & ((1 << 64) - 1)) == v
    u = O.splitmix64_uniform(0, 3)
    assert np.allclose(u, [2 * (v >> 11) / 2.0 ** 53 - 1 for v in vals], rtol=0, atol=0)


# -------------------------------------------------------- rates (Lemma 3.2, Thm 4.2)

def test_sk_and_sknr_rates():
    """Lemma 3.2: SK contracts f - f* by rho_1^2.  Thm 4.2: SK-NR(l) with the
    exact modes V_l(eps) contracts by rho_{l+1}^2."""
    C, a, b, eps, fs, gs = _solved(n=40, m=50, eps=0.02, seed=3)
    V, rho2 = O.spectral_modes_dense(fs, gs, C, a, b, eps, 6)

    def err(f):
        d = f - fs
        d = d - d @ a
        return math.sqrt(a @ d ** 2)

    f = np.zeros(C.shape[0])
    errs = []
    for _ in range(60):
        g = O.c_transform_f(f, C, a, eps)
        f = O.c_transform_g(g, C, b, eps)
        errs.append(err(f))
    assert errs[-1] / errs[-2] == pytest.approx(rho2[0], rel=2e-3)
    for ell in (1, 2):
        f = np.zeros(C.shape[0])
        errs = []
        for _ in range(30):
            f = O.sknr(C, a, b, eps, V[:, :ell], tol=0, max_iter=1, f0=f).f
            errs.append(err(f))
            if errs[-1] < 1e-10:
                break
        assert errs[-1] / errs[-2] == pytest.approx(rho2[ell], rel=1e-2)


def test_sknr_full_basis_is_newton_and_monotone():
    """SK-NR(n-1) with V spanning the a-complement of the constants reaches the
    same optimum as a dense direct Newton solve and as tight Sinkhorn; the
    semi-dual value never decreases along the iterates (Thm 4.2, step 1)."""
    rng = _rng(13)
    n, m, eps = 6, 8, 0.05
    C = O.sq_euclidean_cost(rng.random((n, 2)), rng.random((m, 2)), normalize=True)
    a, b = _simplex(rng, n), _simplex(rng, m)
    sk = O.sinkhorn(C, a, b, eps, tol=1e-14, max_iter=100000)
    fN = O.dense_newton(C, a, b, eps, f0=O.sinkhorn(C, a, b, eps, tol=1e-2).f)
    B = np.eye(n)[:, 1:] - np.ones((n, 1)) * a[1:][None, :]
    f_start = O.sinkhorn(C, a, b, eps, tol=1e-2).f
    res = O.sknr(C, a, b, eps, B, tol=1e-13, max_iter=50, f0=f_start, record=True)
    # inside the basin the full-space Newton step converges quadratically
    assert res.converged and res.iters <= 8
    e = res.err_history
    assert e[-2] < 1e-6 and e[-1] < 1e-13
    for fx in (fN, res.f):
        d = fx - sk.f
        assert np.abs(d - d @ a).max() < 1e-9
    q = res.qsemi_history
    assert all(q[k + 1] >= q[k] - 1e-15 for k in range(len(q) - 1))
    sk2 = O.sinkhorn(C, a, b, eps, tol=1e-12, max_iter=20, record=True)
    qs = []
    f = np.zeros(n)
    for _ in range(20):
        f = O.c_transform_g(O.c_transform_f(f, C, a, eps), C, b, eps)
        qs.append(O.q_semi(f, C, a, b, eps))
    assert all(qs[k + 1] >= qs[k] - 1e-15 for k in range(len(qs) - 1))
    assert len(sk2.err_history) >= 1


def test_gap_vanishes_and_gauge():
    C, a, b, eps, f, g = _solved(n=25, m=35, eps=0.05, seed=14)
    ev = O.evaluate(f, g, C, a, b, eps)
    assert ev["l1"] < 1e-12 and abs(ev["gap"]) < 1e-12
    assert ev["q_dual"] == pytest.approx(ev["q_semi"], abs=1e-12)
    P = O.plan(f, g, C, a, b, eps)
    assert O.primal_value(P, C, a, b, eps) == pytest.approx(ev["q_dual"], abs=1e-12)
    fn, gn = O.gauge_normalize(f + 3.0, g - 3.0, a, b)
    assert fn @ a == pytest.approx(gn @ b, abs=1e-13)
    assert np.allclose(O.plan(fn, gn, C, a, b, eps), P, rtol=1e-10)


def test_duality_gap_by_hand_off_the_optimum():
    """A 2 x 2 pair away from the optimum, worked by hand from Eq. primal_EOT
    and Eq. def_Q.  a = b = (1/2, 1/2), eps = 1, C = [[0, ln 2], [ln 2, 0]],
    f = (0, ln 2), g = 0 give pi = [[1/4, 1/8], [1/4, 1/2]], so pi 1 =
    (3/8, 3/4), pi^T 1 = (1/2, 5/8), sum pi = 9/8, and the gap
    <pi 1 - a, f> + <pi^T 1 - b, g> + eps (sum pi - 1) = ln(2)/4 + 1/8."""
    ln2 = math.log(2.0)
    a = b = np.array([0.5, 0.5])
    C = np.array([[0.0, ln2], [ln2, 0.0]])
    f, g = np.array([0.0, ln2]), np.zeros(2)
    P = O.plan(f, g, C, a, b, 1.0)
    assert np.allclose(P, [[0.25, 0.125], [0.25, 0.5]], rtol=0, atol=1e-15)
    assert O.duality_gap(f, g, C, a, b, 1.0) == pytest.approx(ln2 / 4 + 0.125, rel=1e-14)
    # the same value as the primal value of pi minus the dual value, by hand
    primal = float((P * C).sum() + (P * np.log(P / np.outer(a, b))).sum())
    dual = float(f @ a + g @ b - (P.sum() - 1.0))
    assert primal - dual == pytest.approx(ln2 / 4 + 0.125, rel=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_duality_gap_is_primal_minus_dual_anywhere(seed):
    """At any (f, g), not only at the optimum, the gap equals the primal value
    of pi(f, g) (Eq. primal_EOT, pinned at the optimum against the dual) minus
    Q_eps(f, g) (Eq. def_Q): log(pi / (a b)) = (f + g - C)/eps turns the KL
    term into <pi1, f> + <pi^T 1, g> - <pi, C>.  The value is far from zero
    here, so a sign error or swapped marginal in the gap would show."""
    rng = _rng(100 + seed)
    n, m, eps = 7, 11, 0.3
    C = rng.random((n, m))
    a, b = _simplex(rng, n), _simplex(rng, m)
    f, g = rng.standard_normal(n) * 0.2, rng.standard_normal(m) * 0.2
    P = O.plan(f, g, C, a, b, eps)
    gap = O.duality_gap(f, g, C, a, b, eps)
    assert abs(gap) > 1e-3
    assert gap == pytest.approx(O.primal_value(P, C, a, b, eps) - O.q_dual(f, g, C, a, b, eps),
                                rel=1e-12, abs=1e-14)


def test_eps_schedule():
    lv = O.eps_schedule(1e-1, 1e-3, 0.5)
    assert len(lv) == 8 and lv[0] == 1e-1 and lv[-1] == 1e-3
    assert lv[-2] == pytest.approx(1.5625e-3)
    assert O.eps_schedule(1e-3, 1e-3, 0.5) == [1e-3]


def test_continuation_sknr_beats_sk_iterations():
    """Sec. 5 (qualitative): on a clustered cloud the spectral warm start needs
    far fewer iterations than Sinkhorn at the final eps, same optimum."""
    p = W.gaussian_mixture(160, 160, seed=1)
    C = O.sq_euclidean_cost(p.X, p.Y, normalize=True)
    sk, hs = O.continuation(C, p.a, p.b, 2e-3, tol=1e-8, eps_start=1e-1, ell=0,
                            return_levels=True)
    nr, hn = O.continuation(C, p.a, p.b, 2e-3, tol=1e-8, eps_start=1e-1, ell=20,
                            return_levels=True)
    assert hn[-1]["iters"] * 4 < hs[-1]["iters"]
    f1, g1 = O.gauge_normalize(sk.f, sk.g, p.a, p.b)
    f2, g2 = O.gauge_normalize(nr.f, nr.g, p.a, p.b)
    assert np.abs(f1 - f2).max() < 1e-5 * 2e-3 * 1e3


def test_transposed_problem_has_the_transposed_coupling():
    """Sinkhorn is symmetric in the two sides (Eq. foc_f / foc_g): the problem
    (C^T, b, a) has the coupling pi^T and the potentials (g, f) up to the gauge.
    The batched solver runs problems with more rows than columns this way."""
    p = W.gaussian_mixture(60, 45, seed=3, eps=5e-2)
    C = O.sq_euclidean_cost(p.X, p.Y, normalize=True)
    r1 = O.sinkhorn(C, p.a, p.b, p.eps, tol=1e-13, max_iter=200000)
    r2 = O.sinkhorn(C.T, p.b, p.a, p.eps, tol=1e-13, max_iter=200000)
    P1 = O.plan(r1.f, r1.g, C, p.a, p.b, p.eps)
    P2 = O.plan(r2.f, r2.g, C.T, p.b, p.a, p.eps)
    assert np.abs(P1 - P2.T).max() <= 1e-12
    f1, g1 = O.gauge_normalize(r1.f, r1.g, p.a, p.b)
    g2, f2 = O.gauge_normalize(r2.f, r2.g, p.b, p.a)
    assert np.abs(f1 - f2).max() <= 1e-9 * p.eps and np.abs(g1 - g2).max() <= 1e-9 * p.eps


def test_rounded_inverse_eps_solves_a_nearby_problem():
    """A float32 iteration forms every exponent as (f + g + eps log w - C) k2 with
    k2 = 1/(eps ln 2) rounded, k2 = (1 + d)/(eps ln 2): it iterates Sinkhorn for
    the weights w^(1+d) at eps' = eps/(1 + d).  At eps the row marginals of its
    pair are off by d times the entropy of each row's conditional coupling (to
    first order in d), and the columns by the same total: the size of the error
    that the iteration's own test cannot see."""
    p = W.uniform_square(120, 90, seed=3, eps=2e-2)
    C = O.sq_euclidean_cost(p.X, p.Y, normalize=True)
    eps, d = 2e-2, 1e-5
    a2, b2 = p.a ** (1 + d), p.b ** (1 + d)
    # the raised weights do not balance (sum a^(1+d) != sum b^(1+d)): the
    # iteration settles to the balance error, far below what is measured here
    r = O.sinkhorn(C, a2, b2, eps / (1 + d), tol=1e-11, max_iter=3000)
    ev = O.evaluate(r.f, r.g, C, p.a, p.b, eps)
    P = O.plan(r.f, r.g, C, a2, b2, eps / (1 + d))
    rows = P / P.sum(1, keepdims=True)
    H = -(rows * np.log(np.where(rows > 0, rows, 1.0))).sum(1)
    pred = d * (p.a @ H)
    assert abs(ev["row_l1"] - pred) <= 1e-3 * pred
    assert abs(ev["col_l1"] - ev["row_l1"]) <= 1e-3 * pred


def test_newton_cg_matches_direct_solve():
    """The iterative Newton solve (Sec. 4, remarks on the design) against
    numpy.linalg.solve on SPD systems of the projected Hessian's size (to the
    conditioning times the residual tolerance), and a breakdown (step
    rejected) on an indefinite one, like a failed Cholesky factorisation."""
    rng = np.random.default_rng(11)
    for k in (1, 5, 30, 40):
        Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
        lam = np.geomspace(1.0, 1e-4, k)             # condition number 1e4
        A = (Q * lam) @ Q.T
        rhs = rng.standard_normal(k)
        x, ok = O.newton_cg(A, rhs)
        xd = np.linalg.solve(A, rhs)
        assert ok and np.abs(x - xd).max() <= 1e-8 * np.abs(xd).max()
    A = np.diag([1.0, 2.0, -0.5])
    _, ok = O.newton_cg(A, np.array([1.0, 1.0, 1.0]))
    assert not ok


def test_sknr_with_cg_repeats_the_direct_newton():
    """SK-NR(l) with the Newton system solved by conjugate gradients takes the
    same steps as with the direct solve: same iterations, same accepted and
    rejected steps, the same potentials to rounding.  The tolerance stops the
    run while the semi-dual increase of a step is still well above the float64
    rounding of Q_semi: on this instance it falls to one unit in the last place
    of Q_semi (3e-18) near L1 = 5e-7, where the strict accept test of
    Algorithm 4.1 is decided by rounding whichever way Delta is computed."""
    p = W.gaussian_mixture(150, 130, seed=4)
    C = O.sq_euclidean_cost(p.X, p.Y, normalize=True)
    eps = 5e-3
    start = O.sinkhorn(C, p.a, p.b, 2 * eps, tol=1e-8, max_iter=100000)
    V, _ = O.spectral_modes_dense(start.f, start.g, C, p.a, p.b, 2 * eps, 12)
    r1 = O.sknr(C, p.a, p.b, eps, V, tol=2e-6, max_iter=20000, f0=start.f, hessian="diag_alpha")
    r2 = O.sknr(C, p.a, p.b, eps, V, tol=2e-6, max_iter=20000, f0=start.f, hessian="diag_alpha",
                newton="cg")
    assert r1.converged and r2.converged
    assert (r1.iters, r1.nr_accepted, r1.nr_rejected) == (r2.iters, r2.nr_accepted, r2.nr_rejected)
    assert np.abs(r1.f - r2.f).max() <= 1e-9 * eps


def test_static_mode_continuation_with_cg():
    """The protocol of SK-NR over many problems: modes computed once, at the
    first level (Sec. 5's static warm start), and the Newton system solved by
    conjugate gradients (Sec. 4 design remarks) -- the continuation repeats
    the direct solve's levels step for step (iterations, accepted and rejected
    steps) and ends at the same potentials to rounding."""
    p = W.gaussian_mixture(120, 110, seed=8)
    C = O.sq_euclidean_cost(p.X, p.Y, normalize=True)
    kw = dict(tol=2e-6, eps_start=4e-2, ell=10, sequential=False, hessian="diag_alpha",
              level_tol=1e-4, return_levels=True)
    r1, h1 = O.continuation(C, p.a, p.b, 5e-3, **kw)
    r2, h2 = O.continuation(C, p.a, p.b, 5e-3, newton="cg", **kw)
    steps = lambda h: [(x["iters"], x["nr_accepted"], x["nr_rejected"]) for x in h]  # noqa: E731
    assert steps(h1) == steps(h2), (steps(h1), steps(h2))
    assert sum(x["nr_accepted"] for x in h1) >= 1
    assert r1.converged and np.abs(r1.f - r2.f).max() <= 1e-9 * 5e-3


def test_chebyshev_filtered_subspace_iteration():
    """The Chebyshev-filtered spectral step against numpy.linalg.eigh (same
    Ritz values and subspace as the dense eigendecomposition), and its reason
    to exist: on a clustered spectrum (rho_1^2 near 1) it reaches the same
    residual with fewer applications of M and far fewer Rayleigh-Ritz steps
    than plain subspace iteration."""
    C, a, b, eps, f, g = _solved(n=60, m=70, eps=0.05, seed=12)
    ell = 5
    Vd, rd = O.spectral_modes_dense(f, g, C, a, b, eps, ell)
    Vc, rc, steps, res, apps = O.spectral_modes_chebyshev(f, g, C, a, b, eps, ell, oversample=8,
                                                          degree=4, tol=1e-10, max_iter=2000)
    assert res <= 1e-10 and np.allclose(rc, rd, atol=1e-9)
    assert np.allclose(Vc.T @ (a[:, None] * Vc), np.eye(ell), atol=1e-10)
    assert np.abs(a @ Vc).max() < 1e-10
    Pd = Vd @ Vd.T @ np.diag(a)
    assert np.allclose(Pd @ Vc, Vc, atol=1e-6)
    p = W.gaussian_mixture(200, 180, seed=1, eps=5e-3)
    C2 = O.sq_euclidean_cost(p.X, p.Y, normalize=True)
    r = O.sinkhorn(C2, p.a, p.b, p.eps, tol=1e-10, max_iter=400000)
    _, rho2 = O.spectral_modes_dense(r.f, r.g, C2, p.a, p.b, p.eps, 10)
    assert rho2[0] > 0.99
    _, r_s, it_s, res_s = O.spectral_modes_subspace(r.f, r.g, C2, p.a, p.b, p.eps, 10,
                                                    oversample=10, tol=1e-8, max_iter=20000)
    _, r_c, st_c, res_c, apps_c = O.spectral_modes_chebyshev(r.f, r.g, C2, p.a, p.b, p.eps, 10,
                                                             oversample=10, degree=4, tol=1e-8,
                                                             max_iter=20000)
    assert res_s <= 1e-8 and res_c <= 1e-8
    assert np.abs(r_c - rho2).max() <= 1e-8 and np.abs(r_s - rho2).max() <= 1e-8
    assert apps_c < it_s and 3 * st_c < it_s


def test_spectrum_concentrates_as_eps_decreases():
    """Sec. 3, spectral stability (the paper's figure of the ten smallest
    eigenvalues of Id + K_eps, square against annulus): as eps decreases every
    one of the ten leading rho_k^2 grows towards 1, while the leading
    eigenvectors move little."""
    p = W.square_annulus(160, 160, seed=0)
    C = O.sq_euclidean_cost(p.X, p.Y)
    rho, modes = [], []
    for eps in (0.256, 0.128, 0.064, 0.032, 0.016):
        s = O.sinkhorn(C, p.a, p.b, eps, tol=1e-11, max_iter=200000)
        V, rho2 = O.spectral_modes_dense(s.f, s.g, C, p.a, p.b, eps, 10)
        rho.append(rho2)
        modes.append(V)
    rho = np.array(rho)
    assert np.all(np.diff(rho, axis=0) > 0)          # each rho_k^2 grows as eps halves
    assert rho[-1, 0] > 0.9 and rho[0, 0] < 0.5
    sa = np.sqrt(p.a)[:, None]
    Qu, _ = np.linalg.qr(sa * modes[0][:, :3])
    Qv, _ = np.linalg.qr(sa * modes[2][:, :3])
    # smallest cosine of the principal angles between the leading 3-mode
    # subspaces at eps = 0.256 and eps = 0.064
    assert np.linalg.svd(Qu.T @ Qv, compute_uv=False).min() > 0.95


def test_two_gaussians_protocols_of_section_5():
    """Sec. 5, the 2-D Gaussian experiment (n = 200 against 2n = 400 points,
    uniform weights, raw squared Euclidean cost), its three protocols in
    float64: (1) sequential warm start from eps = 1, halving: with l = 10 modes
    refreshed at every level, every level after the first needs at least 2x
    fewer iterations than Sinkhorn's; (2) static modes computed once at
    eps' = 1: still fewer iterations than Sinkhorn on the first transitions;
    (3) more modes, fewer iterations: at eps = 0.25 from the eps = 1 solution
    with its modes, the count falls strictly with l in {0, 2, 5, 10, 20}."""
    p = W.gaussians_2d(200, seed=0)
    C = O.sq_euclidean_cost(p.X, p.Y)
    _, hs = O.continuation(C, p.a, p.b, 0.25, tol=1e-6, eps_start=1.0, ell=0, return_levels=True)
    _, hn = O.continuation(C, p.a, p.b, 0.25, tol=1e-6, eps_start=1.0, ell=10, return_levels=True)
    _, hst = O.continuation(C, p.a, p.b, 0.25, tol=1e-6, eps_start=1.0, ell=10, sequential=False,
                            return_levels=True)
    sk = [h["iters"] for h in hs]
    seq = [h["iters"] for h in hn]
    static = [h["iters"] for h in hst]
    assert seq[0] == sk[0] == static[0]              # the first level has no modes yet
    assert all(2 * q <= s for q, s in zip(seq[1:], sk[1:])), (seq, sk)
    assert all(q < s for q, s in zip(static[1:], sk[1:])), (static, sk)
    s1 = O.sinkhorn(C, p.a, p.b, 1.0, tol=1e-10, max_iter=100000)
    counts = []
    for ell in (0, 2, 5, 10, 20):
        V = None
        if ell:
            V, _ = O.spectral_modes_dense(s1.f, s1.g, C, p.a, p.b, 1.0, ell)
        counts.append(O.sknr(C, p.a, p.b, 0.25, V, tol=1e-6, max_iter=200000, f0=s1.f).iters)
    assert all(b < a for a, b in zip(counts, counts[1:])), counts


def test_gradient_on_modes_delta_form():
    """The device forms the semi-dual gradient on V (Eq. dQ_semi at f_k, with
    g = h = f_k^{C,eps}) as -sum_j d_j W_j, W = pi(f_k, h)^T V and
    d_j = 1 - exp((g_j - h_j)/eps).  Since V^T a = V^T pi(f_k, g_k) 1 when the
    rows of pi(f_k, g_k) sum to a (after the row half-step f_k = g_k^{C,eps}),
    this equals V^T (a - pi(f_k, h) 1) exactly; it does not when the rows do
    not match."""
    C, a, b, eps, f_opt, g_opt = _solved(n=70, m=50, eps=0.05, seed=21)
    V, _ = O.spectral_modes_dense(f_opt, g_opt, C, a, b, eps, 6)
    rng = np.random.default_rng(2)
    g = g_opt + 0.3 * eps * rng.standard_normal(b.shape)     # an iterate away from the optimum
    f = O.c_transform_g(g, C, b, eps)                         # row half-step: rows of pi(f, g) = a
    h = O.c_transform_f(f, C, a, eps)
    P = O.plan(f, h, C, a, b, eps)
    grad = V.T @ (a - P.sum(axis=1))
    W = P.T @ V
    d = 1.0 - np.exp((g - h) / eps)
    delta_form = -(d[:, None] * W).sum(axis=0)
    assert np.abs(grad - delta_form).max() <= 1e-12 * max(1.0, np.abs(grad).max())
    assert np.abs(grad).max() > 1e-6                          # a non-trivial gradient
    f_off = f + 0.1 * eps * rng.standard_normal(a.shape)      # rows no longer match a
    h2 = O.c_transform_f(f_off, C, a, eps)
    P2 = O.plan(f_off, h2, C, a, b, eps)
    d2 = 1.0 - np.exp((g - h2) / eps)
    assert np.abs(V.T @ (a - P2.sum(axis=1)) + (d2[:, None] * (P2.T @ V)).sum(axis=0)).max() > 1e-6


def test_diag_alpha_hessian_equals_exact_at_the_optimum():
    """Reading R6: the device's projected Hessian replaces D_r, r = pi(f, h) 1
    (Eq. d2Q_semi), by D_a.  At the optimum r = a, so both agree on V; away
    from it they differ by V^T diag(r - a) V / eps."""
    C, a, b, eps, f_opt, g_opt = _solved(n=60, m=45, eps=0.05, seed=8)
    V, _ = O.spectral_modes_dense(f_opt, g_opt, C, a, b, eps, 5)

    def h_diag_alpha(f):
        h = O.c_transform_f(f, C, a, eps)
        W = O.plan(f, h, C, a, b, eps).T @ V
        return -(1.0 / eps) * (V.T @ (a[:, None] * V) - W.T @ (W / b[:, None]))

    exact = V.T @ O.hess_semi(f_opt, C, a, b, eps) @ V
    assert np.abs(exact - h_diag_alpha(f_opt)).max() <= 1e-8 * np.abs(exact).max()
    f = f_opt + 0.5 * eps * np.random.default_rng(1).standard_normal(a.shape)
    h = O.c_transform_f(f, C, a, eps)
    r = O.plan(f, h, C, a, b, eps).sum(axis=1)
    diff = V.T @ O.hess_semi(f, C, a, b, eps) @ V - h_diag_alpha(f)
    assert np.allclose(diff, -(1.0 / eps) * V.T @ ((r - a)[:, None] * V), atol=1e-10)
    assert np.abs(diff).max() > 1e-4


def test_newton_step_intermediates():
    """The Newton part of Algorithm 4.1 (``newton_step``): its gradient and
    Hessian on V are the full semi-dual gradient and Hessian (pinned by finite
    differences above) restricted to V; Delta solves the Newton system; the
    two forms of the objective change agree; the exact Hessian's step
    increases Q_semi here."""
    rng = _rng(31)
    n, m, eps, ell = 12, 15, 0.1, 4
    C = rng.random((n, m))
    a, b = _simplex(rng, n), _simplex(rng, m)
    g = rng.standard_normal(m) * 0.05
    f = O.c_transform_g(g, C, b, eps)
    V = rng.standard_normal((n, ell))
    st = O.newton_step(f, C, a, b, eps, V, hessian="exact")
    Vg = V.T @ O.grad_semi(f, C, a, b, eps)
    VHV = V.T @ O.hess_semi(f, C, a, b, eps) @ V
    assert np.allclose(st["grad"], Vg, rtol=1e-12, atol=1e-14)
    assert np.allclose(st["H"], VHV, rtol=1e-10, atol=1e-12)
    assert st["ok"]
    assert np.allclose(-st["H"] @ st["delta"], st["grad"], rtol=1e-10, atol=1e-13)
    assert np.allclose(st["f_trial"], f + V @ st["delta"], rtol=0, atol=1e-15)
    assert st["dq"] == pytest.approx(st["dq_diff"], rel=1e-9, abs=1e-15)
    assert st["accepted"] and st["dq"] > 0
    # the D_a variant differs by V^T diag(r - a) V / eps
    sa = O.newton_step(f, C, a, b, eps, V, hessian="diag_alpha")
    r = O.plan(f, st["h"], C, a, b, eps).sum(axis=1)
    assert np.allclose(sa["H"] - st["H"], -(V.T @ ((a - r)[:, None] * V)) / eps, rtol=1e-9,
                       atol=1e-12)


def test_gram_form_of_the_cost_matches_entrywise_loop():
    """|x|^2 + |y|^2 - 2 x.y (one matrix product) against ||x - y||^2 entry by
    entry, for the on-the-fly workload's clouds (N(0, I)/8 in R^64)."""
    prob = W.gaussian_cloud(40, 50, d=64, seed=3)
    Cg = O.sq_euclidean_cost_gram(prob.X, prob.Y)
    for i in range(0, 40, 7):
        for j in range(0, 50, 9):
            d = prob.X[i].astype(np.float64) - prob.Y[j].astype(np.float64)
            assert Cg[i, j] == pytest.approx(float(d @ d), rel=0, abs=1e-14)


def test_plan_is_the_derivative_of_the_optimal_value_in_the_cost():
    """Envelope theorem (Eq. def_Q at the optimum): the optimal value of the
    entropic dual as a function of the cost has d/dC_ij = pi_ij, the coupling
    of the optimal potentials.  Central differences of the converged value
    against the plan, entry by entry, on a small random problem."""
    rng = np.random.default_rng(21)
    n, m, eps = 6, 5, 0.3
    C = rng.random((n, m))
    a = rng.random(n) + 0.2
    a /= a.sum()
    b = rng.random(m) + 0.2
    b /= b.sum()

    def value(Cc):
        r = O.sinkhorn(Cc, a, b, eps, tol=1e-15, max_iter=100000)
        return O.q_dual(r.f, r.g, Cc, a, b, eps), r

    _, r = value(C)
    P = O.plan(r.f, r.g, C, a, b, eps)
    h = 1e-5
    for i, j in [(0, 0), (2, 3), (5, 4), (3, 1)]:
        Cp, Cm = C.copy(), C.copy()
        Cp[i, j] += h
        Cm[i, j] -= h
        d = (value(Cp)[0] - value(Cm)[0]) / (2 * h)
        assert abs(d - P[i, j]) < 1e-8, (i, j, d, P[i, j])
    # the primal value at the optimum equals the dual one (zero gap)
    assert abs(O.primal_value(P, C, a, b, eps) - O.q_dual(r.f, r.g, C, a, b, eps)) < 1e-12
