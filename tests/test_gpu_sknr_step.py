"""One SK-NR iteration (Algorithm 4.1, lines 4-16) on the device against the
oracle's ``newton_step``, element by element, from the same g_k and modes V.

Inputs come from the oracle only: at 512^2 (the Gaussian-mixture recipe of the
benchmark) the oracle's continuation to eps' = 2e-3, its dense modes there
(the sequential warm start of Sec. 5), Sinkhorn at eps = 1e-3 until the L1
marginal error is below 3e-3 (with the D_a Hessian the Newton system is
positive definite only near the optimum), then three iterations, each started
from the oracle's own previous iterate; at 4096^2 (the benchmark's size) the
oracle's SK-NR(30) iterate of the benchmark's continuation early in its last
level (``tests/golden/sknr_state_4096.npz``, written by
``tests/golden/make_sknr_state_4096.py``).  The device rounds V to float32;
the oracle is given the same rounded V.

Tolerances follow the device arithmetic (float32 exponentials and sums,
exponents formed exactly, float64 potentials; tensor-core products in 3xTF32;
a float32 factorisation of the l x l system) and the propagation of each
stage's measured error into the next:
  f_k, h            1e-5 eps (a single transform) and 2e-5 eps (a transform of
                    a transform);
  W                 5e-5 of max |W| (products 2e-5, plus the exponent error of
                    f_k);
  GV, WtDW          1e-5 and 5e-5 of their largest entries;
  grad              the gradient weights d_j = 1 - exp((g_j - h_j)/eps) carry
                    the error of h over eps (<= 2e-5 (1 + |d_j|)), W its own:
                    |d grad| <= 2e-5 sum_j |W_j| (1 + |d_j|) + 5e-5 sum_j |d_j| |W_j|;
  delta             the normwise perturbation bound of a linear solve,
                    kappa (|dA|/|A| + |dgrad|/|grad|) / (1 - kappa |dA|/|A|),
                    with the measured dA (GV - WtDW) and dgrad, plus float32
                    factorisation rounding (kappa 1e-6);
  f', h'            f_k's error plus |V| |d delta| and the float32 correction;
                    h' adds a transform's 1e-5 eps;
  dq                <V delta, a> and <h' - h, b> with the errors above;
  accept            identical wherever |dq| exceeds that bound.
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_2506_14780_gb300 as p
    p.load()
    return p


def _dev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    return (t if dtype is None else t.to(dtype)).cuda()


def _step(pkg, C32, a, b, eps, g, V32, newton_solver=0):
    n, m = C32.shape
    ell = V32.shape[1]
    z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")  # noqa: E731
    out = {"f_k": z(n), "h": z(m), "W": torch.zeros((m, ell), dtype=torch.float32, device="cuda"),
           "grad": z(ell), "GV": torch.zeros((ell, ell), dtype=torch.float64, device="cuda"),
           "WtDW": torch.zeros((ell, ell), dtype=torch.float64, device="cuda"),
           "delta": z(ell), "f_trial": z(n), "h_trial": z(m)}
    st, info = pkg.eot_sknr_step(n, m, ell, _dev(C32), _dev(a), _dev(b), eps, _dev(g), _dev(V32),
                                 newton_solver=newton_solver, **out)
    assert st == pkg.EOT_OK, pkg.last_error()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}, info


def _compare(pkg, C32, a, b, eps, g, V32, newton_solver=0):
    """Run one device step and the oracle's from the same (g, V); assert every
    bound; return the oracle's step (for chaining) and a short report.
    newton_solver 1: both solve the Newton system by conjugate gradients (the
    device in float32 to a relative residual of 1e-6, which bounds its error by
    kappa 1e-6 like the factorisation's rounding; 1e-5 allows for the
    residual's float32 floor)."""
    C = C32.astype(np.float64)
    d, info = _step(pkg, C32, a, b, eps, g, V32, newton_solver)
    f_k = O.c_transform_g(g, C, b, eps)
    o = O.newton_step(f_k, C, a, b, eps, V32, hessian="diag_alpha",
                      newton="cg" if newton_solver else "direct")
    solve_tol = 1e-5 if newton_solver else 1e-6
    rep = {}
    # line 4 and the column transform at f_k
    e_f = np.abs(d["f_k"] - f_k).max()
    e_h = np.abs(d["h"] - o["h"]).max()
    assert e_f <= 1e-5 * eps, e_f / eps
    assert e_h <= 2e-5 * eps, e_h / eps
    dj = -np.expm1((g - o["h"]) / eps)
    col_l1 = float(b @ np.abs(np.expm1((g - o["h"]) / eps)))
    assert abs(info["col_l1"] - col_l1) <= 3e-5 * (1.0 + col_l1), (info["col_l1"], col_l1)
    assert abs(info["q_semi"] - o["q_semi"]) <= 3e-5 * eps
    # products and Gram matrices
    Wo = o["W"]
    e_W = np.abs(d["W"] - Wo).max()
    assert e_W <= 5e-5 * np.abs(Wo).max(), e_W / np.abs(Wo).max()
    e_GV = np.abs(d["GV"] - o["GV"]).max()
    assert e_GV <= 1e-5 * np.abs(o["GV"]).max()
    e_WW = np.abs(d["WtDW"] - o["WtDW"]).max()
    assert e_WW <= 5e-5 * np.abs(o["WtDW"]).max(), e_WW / np.abs(o["WtDW"]).max()
    # gradient on V (the delta form of the device equals V^T (a - pi 1) here)
    aW = np.abs(Wo)
    tol_g = 2e-5 * ((1.0 + np.abs(dj))[:, None] * aW).sum(0) + 5e-5 * (np.abs(dj)[:, None] * aW).sum(0)
    e_g = np.abs(d["grad"] - o["grad"])
    assert np.all(e_g <= tol_g + 1e-15), (e_g / tol_g).max()
    rep.update(e_f=e_f / eps, e_h=e_h / eps, e_W=e_W / np.abs(Wo).max(),
               e_grad=(e_g / np.abs(o["grad"]).max()).max(), col_l1=col_l1)
    # Newton system and step
    A = o["GV"] - o["WtDW"]                          # = -H_V eps
    dA = (d["GV"] - d["WtDW"]) - A
    kappa = np.linalg.cond(0.5 * (A + A.T))
    rA = np.linalg.norm(dA, 2) / np.linalg.norm(A, 2)
    rg = np.linalg.norm(d["grad"] - o["grad"]) / np.linalg.norm(o["grad"])
    assert info["newton_ok"] == (1 if o["ok"] else 0)
    if not o["ok"]:
        return o, rep
    if kappa * rA < 0.5:
        tol_d = kappa * (rA + rg) / (1.0 - kappa * rA) + kappa * solve_tol
        e_d = np.linalg.norm(d["delta"] - o["delta"]) / np.linalg.norm(o["delta"])
        assert e_d <= tol_d, (e_d, tol_d, kappa)
        rep.update(kappa=kappa, e_delta=e_d)
        step_err = np.abs(V32).sum(1).max() * np.abs(d["delta"] - o["delta"]).max()
        corr = np.abs(V32 @ o["delta"]).max()
        e_ft = np.abs(d["f_trial"] - o["f_trial"]).max()
        assert e_ft <= e_f + 1.01 * step_err + 1e-6 * corr + 1e-15, (e_ft, e_f, step_err)
        # <V delta, a> and <h' - h, b> with the errors above
        tol_dq = (np.abs(a @ V32) @ np.abs(d["delta"] - o["delta"])
                  + 2 * (e_ft + 2e-5 * eps) + 2 * e_h + 1e-6 * abs(o["dq_diff"]))
        assert abs(info["dq"] - o["dq_diff"]) <= tol_dq, (info["dq"], o["dq_diff"], tol_dq)
        if abs(o["dq_diff"]) > tol_dq:
            assert info["accepted"] == (1 if o["accepted"] else 0), (info, o["dq"])
        if e_ft <= 1e-3 * eps:
            # the trial transform, where f' itself is close
            assert np.abs(d["h_trial"] - o["h_trial"]).max() <= e_ft + 2e-5 * eps
        rep.update(dq=o["dq_diff"], dq_dev=info["dq"], tol_dq=tol_dq, accepted=o["accepted"])
    return o, rep


def _modes32(V):
    return V.astype(np.float32).astype(np.float64)


def test_sknr_step_matches_oracle_512(pkg):
    prob = W.gaussian_mixture(512, 512, seed=0, eps=1e-3)
    C32 = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32)
    C = C32.astype(np.float64)
    a, b = prob.a, prob.b
    prev = O.continuation(C, a, b, 2e-3, tol=1e-6, eps_start=1e-1, ell=0, level_tol=1e-4)
    V, _ = O.spectral_modes_dense(prev.f, prev.g, C, a, b, 2e-3, 30)
    V32 = _modes32(V)
    eps = 1e-3
    g = O.sinkhorn(C, a, b, eps, tol=3e-3, max_iter=10000, f0=prev.f).g
    accepted = 0
    for k in range(3):
        o, rep = _compare(pkg, C32, a, b, eps, g, V32)
        print(f"512^2 step {k}: {rep}")
        accepted += bool(o["accepted"])
        g = o["h_trial"] if o["ok"] and o["accepted"] else o["h"]
    assert accepted >= 1


def test_sknr_step_conjugate_gradients_512(pkg):
    """The Newton system solved by conjugate gradients on the device
    (newton_solver = 1) against the oracle's newton_cg (Sec. 4 design
    remarks), on the same three iterations as the factorised test."""
    prob = W.gaussian_mixture(512, 512, seed=0, eps=1e-3)
    C32 = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32)
    C = C32.astype(np.float64)
    a, b = prob.a, prob.b
    prev = O.continuation(C, a, b, 2e-3, tol=1e-6, eps_start=1e-1, ell=0, level_tol=1e-4)
    V, _ = O.spectral_modes_dense(prev.f, prev.g, C, a, b, 2e-3, 30)
    V32 = _modes32(V)
    eps = 1e-3
    g = O.sinkhorn(C, a, b, eps, tol=3e-3, max_iter=10000, f0=prev.f).g
    accepted = 0
    for k in range(3):
        o, rep = _compare(pkg, C32, a, b, eps, g, V32, newton_solver=1)
        print(f"512^2 CG step {k}: {rep}")
        accepted += bool(o["accepted"])
        g = o["h_trial"] if o["ok"] and o["accepted"] else o["h"]
    assert accepted >= 1


def test_solve_with_conjugate_gradients(pkg):
    """SK-NR(20) solves with the Newton system by conjugate gradients reach the
    tolerance (the oracle's float64 evaluation) in about as many iterations as
    with the factorisation; an unknown solver is rejected."""
    prob = W.gaussian_mixture(512, 640, seed=21, eps=5e-3)
    C = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32).astype(np.float64)
    out = {}
    for ns in (0, 1):
        f, g, res = pkg.solve(prob, tol=1e-6, max_iter=100000, ell=20, eps_start=1e-1,
                              newton_solver=ns)
        assert res["return_status"] == pkg.EOT_OK, res
        assert O.evaluate(f, g, C, prob.a, prob.b, prob.eps)["l1"] <= 1e-6
        out[ns] = res
    print({ns: (r["total_iters"], r["nr_accepted"], r["nr_rejected"]) for ns, r in out.items()})
    assert out[1]["nr_accepted"] >= 1
    assert out[1]["total_iters"] <= 1.5 * out[0]["total_iters"] + 5, out
    _, _, bad = pkg.solve(prob, tol=1e-6, ell=20, newton_solver=2)
    assert bad["return_status"] == pkg.EOT_EINVAL


def test_sknr_step_matches_oracle_4096(pkg):
    prob = W.gaussian_mixture(4096, 4096, seed=0, eps=1e-3)
    C32 = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32)
    a, b = prob.a, prob.b
    state = np.load(os.path.join(GOLDEN, "sknr_state_4096.npz"))
    eps = float(state["eps"])
    g, V32 = state["g"], state["V"].astype(np.float64)
    o, rep = _compare(pkg, C32, a, b, eps, g, V32)
    print(f"4096^2 step: {rep}")
    assert o["ok"]


def test_sknr_step_rejects_bad_arguments(pkg):
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    c = torch.zeros(16, dtype=torch.float32, device="cuda")
    st, _ = pkg.eot_sknr_step(4, 4, 4, c, x, x, 1e-2, x, x)     # ell must be < n
    assert st == pkg.EOT_EINVAL
    st, _ = pkg.eot_sknr_step(2, 8, 1, c, x, x, 1e-2, x, x)     # n >= 3
    assert st == pkg.EOT_EINVAL
