"""The stall check of a continuation level (eot_options.stall_window).

A tolerance far below what the float32 passes can reach makes the L1 marginal
error stop falling at the rounding floor; with the check the level stops at the
next checkpoint that finds less than a 1% gain over one window (status
EOT_NOT_CONVERGED, result.stalled = 1) instead of running to max_iter, and the
returned pair is the floor's, scored by the float64 oracle.  Covered: the
graph-driven and cooperative Sinkhorn loops, the SK-NR loop and the persistent
batch.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WINDOW = 200
CAP = 50000


@pytest.fixture(scope="module")
def pkg():
    import paper_2506_14780_gb300 as p
    p.load()
    return p


def _cost(p):
    return O.sq_euclidean_cost(p.X, p.Y, normalize=True).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("n,m,ell", [(512, 640, 0), (4096, 4096, 0), (700, 900, 10)])
def test_unreachable_tolerance_stops_on_stall(pkg, n, m, ell):
    p = W.gaussian_mixture(n, m, seed=3, eps=0.05)
    f, g, res = pkg.solve(p, tol=1e-12, max_iter=CAP, ell=ell, stall_window=WINDOW)
    assert res["return_status"] == pkg.EOT_NOT_CONVERGED, res
    assert res["stalled"] == 1, res
    # stopped within a few windows of the floor, far below the cap
    assert WINDOW <= res["iters"] <= 20 * WINDOW, res
    ev = O.evaluate(f, g, _cost(p), p.a, p.b, p.eps)
    assert ev["l1"] < 1e-5, ev
    assert abs(ev["l1"] - res["l1_marginal"]) <= 1e-6 + 0.1 * ev["l1"], (ev["l1"], res)
    # a solve that reaches its tolerance never reports a stall
    f2, g2, r2 = pkg.solve(p, tol=1e-5, max_iter=CAP, ell=ell, stall_window=WINDOW)
    assert r2["return_status"] == pkg.EOT_OK and r2["stalled"] == 0, r2


@pytest.mark.parametrize("n,m", [(512, 640), (4096, 4096)])
def test_without_the_check_the_level_runs_to_max_iter(pkg, n, m):
    p = W.gaussian_mixture(n, m, seed=3, eps=0.05)
    f, g, res = pkg.solve(p, tol=1e-12, max_iter=3000, stall_window=0)
    assert res["return_status"] == pkg.EOT_NOT_CONVERGED, res
    assert res["stalled"] == 0 and res["iters"] == 3000, res


def test_negative_window_is_rejected(pkg):
    p = W.gaussian_mixture(64, 64, seed=0, eps=0.05)
    _, _, res = pkg.solve(p, tol=1e-6, stall_window=-1)
    assert res["return_status"] == pkg.EOT_EINVAL, res


def test_batch_members_stop_on_stall(pkg):
    probs = W.batch_problems(count=6, seed=7, n_lo=200, n_hi=900, eps_lo=0.02, eps_hi=0.1)
    keep = []
    cp = [pkg.make_problem(q.a, q.b, X=q.X, Y=q.Y, eps=q.eps, normalize_cost=True, keep=keep)
          for q in probs]
    fo = [np.zeros(q.a.shape[0]) for q in probs]
    go = [np.zeros(q.b.shape[0]) for q in probs]
    st, rs = pkg.eot_solve_batch(cp, pkg.default_options(tol=1e-12, max_iter=CAP,
                                                         stall_window=WINDOW), fo, go)
    assert st in (pkg.EOT_OK, pkg.EOT_NOT_CONVERGED)
    for q, f, g, r in zip(probs, fo, go, rs):
        assert r.status == pkg.EOT_NOT_CONVERGED and r.stalled == 1, r.as_dict()
        assert r.iters <= 20 * WINDOW, r.as_dict()
        assert O.evaluate(f, g, _cost(q), q.a, q.b, q.eps)["l1"] < 1e-5


def test_sknr_on_an_unaligned_cost_pitch_reaches_tol(pkg):
    """m = 15482: the cost rows are not 16-byte aligned, so the SK-NR column
    pass runs its non-TMA variant over segments of thousands of rows; its
    column sums are compensated, so the L1 test reaches 1e-6 about as soon as
    Sinkhorn's does (an uncompensated float32 sum floored the estimate above
    the tolerance and the level ran to its stall check)."""
    p = W.gaussian_cloud(12511, 15482, d=64, seed=11, eps=1e-2)
    p.normalize_cost = True
    _, _, sk = pkg.solve(p, tol=1e-6, max_iter=20000, eps_start=1e-1, level_tol=1e-4, ell=0)
    f, g, nr = pkg.solve(p, tol=1e-6, max_iter=20000, eps_start=1e-1, level_tol=1e-4, ell=30)
    assert sk["return_status"] == pkg.EOT_OK and nr["return_status"] == pkg.EOT_OK, (sk, nr)
    assert nr["stalled"] == 0, nr
    assert nr["iters"] <= sk["iters"] + 10, (nr["iters"], sk["iters"])
    assert O.evaluate(f, g, _cost(p), p.a, p.b, p.eps)["l1"] <= 1e-6
