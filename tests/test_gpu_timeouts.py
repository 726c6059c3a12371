"""Bounded device waits: a wait of one CTA on others that exceeds
``eot_options.wait_limit_s`` gives up, the call returns EOT_ETIMEDOUT, and the
device and the library stay usable (the next call on the same shapes is
correct, scored by the float64 oracle).

The waits are made to run out by a limit of 1 ns, so that any CTA that reaches
a barrier before the last one of its group gives up: nothing faults, traps or
hangs, every wait ends within its limit.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_2506_14780_gb300 as p
    p.load()
    return p


def _batch(pkg, probs, **kw):
    keep = []
    ps = [pkg.make_problem(q.a, q.b, X=q.X, Y=q.Y, eps=q.eps, normalize_cost=True, keep=keep)
          for q in probs]
    o = pkg.default_options(tol=1e-6, max_iter=50000, eps_start=1e-1, **kw)
    fs = [np.zeros(q.n) for q in probs]
    gs = [np.zeros(q.m) for q in probs]
    st, res = pkg.eot_solve_batch(ps, o, fs, gs)
    return st, res, fs, gs


def test_batch_gang_wait_gives_up(pkg, monkeypatch):
    """Gangs of 4 CTAs per problem with a 1 ns wait limit: gang barriers give up,
    the problems report EOT_ETIMEDOUT (a member whose every barrier happened to
    release in time reports a correct result); the same batch with the default
    limit then converges."""
    probs = W.batch_problems(6, seed=3, n_lo=200, n_hi=900)
    monkeypatch.setenv("EOT_BATCH_GANG", "4")
    st, res, fs, gs = _batch(pkg, probs, wait_limit_s=1e-9)
    assert st == pkg.EOT_ETIMEDOUT, (st, pkg.last_error())
    timed_out = [r.status == pkg.EOT_ETIMEDOUT for r in res]
    assert any(timed_out)
    for q, r, f, g, t in zip(probs, res, fs, gs, timed_out):
        if not t:
            assert r.status == pkg.EOT_OK
            C = O.sq_euclidean_cost(q.X, q.Y, normalize=True).astype(np.float32)
            assert O.evaluate(f, g, C.astype(np.float64), q.a, q.b, q.eps)["l1"] <= 1e-6
    st, res, fs, gs = _batch(pkg, probs)
    assert st == pkg.EOT_OK, pkg.last_error()
    for q, r, f, g in zip(probs, res, fs, gs):
        C = O.sq_euclidean_cost(q.X, q.Y, normalize=True).astype(np.float32).astype(np.float64)
        assert O.evaluate(f, g, C, q.a, q.b, q.eps)["l1"] <= 1e-6


def test_cooperative_grid_wait_gives_up(pkg):
    """The cooperative Sinkhorn loop (one launch, grid barriers between the
    half-steps) with a 1 ns wait limit gives up at its first barrier and the
    solve returns EOT_ETIMEDOUT; the next solve of the same shape (a fresh
    solver: the aborted launch left passes unfinished) is correct."""
    prob = W.gaussian_mixture(640, 804, seed=9, eps=1e-2)
    _, _, res = pkg.solve(prob, tol=1e-6, ell=0, eps_start=0.0, max_iter=100000,
                          wait_limit_s=1e-9)
    assert res["return_status"] == pkg.EOT_ETIMEDOUT, res
    assert "wait" in pkg.last_error()
    f, g, res = pkg.solve(prob, tol=1e-6, ell=0, eps_start=0.0, max_iter=100000)
    assert res["return_status"] == pkg.EOT_OK, res
    C = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32).astype(np.float64)
    assert O.evaluate(f, g, C, prob.a, prob.b, prob.eps)["l1"] <= 1e-6
