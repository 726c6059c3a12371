"""The seeded synthetic inputs match the recipes stated for each configuration
(shapes, ranges, distributions) and are reproducible from their seeds."""
import numpy as np

import workloads as W


def test_batch_problems_recipe():
    probs = W.batch_problems(512, seed=0)
    n = np.array([p.n for p in probs])
    m = np.array([p.m for p in probs])
    eps = np.array([p.eps for p in probs])
    d = np.array([p.X.shape[1] for p in probs])
    assert len(probs) == 512
    assert n.min() >= 64 and n.max() <= 4096 and m.min() >= 64 and m.max() <= 4096
    assert set(d) == {2, 3}
    assert eps.min() >= 1e-3 and eps.max() <= 1e-1
    # log-uniform: the logs' means sit mid-range (standard error ~ range/sqrt(12*512))
    for v, lo, hi in ((n, 64, 4096), (m, 64, 4096), (eps, 1e-3, 1e-1)):
        mid = 0.5 * (np.log(lo) + np.log(hi))
        assert abs(np.log(v).mean() - mid) < 0.1 * (np.log(hi) - np.log(lo))
    for p in probs[:20]:
        assert np.all(p.X >= 0) and np.all(p.X <= 1) and p.X.dtype == np.float32
        assert abs(p.a.sum() - 1) < 1e-12 and np.all(p.a > 0) and p.normalize_cost
    again = W.batch_problems(512, seed=0)
    assert all(np.array_equal(p.X, q.X) and np.array_equal(p.a, q.a) for p, q in zip(probs, again))


def test_served_stream_recipe():
    reqs = W.served_stream(seed=0, rate_per_s=2000.0, duration_s=1.0)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] <= 1.0
    # Poisson(2000/s) over 1 s: count within 5 standard deviations
    assert abs(len(reqs) - 2000) < 5 * np.sqrt(2000)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 2000) < 0.1 / 2000
    ns = np.array([r["problem"].n for r in reqs])
    assert ns.min() >= 128 and ns.max() <= 16384
    assert {r["problem"].X.shape[1] for r in reqs} <= {2, 3, 64}
    assert {r["problem"].eps for r in reqs} <= {1e-1, 1e-2, 1e-3}
    ids = [r["cloud_id"] for r in reqs]
    assert len(set(ids)) < len(ids)     # some requests re-use an earlier cloud


def test_paper_workload_shapes():
    g = W.gaussian_mixture(4096, 4096, d=3, seed=0, eps=1e-3)
    assert g.X.shape == (4096, 3) and g.Y.shape == (4096, 3) and g.normalize_cost
    assert abs(g.a.sum() - 1) < 1e-12 and abs(g.b.sum() - 1) < 1e-12
    c = W.gaussian_cloud(200, 300, d=64, seed=0, eps=1e-3)
    assert c.X.shape == (200, 64) and not c.normalize_cost
    assert abs(c.X.std() - 1 / 8) < 0.01
    e4 = W.gaussians_2d(200, seed=0)
    assert e4.X.shape == (200, 2) and e4.Y.shape == (400, 2)
    assert np.allclose(e4.Y.mean(0), [4, 4], atol=0.2)
