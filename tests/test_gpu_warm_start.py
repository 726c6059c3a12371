"""Warm-start state through the C ABI (eot_problem.g_init, V_init, V_out; the
server's resident modes): the resume side of a checkpoint (f, g, V), the
paper's warm-start idea (Sec. 1, Sec. 4, Sec. 5's static modes).  The oracle
scores every returned pair in float64 and gives the reference modes
(numpy.linalg.eigh of the dense operator)."""
import dataclasses
import time

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


def _cost(p):
    return O.sq_euclidean_cost(p.X, p.Y, normalize=True).astype(np.float32).astype(np.float64)


def _near_optimum(f, g, C, p, ref=None):
    """Potentials of a pair with L1 error l1 lie within about eps l1 / (1 -
    rho_1^2) of the optimum along the slowest mode (Lemma 3.2's contraction).
    ref: the oracle's Sinkhorn solution to 1e-12 (computed if None)."""
    ev = O.evaluate(f, g, C, p.a, p.b, p.eps)
    if ref is None:
        ref = O.sinkhorn(C, p.a, p.b, p.eps, tol=1e-12, max_iter=400000)
    fr, gr = O.gauge_normalize(ref.f, ref.g, p.a, p.b)
    _, rho2 = O.spectral_modes_dense(ref.f, ref.g, C, p.a, p.b, p.eps, 1)
    bound = p.eps * 2.0 * ev["l1"] / (1.0 - rho2[0]) + 1e-5 * p.eps
    err = max(np.abs(f - fr).max(), np.abs(g - gr).max())
    return ev, err, bound


@pytest.mark.parametrize("n,m", [(600, 500), (400, 700)])
def test_g_init_resumes_the_optimum(pkg, n, m):
    """g_init = the optimal g: the first row half-step gives the optimal f,
    so the level stops at its first test; a cold start needs hundreds of
    iterations."""
    p = W.gaussian_mixture(n, m, seed=5, eps=1e-2)
    C = _cost(p)
    r = O.sinkhorn(C, p.a, p.b, p.eps, tol=1e-12, max_iter=400000)
    f, g, res = pkg.solve(p, tol=1e-6, max_iter=1000, g_init=r.g)
    assert res["return_status"] == pkg.EOT_OK, res
    assert res["iters"] <= 2, res
    ev, err, bound = _near_optimum(f, g, C, p, r)
    assert ev["l1"] <= 1e-6 and err <= bound, (ev, err / p.eps, bound / p.eps)
    _, _, cold = pkg.solve(p, tol=1e-6, max_iter=100000)
    assert cold["return_status"] == pkg.EOT_OK and cold["iters"] > 20 * res["iters"], cold


def test_g_init_from_another_eps(pkg):
    """g_init from the optimum at 2 eps: the solve at eps reaches the tolerance
    (scored by the oracle) in fewer iterations than from zero."""
    p = W.gaussian_mixture(500, 450, seed=8, eps=1e-2)
    C = _cost(p)
    r2 = O.sinkhorn(C, p.a, p.b, 2 * p.eps, tol=1e-10, max_iter=400000)
    f, g, res = pkg.solve(p, tol=1e-6, max_iter=100000, g_init=r2.g)
    assert res["return_status"] == pkg.EOT_OK, res
    ev, err, bound = _near_optimum(f, g, C, p)
    assert ev["l1"] <= 1e-6 and err <= bound, (ev, err / p.eps, bound / p.eps)
    _, _, cold = pkg.solve(p, tol=1e-6, max_iter=100000)
    assert res["iters"] < cold["iters"], (res["iters"], cold["iters"])


def test_batch_members_with_g_init(pkg):
    """The persistent batch runs a g_init member as the transposed problem
    (its f is the caller's g): results in the caller's roles, at the optimum
    after one test; members without a warm start alongside are unaffected."""
    probs = [W.gaussian_mixture(300, 420, seed=11, eps=1e-2),
             W.gaussian_mixture(520, 260, seed=12, eps=2e-2),
             W.gaussian_mixture(200, 210, seed=13, eps=1e-2)]
    refs = [O.sinkhorn(_cost(q), q.a, q.b, q.eps, tol=1e-12, max_iter=400000) for q in probs]
    keep = []
    cp = [pkg.make_problem(q.a, q.b, X=q.X, Y=q.Y, eps=q.eps, normalize_cost=True, keep=keep,
                           g_init=(r.g if k < 2 else None))
          for k, (q, r) in enumerate(zip(probs, refs))]
    fo = [np.zeros(q.a.shape[0]) for q in probs]
    go = [np.zeros(q.b.shape[0]) for q in probs]
    st, rs = pkg.eot_solve_batch(cp, pkg.default_options(tol=1e-6, max_iter=100000), fo, go)
    assert st == pkg.EOT_OK, [r.as_dict() for r in rs]
    for k, (q, f, g, r) in enumerate(zip(probs, fo, go, rs)):
        ev, err, bound = _near_optimum(f, g, _cost(q), q, refs[k])
        assert ev["l1"] <= 1e-6 and err <= bound, (k, ev, err / q.eps, bound / q.eps)
        if k < 2:
            assert r.iters <= 2, (k, r.as_dict())
    # the member without a warm start: the same result as in a batch of its own
    f1 = [np.zeros(probs[2].a.shape[0])]
    g1 = [np.zeros(probs[2].b.shape[0])]
    st1, _ = pkg.eot_solve_batch([cp[2]], pkg.default_options(tol=1e-6, max_iter=100000), f1, g1)
    assert st1 == pkg.EOT_OK
    assert np.array_equal(f1[0], fo[2]) and np.array_equal(g1[0], go[2])


def _subspace_dist(V, Vd, a):
    """Largest a-norm of the part of a column of V outside span(Vd) (both
    a-orthonormal)."""
    proj = Vd @ (Vd.T @ (a[:, None] * V))
    return np.sqrt((a[:, None] * (proj - V) ** 2).sum(0)).max()


def test_V_out_are_the_modes_of_the_returned_pair(pkg):
    p = W.gaussian_mixture(512, 640, seed=21, eps=5e-3)
    C = _cost(p)
    ell = 10
    f, g, res = pkg.solve(p, tol=1e-6, max_iter=100000, ell=ell, eps_start=1e-1,
                          eig_tol=1e-5, eig_max_iter=400, return_modes=True)
    assert res["return_status"] == pkg.EOT_OK, res
    assert O.evaluate(f, g, C, p.a, p.b, p.eps)["l1"] <= 1e-6
    V = res["V"]
    a = p.a
    assert np.all(np.isfinite(V))
    assert np.abs(V.T @ (a[:, None] * V) - np.eye(ell)).max() < 1e-5
    assert np.abs(a @ V).max() < 1e-6
    Vd1, rho2 = O.spectral_modes_dense(f, g, C, a, p.b, p.eps, ell + 1)
    gap = rho2[ell - 1] - rho2[ell]
    dist = _subspace_dist(V, Vd1[:, :ell], a)
    assert dist <= 2.0 * 1e-5 / gap + 1e-4, (dist, gap)
    # without V_out the same solve returns the same pair, bit for bit, and
    # runs one mode computation fewer
    f2, g2, r2 = pkg.solve(p, tol=1e-6, max_iter=100000, ell=ell, eps_start=1e-1,
                           eig_tol=1e-5, eig_max_iter=400)
    assert np.array_equal(f, f2) and np.array_equal(g, g2)
    assert r2["eig_iters"] < res["eig_iters"] and r2["kernel_launches"] < res["kernel_launches"]


def test_V_init_static_modes_resume(pkg):
    """Checkpoint at eps' = 2 eps (f', V'), resume at eps with f_init = f' and
    V_init = V' in one level: SK-NR runs from the first iteration (Sec. 5's
    static modes), in fewer iterations than the same warm start with plain
    Sinkhorn.  A mixed and rescaled basis of the same span does too, and so
    does a basis with a constant and a repeated column (both dropped)."""
    p = W.gaussian_mixture(600, 500, seed=22, eps=2.5e-3)
    C = _cost(p)
    ell = 20
    p2 = dataclasses.replace(p, eps=2 * p.eps)
    f1, g1, r1 = pkg.solve(p2, tol=1e-6, max_iter=100000, ell=ell, eps_start=1e-1,
                           return_modes=True)
    assert r1["return_status"] == pkg.EOT_OK, r1
    V1 = r1["V"]
    f, g, res = pkg.solve(p, tol=1e-6, max_iter=100000, ell=ell, f_init=f1, V_init=V1)
    assert res["return_status"] == pkg.EOT_OK, res
    assert res["levels"] == 1 and res["nr_accepted"] >= 1 and res["eig_iters"] == 0, res
    assert O.evaluate(f, g, C, p.a, p.b, p.eps)["l1"] <= 1e-6
    _, _, sk = pkg.solve(p, tol=1e-6, max_iter=100000, ell=0, f_init=f1)
    assert sk["return_status"] == pkg.EOT_OK
    print("static-mode resume:", res["iters"], "SK-NR iterations against", sk["iters"])
    assert res["iters"] < sk["iters"], (res["iters"], sk["iters"])
    # the same span in another basis, columns of scales 1e-2 .. 1e2: the
    # Newton steps live on the same subspace
    rng = np.random.default_rng(3)
    R = rng.standard_normal((ell, ell)) + 4 * np.eye(ell)
    Vmix = (V1 @ R) * np.logspace(-2, 2, ell)[None, :]
    fm, gm, rm = pkg.solve(p, tol=1e-6, max_iter=100000, ell=ell, f_init=f1, V_init=Vmix)
    assert rm["return_status"] == pkg.EOT_OK, rm
    assert O.evaluate(fm, gm, C, p.a, p.b, p.eps)["l1"] <= 1e-6
    assert rm["nr_accepted"] >= 1 and rm["iters"] < sk["iters"], rm
    # a constant column (nothing outside the constants) and a repeated one
    # are dropped (zeroed); the remaining ell - 2 modes still speed the level
    Vdup = np.concatenate([np.ones((V1.shape[0], 1)), V1[:, : ell - 2], V1[:, :1]], axis=1)
    fd, gd, rd = pkg.solve(p, tol=1e-6, max_iter=100000, ell=ell, f_init=f1, V_init=Vdup)
    assert rd["return_status"] == pkg.EOT_OK, rd
    assert O.evaluate(fd, gd, C, p.a, p.b, p.eps)["l1"] <= 1e-6
    assert rd["nr_accepted"] >= 1 and rd["iters"] < sk["iters"], rd
    print("mixed basis:", rm["iters"], "with dropped columns:", rd["iters"])


def test_device_memory_warm_start(pkg):
    """All arrays on the device (eot_mem DEVICE): g_init, V_init and V_out as
    tensors give the host call's results."""
    p = W.gaussian_mixture(300, 260, seed=23, eps=1e-2)
    C32 = O.sq_euclidean_cost(p.X, p.Y, normalize=True).astype(np.float32)
    ell = 8
    r = O.sinkhorn(C32.astype(np.float64), p.a, p.b, 2 * p.eps, tol=1e-10, max_iter=400000)
    rng = np.random.default_rng(0)
    V0 = rng.standard_normal((300, ell))
    out = {}
    for dev in (False, True):
        t = (lambda x: torch.as_tensor(np.ascontiguousarray(x)).cuda()) if dev else (lambda x: x)
        keep = []
        Vo = torch.zeros((300, ell), dtype=torch.float64, device="cuda") if dev else np.zeros((300, ell))
        q = pkg.make_problem(t(p.a), t(p.b), C=t(C32), eps=p.eps, keep=keep, g_init=t(r.g),
                             V_init=t(V0), V_out=Vo)
        f = torch.zeros(300, dtype=torch.float64, device="cuda") if dev else np.zeros(300)
        g = torch.zeros(260, dtype=torch.float64, device="cuda") if dev else np.zeros(260)
        st, res = pkg.eot_solve(q, pkg.default_options(tol=1e-6, max_iter=100000, ell=ell), f, g)
        assert st == pkg.EOT_OK, (st, pkg.last_error())
        cv = (lambda x: x.cpu().numpy()) if dev else (lambda x: x)
        out[dev] = (cv(f), cv(g), cv(Vo), res.as_dict())
    fh, gh, Vh, rh = out[False]
    fd, gd, Vd, rd = out[True]
    assert np.array_equal(fh, fd) and np.array_equal(gh, gd) and np.array_equal(Vh, Vd)
    assert rh["iters"] == rd["iters"]
    assert np.abs(Vh.T @ (p.a[:, None] * Vh) - np.eye(ell)).max() < 1e-5


def test_warm_start_arguments_are_checked(pkg):
    p = W.gaussian_mixture(64, 70, seed=0, eps=5e-2)
    bad_g = np.zeros(70)
    bad_g[3] = np.nan
    _, _, r = pkg.solve(p, tol=1e-6, g_init=bad_g)
    assert r["return_status"] == pkg.EOT_EINVAL, r
    V = np.ones((64, 4))
    _, _, r = pkg.solve(p, tol=1e-6, ell=0, V_init=V)
    assert r["return_status"] == pkg.EOT_EINVAL, r
    _, _, r = pkg.solve(p, tol=1e-6, ell=0, return_modes=True)
    assert r["return_status"] == pkg.EOT_EINVAL, r
    V[5, 2] = np.inf
    _, _, r = pkg.solve(p, tol=1e-6, ell=4, V_init=V)
    assert r["return_status"] == pkg.EOT_EINVAL, r


def test_server_keeps_the_modes_of_a_cloud(pkg):
    """Two SK-NR requests on one cloud: the second warm-starts from the first's
    potentials and modes, so its first (and only) level runs SK-NR at once;
    the same request on a fresh cloud id starts its first level with plain
    Sinkhorn (no modes yet)."""
    o = pkg.default_options(tol=1e-6, max_iter=200000, eps_start=1e-1, ell=10)
    srv = pkg.Server(o, hbm_budget_bytes=4 << 30, max_slots=1)
    p1 = W.gaussian_mixture(500, 450, seed=24, eps=1e-2)
    p2 = dataclasses.replace(p1, eps=5e-3)

    def run(prob, cid):
        t = srv.submit(prob, cloud_id=cid)
        deadline = time.time() + 120
        while True:
            st, f, g, res = srv.poll(t)
            if st != pkg.EOT_PENDING:
                return st, f, g, res
            assert time.time() < deadline
            time.sleep(0.002)

    try:
        st, f, g, r1 = run(p1, 7)
        assert st == pkg.EOT_OK, r1
        st, f, g, r2 = run(p2, 7)
        assert st == pkg.EOT_OK, r2
        assert r2["levels"] == 1 and r2["nr_accepted"] >= 1, r2
        assert O.evaluate(f, g, _cost(p2), p2.a, p2.b, p2.eps)["l1"] <= 1e-6
        # a cold request on a new cloud: its first level has no modes
        st, f, g, r3 = run(p2, 8)
        assert st == pkg.EOT_OK and r3["levels"] > 1, r3
    finally:
        srv.close()
