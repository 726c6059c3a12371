"""GPU tests of the float64 path (EOT_PREC_FP64): n = m = 256 points uniform in
[0,1]^2, uniform weights, squared-Euclidean cost normalised to max 1,
eps = 1e-2, plain log-domain Sinkhorn and SK-NR to an L1 marginal error of
1e-9, compared with the float64 oracle on the same float64 cost."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-9


@pytest.fixture(scope="module")
def pkg():
    import paper_2506_14780_gb300 as p
    p.load()
    return p


@pytest.fixture(scope="module")
def c1():
    p = W.uniform_square(256, 256, seed=0, eps=1e-2)
    C = O.sq_euclidean_cost(p.X, p.Y, normalize=True)
    ref = O.sinkhorn(C, p.a, p.b, p.eps, tol=1e-13, max_iter=400000)
    fr, gr = O.gauge_normalize(ref.f, ref.g, p.a, p.b)
    return p, C, fr, gr


def _check(pkg, p, C, fr, gr, f, g, res):
    assert res["return_status"] == pkg.EOT_OK, res
    ev = O.evaluate(f, g, C, p.a, p.b, p.eps)
    # the float64 passes reach the tolerance measured by the oracle itself
    assert ev["l1"] <= TOL, ev
    # potentials: the marginal error 1e-9 bounds the distance to the optimum by
    # about eps * 1e-9 / (1 - rho_1^2) with rho_1^2 = 0.92 here (1.3e-8 eps);
    # 2e-7 eps leaves room for the gauge and the evaluation order
    assert np.abs(f - fr).max() <= 2e-7 * p.eps
    assert np.abs(g - gr).max() <= 2e-7 * p.eps
    assert abs(res["l1_marginal"] - ev["l1"]) <= 1e-12


def test_fp64_sinkhorn_point_clouds(pkg, c1):
    p, C, fr, gr = c1
    f, g, res = pkg.solve(p, tol=TOL, ell=0, eps_start=0.0, max_iter=200000,
                          prec=pkg.EOT_PREC_FP64)
    _check(pkg, p, C, fr, gr, f, g, res)
    # the oracle's own Sinkhorn needs the same number of iterations up to the
    # rounding of the last one
    ref = O.sinkhorn(C, p.a, p.b, p.eps, tol=TOL, max_iter=200000)
    assert abs(res["iters"] - ref.iters) <= 2


def test_fp64_sknr_point_clouds(pkg, c1):
    p, C, fr, gr = c1
    f, g, res = pkg.solve(p, tol=TOL, ell=8, eps_start=1e-1, max_iter=200000,
                          prec=pkg.EOT_PREC_FP64)
    _check(pkg, p, C, fr, gr, f, g, res)
    assert res["nr_accepted"] >= 1


def test_fp64_given_cost_matrix(pkg, c1):
    """The cost given as a float64 matrix: host and device inputs give the same
    potentials bit for bit, both within the oracle's tolerance."""
    p, C, fr, gr = c1
    q = W.Problem(a=p.a, b=p.b, C=C, eps=p.eps, normalize_cost=False)
    f, g, res = pkg.solve(q, tol=TOL, ell=0, eps_start=0.0, max_iter=200000,
                          prec=pkg.EOT_PREC_FP64)
    _check(pkg, p, C, fr, gr, f, g, res)
    keep = []
    dp = pkg.make_problem(torch.as_tensor(p.a).cuda(), torch.as_tensor(p.b).cuda(),
                          C=torch.as_tensor(C).cuda(), eps=p.eps, keep=keep,
                          cost_dtype=np.float64)
    o = pkg.default_options(tol=TOL, ell=0, eps_start=0.0, max_iter=200000,
                            prec=pkg.EOT_PREC_FP64)
    fd = torch.zeros(256, dtype=torch.float64, device="cuda")
    gd = torch.zeros(256, dtype=torch.float64, device="cuda")
    st, _ = pkg.eot_solve(dp, o, fd, gd)
    assert st == pkg.EOT_OK, pkg.last_error()
    assert np.array_equal(fd.cpu().numpy(), f) and np.array_equal(gd.cpu().numpy(), g)


def test_fp64_normalised_given_cost(pkg, c1):
    """normalize_cost on a float64 matrix divides by its float64 maximum."""
    p, C, fr, gr = c1
    q = W.Problem(a=p.a, b=p.b, C=C * 3.0, eps=p.eps, normalize_cost=True)
    f, g, res = pkg.solve(q, tol=TOL, ell=0, eps_start=0.0, max_iter=200000,
                          prec=pkg.EOT_PREC_FP64)
    _check(pkg, p, C, fr, gr, f, g, res)


def test_fp64_rejects_nonfinite_cost(pkg):
    p = W.uniform_square(40, 30, seed=1, eps=0.05)
    C = O.sq_euclidean_cost(p.X, p.Y, normalize=True)
    C[3, 4] = np.inf
    q = W.Problem(a=p.a, b=p.b, C=C, eps=p.eps)
    f, g, res = pkg.solve(q, prec=pkg.EOT_PREC_FP64)
    assert res["return_status"] == pkg.EOT_EINVAL
