"""eot_plan: the coupling of a pair of potentials (Eq. pi(f,g)) and its
scalars (transport cost, mass, primal value of Eq. primal_EOT), element by
element against the float64 oracle; at a solution the primal value meets the
dual one, and the plan is the derivative of the optimal value in C (the pin
in tests/test_oracle_pins.py)."""
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


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("n,m,eps,converged", [(300, 257, 0.02, True), (129, 700, 0.05, False),
                                               (1, 33, 0.1, False)])
def test_plan_parity(pkg, n, m, eps, converged):
    prob = W.random_cost(n, m, seed=n + m)
    C = prob.C.astype(np.float32)
    C64 = C.astype(np.float64)
    a, b = prob.a, prob.b
    if converged:
        r = O.sinkhorn(C64, a, b, eps, tol=1e-12, max_iter=200000)
        f, g = r.f, r.g
    else:   # an arbitrary pair (the scalars are defined for any potentials)
        rng = np.random.default_rng(n)
        g = rng.standard_normal(m) * 0.05
        f = O.c_transform_g(g, C64, b, eps) + rng.standard_normal(n) * 1e-3
    P = torch.zeros((n, m), dtype=torch.float32, device="cuda")
    st, cost, mass, primal = pkg.eot_plan(n, m, dev(C), dev(f), dev(g), dev(a), dev(b), eps, P)
    assert st == pkg.EOT_OK, pkg.last_error()
    Pr = O.plan(f, g, C64, a, b, eps)
    Pd = P.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Pd - Pr) <= 1e-7 * Pr + 1e-300)
    assert abs(cost - (Pr * C64).sum()) <= 1e-12 * max(1.0, abs(cost))
    assert abs(mass - Pr.sum()) <= 1e-12
    assert abs(primal - O.primal_value(Pr, C64, a, b, eps)) <= 1e-12 * max(1.0, abs(primal))
    gap = primal - O.q_dual(f, g, C64, a, b, eps)
    assert abs(gap - O.duality_gap(f, g, C64, a, b, eps)) <= 1e-11
    if converged:
        assert abs(gap) < 1e-10 and abs(mass - 1.0) < 1e-10
    # scalars only (no plan buffer): the same values
    st, c2, m2, p2 = pkg.eot_plan(n, m, dev(C), dev(f), dev(g), dev(a), dev(b), eps)
    assert st == pkg.EOT_OK and (c2, m2, p2) == (cost, mass, primal)


def test_plan_of_the_benchmark_solution(pkg):
    """The 4096^2 benchmark workload solved by the library: the plan's scalars
    against the oracle, its mass 1 and its duality gap small at the solve's
    accuracy (L1 below 1e-6)."""
    prob = W.gaussian_mixture(4096, 4096, seed=0, eps=1e-3)
    f, g, res = pkg.solve(prob, tol=1e-6, ell=30, eps_start=1e-1, level_tol=1e-4, max_iter=200000)
    assert res["return_status"] == pkg.EOT_OK, res
    C = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32)
    st, cost, mass, primal = pkg.eot_plan(4096, 4096, dev(C), dev(f), dev(g), dev(prob.a),
                                          dev(prob.b), prob.eps)
    assert st == pkg.EOT_OK
    C64 = C.astype(np.float64)
    Pr = O.plan(f, g, C64, prob.a, prob.b, prob.eps)
    assert abs(cost - (Pr * C64).sum()) <= 1e-10 * abs(cost)
    assert abs(mass - Pr.sum()) <= 1e-12 and abs(mass - 1.0) < 1e-6
    gap = primal - O.q_dual(f, g, C64, prob.a, prob.b, prob.eps)
    assert abs(gap - O.duality_gap(f, g, C64, prob.a, prob.b, prob.eps)) <= 1e-10
    assert abs(gap) < 1e-6, gap


def test_plan_rejects_bad_arguments(pkg):
    C = torch.zeros((2, 2), dtype=torch.float32, device="cuda")
    v = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert pkg.eot_plan(2, 2, C, v, v, v, v, 0.0)[0] == pkg.EOT_EINVAL
