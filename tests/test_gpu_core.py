"""Parity of the CUDA hot path with the float64 oracle, through the C ABI.

Tolerances (float32 exponentials and sums, exponents formed exactly, float64
potentials): a single (C, eps)-transform matches the oracle to 1e-5 * eps when
its shift (the current potential on the output side) is within a few eps of
the result, as in the iterations; a shift |off| away adds the float32 rounding
of exponents of size |off| / eps, |off| 2^-22;
products Op(pi) Z and Op(pi)^T Z to 2e-5 relative; the cost is bit-exact
(same float64 operations, one rounding).  Solves are scored by the oracle's
float64 evaluation of the returned potentials: L1 marginal error <= 1e-6.
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


def dev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


SHAPES = [(1, 1), (3, 5), (31, 33), (128, 128), (257, 300), (1000, 1203), (2048, 4096)]


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("eps", [1e-1, 1e-3])
def test_ctransform_parity(pkg, n, m, eps):
    prob = W.random_cost(n, m, seed=n * 7 + m)
    C = prob.C
    C64 = C.astype(np.float64)
    rng = np.random.default_rng(n + m)
    f = rng.random(n) * 0.5
    g_true = O.c_transform_f(f, C64, prob.a, eps)
    shift = g_true + rng.standard_normal(m) * 3 * eps      # a nearby shift
    dC = dev(C)
    for sh in (shift, None):
        out = torch.zeros(m, dtype=torch.float64, device="cuda")
        lr = torch.zeros(m, dtype=torch.float64, device="cuda")
        st = pkg.eot_ctransform(pkg.EOT_SIDE_COL, n, m, dC, dev(f), dev(prob.a),
                                None if sh is None else dev(sh), eps, out, lr)
        assert st == pkg.EOT_OK, pkg.last_error()
        o = out.cpu().numpy()
        assert np.abs(o - g_true).max() <= 1e-5 * eps + 1e-12, np.abs(o - g_true).max() / eps
        if sh is not None:
            ratio = (sh - g_true) / eps
            assert np.abs(lr.cpu().numpy() - ratio).max() <= 2e-5 * (1 + np.abs(ratio).max())
    # row direction: f = g^{C,eps}
    g = rng.random(m) * 0.5
    f_true = O.c_transform_g(g, C64, prob.b, eps)
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = pkg.eot_ctransform(pkg.EOT_SIDE_ROW, n, m, dC, dev(g), dev(prob.b),
                            dev(f_true + 2 * eps), eps, out, None)
    assert st == pkg.EOT_OK, pkg.last_error()
    assert np.abs(out.cpu().numpy() - f_true).max() <= 1e-5 * eps + 1e-12


# Shapes for the staged stream passes (m % 4 == 0): a single tile, a grid
# with fewer tiles than CTAs, tall (many contributors per column block), wide
# (many per row block), ragged in both directions.
STREAM_SHAPES = [(4, 4), (64, 8), (5003, 260), (40, 9000), (777, 1024)]


@pytest.mark.parametrize("n,m", STREAM_SHAPES)
def test_ctransform_stream_shapes(pkg, n, m):
    eps = 2e-3
    prob = W.random_cost(n, m, seed=n + 3 * m)
    C64 = prob.C.astype(np.float64)
    rng = np.random.default_rng(n * m)
    dC = dev(prob.C)
    f = rng.random(n) * 0.5
    g_true = O.c_transform_f(f, C64, prob.a, eps)
    out = torch.zeros(m, dtype=torch.float64, device="cuda")
    st = pkg.eot_ctransform(pkg.EOT_SIDE_COL, n, m, dC, dev(f), dev(prob.a),
                            dev(g_true + rng.standard_normal(m) * eps), eps, out, None)
    assert st == pkg.EOT_OK, pkg.last_error()
    assert np.abs(out.cpu().numpy() - g_true).max() <= 1e-5 * eps + 1e-12
    g = rng.random(m) * 0.5
    f_true = O.c_transform_g(g, C64, prob.b, eps)
    for off in (2 * eps, -0.3):   # near shift, and one far enough to move the reference
        out = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = pkg.eot_ctransform(pkg.EOT_SIDE_ROW, n, m, dC, dev(g), dev(prob.b),
                                dev(f_true + off), eps, out, None)
        assert st == pkg.EOT_OK, pkg.last_error()
        # the exponents are float32 values of size |off| / eps: their rounding
        # adds |off| 2^-22 to the 1e-5 eps of a transform near its shift
        assert np.abs(out.cpu().numpy() - f_true).max() <= 1e-5 * eps + abs(off) * 2.0 ** -22


def test_ctransform_unaligned_cost_rows(pkg):
    """A cost whose rows are not 16-byte aligned takes the striped kernels:
    same results as the aligned copy."""
    n, m, eps = 300, 256, 1e-2
    prob = W.random_cost(n, m, seed=11)
    f = np.linspace(0, 0.3, n)
    g_true = O.c_transform_f(f, prob.C.astype(np.float64), prob.a, eps)
    big = torch.zeros(n * m + 1, dtype=torch.float32, device="cuda")
    big[1:] = torch.as_tensor(prob.C.ravel()).cuda()
    unaligned = big[1:]
    assert unaligned.data_ptr() % 16 != 0
    out = torch.zeros(m, dtype=torch.float64, device="cuda")
    st = pkg.eot_ctransform(pkg.EOT_SIDE_COL, n, m, unaligned, dev(f), dev(prob.a), None, eps,
                            out, None)
    assert st == pkg.EOT_OK, pkg.last_error()
    assert np.abs(out.cpu().numpy() - g_true).max() <= 1e-5 * eps + 1e-12


def test_ctransform_extreme_exponents(pkg):
    """Shifts far from the transform (terms near float32 over/underflow) are
    re-centred by the running log-sum-exp."""
    n, m, eps = 300, 200, 1e-3
    prob = W.random_cost(n, m, seed=5)
    C64 = prob.C.astype(np.float64)
    f = np.linspace(0, 1, n)
    g_true = O.c_transform_f(f, C64, prob.a, eps)
    for off in (-0.5, 0.5):   # exponents of +-500 natural units relative to the shift
        out = torch.zeros(m, dtype=torch.float64, device="cuda")
        st = pkg.eot_ctransform(pkg.EOT_SIDE_COL, n, m, dev(prob.C), dev(f), dev(prob.a),
                                dev(g_true + off), eps, out, None)
        assert st == pkg.EOT_OK
        # float32 exponents of size |off| / eps: rounding |off| 2^-22 beyond 1e-5 eps
        assert np.abs(out.cpu().numpy() - g_true).max() <= 1e-5 * eps + abs(off) * 2.0 ** -22


# m % 4 != 0 takes the CUDA-core kernels, m % 4 == 0 the staged tensor-core
# kernels (ragged row and column blocks, every template width); the last two
# the staged kernels merge the segments of an output block either in a
# thread-block cluster or through global records, whichever the plan costs
# lower: most of these shapes take clusters; the tall 16384 x 256 cost
# merges its many column segments through global records
@pytest.mark.parametrize("n,m,k", [(50, 70, 8), (257, 129, 33), (1024, 900, 40),
                                   (300, 260, 17), (130, 516, 48), (2049, 1028, 30),
                                   (33, 4, 5), (4100, 132, 48), (4096, 4096, 40),
                                   (6507, 3816, 30), (16384, 256, 30)])
def test_kapply_parity(pkg, n, m, k):
    prob = W.uniform_square(n, m, seed=11, eps=0.05)
    C = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32)
    C64 = C.astype(np.float64)
    ref = O.sinkhorn(C64, prob.a, prob.b, 0.05, tol=1e-10, max_iter=5000)
    rng = np.random.default_rng(3)
    Zc = rng.standard_normal((n, k)).astype(np.float32)
    Zr = rng.standard_normal((m, k)).astype(np.float32)
    outc = torch.zeros((m, k), dtype=torch.float32, device="cuda")
    outr = torch.zeros((n, k), dtype=torch.float32, device="cuda")
    args = (dev(C), dev(ref.f), dev(ref.g), dev(prob.a), dev(prob.b), 0.05)
    assert pkg.eot_kapply(pkg.EOT_SIDE_COL, n, m, k, *args, dev(Zc), outc) == pkg.EOT_OK
    assert pkg.eot_kapply(pkg.EOT_SIDE_ROW, n, m, k, *args, dev(Zr), outr) == pkg.EOT_OK
    ec = O.op_pi_T(Zc.astype(np.float64), ref.f, ref.g, C64, prob.a, prob.b, 0.05)
    er = O.op_pi(Zr.astype(np.float64), ref.f, ref.g, C64, prob.a, prob.b, 0.05)
    sc = np.abs(ec).max()
    sr = np.abs(er).max()
    assert np.abs(outc.cpu().numpy() - ec).max() <= 2e-5 * sc
    assert np.abs(outr.cpu().numpy() - er).max() <= 2e-5 * sr


@pytest.mark.parametrize("n,m,d,norm", [(7, 9, 2, True), (300, 257, 3, True), (64, 100, 64, False),
                                        (2048, 1500, 3, True), (1000, 777, 16, True),
                                        (40, 3000, 500, True), (33, 65, 1, True)])
def test_cost_bit_exact(pkg, n, m, d, norm):
    """C = ||x - y||^2 in float64, divided by its float64 maximum, rounded once:
    bit for bit the float32 rounding of the float64 definition (many tied
    maxima on the 1-D grid; 500 coordinates take the untiled kernels)."""
    rng = np.random.default_rng(d)
    X = rng.random((n, d)).astype(np.float32)
    Y = rng.random((m, d)).astype(np.float32)
    if d == 1:
        X = (np.arange(n, dtype=np.float32) / 8).reshape(n, 1)
        Y = (np.arange(m, dtype=np.float32) / 8)[::-1].copy().reshape(m, 1)
    out = torch.zeros((n, m), dtype=torch.float32, device="cuda")
    cmax = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert pkg.eot_cost(n, m, d, dev(X), dev(Y), norm, out, cmax) == pkg.EOT_OK
    ref = O.sq_euclidean_cost(X, Y, normalize=norm).astype(np.float32)
    got = out.cpu().numpy()
    assert np.array_equal(got, ref)
    assert cmax.item() == O.sq_euclidean_cost(X, Y).max()


def test_cost_rounding_at_float32_midpoints(pkg):
    """Normalised costs whose float64 value sits exactly on, or one float64
    unit above, a float32 rounding midpoint (1.5625 + 2^-24 has the bit just
    below float32 precision set and nothing under it; 2^-52 more is one unit
    above): the kernel's fast quotient path hands these to the corrected
    quotient, and the result is still the float32 rounding of the float64
    definition, bit for bit."""
    X = np.zeros((2, 3), dtype=np.float32)
    X[1] = [0.5, 0.0, 0.0]
    Y = np.array([[1.25, 2.0 ** -12, 0.0], [1.25, 2.0 ** -12, 2.0 ** -26], [2.0, 0.0, 0.0],
                  [1.25, 0.0, 2.0 ** -12], [0.75, 2.0 ** -13, 2.0 ** -27]], dtype=np.float32)
    n, m = X.shape[0], Y.shape[0]
    out = torch.zeros((n, m), dtype=torch.float32, device="cuda")
    assert pkg.eot_cost(n, m, 3, dev(X), dev(Y), True, out) == pkg.EOT_OK
    ref = O.sq_euclidean_cost(X, Y, normalize=True).astype(np.float32)
    assert np.array_equal(out.cpu().numpy(), ref)


def test_marginal_error_parity(pkg):
    prob = W.random_cost(333, 211, seed=9)
    C64 = prob.C.astype(np.float64)
    rng = np.random.default_rng(1)
    eps = 0.02
    f = O.c_transform_g(rng.random(211) * 0.1, C64, prob.b, eps)
    g = O.c_transform_f(f, C64, prob.a, eps) + rng.standard_normal(211) * 1e-4
    st, r, c = pkg.eot_marginal_error(333, 211, dev(prob.C), dev(f), dev(g), dev(prob.a),
                                      dev(prob.b), eps)
    assert st == pkg.EOT_OK
    rr, cc = O.marginal_errors(f, g, C64, prob.a, prob.b, eps)
    assert abs(r - rr) <= 1e-6 + 1e-4 * rr and abs(c - cc) <= 1e-6 + 1e-4 * cc


def _score(prob, f, g, eps):
    if prob.C is not None:
        C = prob.C.astype(np.float64)
    else:
        C = O.sq_euclidean_cost(prob.X, prob.Y, normalize=prob.normalize_cost).astype(np.float32).astype(np.float64)
    return C, O.evaluate(f, g, C, prob.a, prob.b, eps)


@pytest.mark.parametrize("ell", [0, 8])
def test_solve_small_parity(pkg, ell):
    prob = W.uniform_square(64, 80, seed=2, eps=2e-2)
    f, g, res = pkg.solve(prob, tol=3e-7, ell=ell, eps_start=1e-1, max_iter=50000)
    assert res["return_status"] == pkg.EOT_OK, res
    C, ev = _score(prob, f, g, prob.eps)
    assert ev["l1"] <= 1e-6, ev
    ref = O.continuation(C, prob.a, prob.b, prob.eps, tol=1e-13, eps_start=1e-1, ell=0)
    fr, gr = O.gauge_normalize(ref.f, ref.g, prob.a, prob.b)
    # a pair whose marginal error is l1 lies within about eps l1 / (1 - rho_1^2)
    # of the optimum along the slowest mode (Lemma 3.2's contraction rho_1^2)
    _, rho2 = O.spectral_modes_dense(ref.f, ref.g, C, prob.a, prob.b, prob.eps, 1)
    bound = prob.eps * 2.0 * ev["l1"] / (1.0 - rho2[0]) + 1e-5 * prob.eps
    err = max(np.abs(f - fr).max(), np.abs(g - gr).max())
    assert err <= bound, (err / prob.eps, bound / prob.eps)
    # the reported L1 comes from evaluation passes at eps itself with an
    # unbiased exponential: it agrees with the float64 evaluation up to the
    # float32 rounding noise of the terms (no systematic part)
    d = res["l1_marginal"] - ev["l1"]
    assert abs(d) <= 3e-8 + 0.25 * ev["l1"], (res["l1_marginal"], ev["l1"])
    assert abs(res["q_dual"] - ev["q_dual"]) <= 1e-9 + 1e-6 * abs(ev["q_dual"])


def test_plain_sinkhorn_many_tiles(pkg):
    """Plain Sinkhorn over a cost of many tiles with ragged edges (the
    cooperative iteration loop when the rows are 16-byte aligned): the oracle
    scores the returned pair, and the iteration count of the last level equals
    the oracle's Sinkhorn on the same float32 cost from the same start, run to
    the device's stop target on the last level (0.75 tol, the margin for the
    float32 test), up to the rounding of the last test."""
    prob = W.gaussian_mixture(640, 804, seed=9, eps=1e-2)
    f, g, res = pkg.solve(prob, tol=1e-6, ell=0, eps_start=0.0, max_iter=100000)
    assert res["return_status"] == pkg.EOT_OK, res
    C, ev = _score(prob, f, g, prob.eps)
    assert ev["l1"] <= 1e-6, ev
    ref = O.sinkhorn(C, prob.a, prob.b, prob.eps, tol=0.75e-6, max_iter=100000)
    assert abs(res["iters"] - ref.iters) <= max(3, ref.iters // 50), (res["iters"], ref.iters)
    fr, gr = O.gauge_normalize(ref.f, ref.g, prob.a, prob.b)
    _, rho2 = O.spectral_modes_dense(ref.f, ref.g, C, prob.a, prob.b, prob.eps, 1)
    assert np.abs(f - fr).max() <= prob.eps * 2e-6 / (1 - rho2[0]) + 1e-5 * prob.eps


def test_solve_sknr_beats_sk_iterations(pkg):
    prob = W.gaussian_mixture(512, 512, seed=0, eps=1e-3)
    _, _, sk = pkg.solve(prob, tol=1e-6, ell=0, eps_start=1e-1, max_iter=100000)
    f, g, nr = pkg.solve(prob, tol=1e-6, ell=30, eps_start=1e-1, max_iter=100000)
    assert sk["return_status"] == pkg.EOT_OK and nr["return_status"] == pkg.EOT_OK, (sk, nr)
    assert nr["iters"] * 5 < sk["iters"], (nr["iters"], sk["iters"])
    _, ev = _score(prob, f, g, prob.eps)
    assert ev["l1"] <= 1e-6, ev
