"""The exponentials of the float32 passes against float64 (eot_exp2).

The evaluation passes that verify a result form each term as 2^(p + q) with
p a float32 exponent and q a small correction (its rounding error and the
potentials' low parts), by range reduction and a degree-7 Taylor series of e^x
in float32 (ex2_pq).  Bounds, for |x| = |(p - rint(p) + q) ln 2| <= 0.53:
the series' remainder is below x^8 e^x / 8! < 2.3e-7 relative, the Horner
evaluation adds a few float32 roundings (each 2^-24 = 6e-8 relative), so the
relative error stays below 6e-7; with |q| <= 1e-4 the remainder is below 2e-8
and the roundings, round-to-nearest, average out: the mean relative error
over many arguments is below 2e-9.  The iterations' hardware approximation
(ex2.approx) has a mean relative error of the order of -5e-8 over [-30, 0],
every term biased the same way: that bias is why the verification does not
reuse it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_2506_14780_gb300 as p
    p.load()
    return p


def _run(pkg, p, q, variant):
    pd = torch.as_tensor(p).cuda()
    qd = torch.as_tensor(q).cuda()
    out = torch.empty_like(pd)
    assert pkg.eot_exp2(pd, qd, variant, out) == pkg.EOT_OK, pkg.last_error()
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = np.exp2(p.astype(np.float64) + q.astype(np.float64))
    return got / ref - 1.0


@pytest.mark.parametrize("lo,hi,qmax", [(-30.0, 0.0, 1e-4), (-120.0, 60.0, 1e-4),
                                        (-30.0, 0.0, 0.25)])
def test_ex2_pq_error_bounds(pkg, lo, hi, qmax):
    rng = np.random.default_rng(7)
    N = 1 << 22
    p = rng.uniform(lo, hi, N).astype(np.float32)
    q = rng.uniform(-qmax, qmax, N).astype(np.float32)
    rel = _run(pkg, p, q, 0)
    print(f"ex2_pq on [{lo}, {hi}], |q| <= {qmax}: max {np.abs(rel).max():.2e}, "
          f"mean {rel.mean():.2e}")
    assert np.abs(rel).max() <= 6e-7
    if qmax <= 1e-4:
        assert abs(rel.mean()) <= 2e-9


def test_ex2_pq_below_the_normal_range_and_masked_terms(pkg):
    p = np.array([-np.inf, -127.5, -200.0, -126.0, 0.0, 1.0], dtype=np.float32)
    q = np.zeros_like(p)
    pd, qd = torch.as_tensor(p).cuda(), torch.as_tensor(q).cuda()
    out = torch.empty_like(pd)
    assert pkg.eot_exp2(pd, qd, 0, out) == pkg.EOT_OK
    o = out.cpu().numpy()
    assert o[0] == 0.0 and o[1] == 0.0 and o[2] == 0.0
    assert o[3] == np.float32(2.0 ** -126) and o[4] == 1.0 and o[5] == 2.0


def test_hardware_exponential_is_biased(pkg):
    """The iterations' exponential: accurate to a few ulps, but every term low
    by a few 1e-8 on average (the reason for the separate verification)."""
    rng = np.random.default_rng(8)
    N = 1 << 22
    p = rng.uniform(-30.0, 0.0, N).astype(np.float32)
    q = np.zeros(N, dtype=np.float32)
    rel = _run(pkg, p, q, 1)
    pq = _run(pkg, p, q, 0)
    print(f"ex2.approx mean {rel.mean():.2e} max {np.abs(rel).max():.2e}; "
          f"ex2_pq mean {pq.mean():.2e}")
    assert np.abs(rel).max() <= 5e-7
    assert rel.mean() < -5e-9
    assert abs(pq.mean()) < 0.2 * abs(rel.mean())


def test_exp2_rejects_bad_arguments(pkg):
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    assert pkg.eot_exp2(x, x, 2, x) == pkg.EOT_EINVAL
