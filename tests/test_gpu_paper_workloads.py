"""The paper's Sec. 5 workloads through the CUDA path (eot_solve), every
returned pair scored by the float64 oracle.

* The 2-D Gaussian experiment (Fig. 5.1): 200 points ~ N(0, I) against 400
  points ~ N((4, 4), [[1, -.8], [-.8, 1]]), uniform weights, raw squared
  Euclidean cost; the three protocols: sequential warm start from eps = 1
  (modes refreshed at every level), static modes computed once at eps' = 1,
  and the number of modes l at eps = 0.25 from the eps = 1 solution.  The
  paper prints no iteration counts (figures only); the claims checked are its
  qualitative ones, which the oracle reproduces in float64
  (tests/test_oracle_pins.py): SK-NR needs fewer iterations than Sinkhorn at
  every level after the first, and more modes need fewer iterations.
* The single-cell shapes of Fig. 5.2 (6507 x 3815 and 3815 x 2982 points in
  R^30; the data set itself is not available, synthetic N(0, I)/8 clouds
  stand in for it), cost normalised to max 1, eps from 1.0 halving, l = 30.
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


@pytest.fixture(scope="module")
def gauss2d():
    p = W.gaussians_2d(200, seed=0)
    C = O.sq_euclidean_cost(p.X, p.Y).astype(np.float32).astype(np.float64)
    return p, C


def _level_iters(pkg, p, C, eps, **opts):
    p.eps = eps
    f, g, res = pkg.solve(p, tol=1e-6, max_iter=200000, eps_start=1.0, eps_factor=0.5, **opts)
    assert res["return_status"] == pkg.EOT_OK, res
    assert O.evaluate(f, g, C, p.a, p.b, eps)["l1"] <= 1e-6
    return res["iters"]


def test_two_gaussians_sequential_and_static_warm_starts(pkg, gauss2d):
    p, C = gauss2d
    levels = (1.0, 0.5, 0.25)
    sk = [_level_iters(pkg, p, C, e, ell=0) for e in levels]
    seq = [_level_iters(pkg, p, C, e, ell=10, sequential_modes=1) for e in levels]
    static = [_level_iters(pkg, p, C, e, ell=10, sequential_modes=0) for e in levels]
    print(f"iterations per level (eps 1, 0.5, 0.25): Sinkhorn {sk}, sequential SK-NR(10) {seq}, "
          f"static SK-NR(10) {static}")
    assert seq[0] == sk[0] == static[0]        # no modes yet at the first level
    assert all(2 * q <= s for q, s in zip(seq[1:], sk[1:])), (seq, sk)
    assert all(q < s for q, s in zip(static[1:], sk[1:])), (static, sk)


def test_two_gaussians_more_modes_fewer_iterations(pkg, gauss2d):
    p, C = gauss2d
    p.eps = 0.25
    counts = []
    for ell in (0, 2, 5, 10, 20):
        f, g, res = pkg.solve(p, tol=1e-6, max_iter=200000, eps_start=1.0, eps_factor=0.25,
                              ell=ell)
        assert res["return_status"] == pkg.EOT_OK and res["levels"] == 2, res
        assert O.evaluate(f, g, C, p.a, p.b, 0.25)["l1"] <= 1e-6
        counts.append(res["iters"])
    print(f"iterations at eps = 0.25 with l = 0, 2, 5, 10, 20 modes from eps' = 1: {counts}")
    assert all(b <= a for a, b in zip(counts, counts[1:])), counts
    assert 4 * counts[-1] < counts[0], counts


@pytest.mark.parametrize("n,m", [(6507, 3815), (3815, 2982)])
def test_single_cell_shapes(pkg, n, m):
    p = W.gaussian_cloud(n, m, d=30, seed=n, eps=1.0 / 64)
    p.normalize_cost = True
    C = O.sq_euclidean_cost(p.X, p.Y, normalize=True).astype(np.float32).astype(np.float64)
    out = {}
    for ell in (0, 30):
        f, g, res = pkg.solve(p, tol=1e-6, max_iter=200000, eps_start=1.0, eps_factor=0.5,
                              ell=ell)
        assert res["return_status"] == pkg.EOT_OK, res
        assert O.evaluate(f, g, C, p.a, p.b, p.eps)["l1"] <= 1e-6
        out[ell] = res
    print(f"{n}x{m}: Sinkhorn {out[0]['total_iters']} iterations ({out[0]['seconds']*1e3:.1f} ms),"
          f" SK-NR(30) {out[30]['total_iters']} ({out[30]['seconds']*1e3:.1f} ms)")
    assert out[30]["total_iters"] < out[0]["total_iters"]


def test_spectrum_concentrates_on_the_device(pkg):
    """Sec. 3, spectral stability, through the library: the square against
    the annulus (160 x 160, raw cost) solved at eps = 0.256 ... 0.016, then the
    ten leading modes of Op(pi) o Op(pi)^T by the device's subspace iteration
    (eot_spectral_modes).  Its rho_k^2 equal numpy.linalg.eigh of the dense
    operator at the same pair; each grows as eps halves (towards 1), while the
    leading three-mode subspace moves little (the oracle's pin of the same
    claims: test_spectrum_concentrates_as_eps_decreases)."""
    p = W.square_annulus(160, 160, seed=0)
    C32 = O.sq_euclidean_cost(p.X, p.Y).astype(np.float32)
    C = C32.astype(np.float64)
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x)).cuda()
    rho, modes = [], []
    for eps in (0.256, 0.128, 0.064, 0.032, 0.016):
        p.eps = eps
        f, g, res = pkg.solve(p, tol=1e-6, max_iter=200000)
        assert res["return_status"] == pkg.EOT_OK, res
        V = torch.zeros((160, 10), dtype=torch.float64, device="cuda")
        r2 = torch.zeros(10, dtype=torch.float64, device="cuda")
        st, it, resid = pkg.eot_spectral_modes(160, 160, dev(C32), dev(f), dev(g), dev(p.a),
                                               dev(p.b), eps, 10, 10, 1e-5, 500, False, V, r2)
        assert st == pkg.EOT_OK and resid <= 1e-5, (eps, st, it, resid)
        _, rd = O.spectral_modes_dense(f, g, C, p.a, p.b, eps, 10)
        r2 = r2.cpu().numpy()
        assert np.abs(r2 - rd).max() < 1e-5, (eps, r2, rd)
        rho.append(r2)
        modes.append(V.cpu().numpy())
    rho = np.array(rho)
    print("rho_k^2 (rows: eps 0.256 ... 0.016):", np.round(rho[:, :4], 4).tolist())
    assert np.all(np.diff(rho, axis=0) > 0)
    assert rho[-1, 0] > 0.9 and rho[0, 0] < 0.5
    sa = np.sqrt(p.a)[:, None]
    Qu, _ = np.linalg.qr(sa * modes[0][:, :3])
    Qv, _ = np.linalg.qr(sa * modes[2][:, :3])
    assert np.linalg.svd(Qu.T @ Qv, compute_uv=False).min() > 0.95
