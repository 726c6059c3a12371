"""eot_ctransform_noalloc: the transform for callers that may not allocate
device memory (for example code running inside another allocator's fixed
device pool, or latency-critical loops where cudaMalloc may synchronise the
device).  It keeps its temporaries in a static device array instead of
allocating them, and must give the same results as eot_ctransform.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_2506_14780_gb300 as p
    p.load()
    return p


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


@pytest.mark.gpu
def test_noalloc_matches_allocating_transform(pkg):
    eps = 2e-3
    cases = [(pkg.EOT_SIDE_COL, 1000, 1203, 11), (pkg.EOT_SIDE_ROW, 777, 2048, 12)]
    # two calls in a row, each compared with the existing entry point
    for side, n, m, seed in cases:
        prob = W.random_cost(n, m, seed=seed)
        C64 = prob.C.astype(np.float64)
        rng = np.random.default_rng(seed)
        if side == pkg.EOT_SIDE_COL:
            pot, w, nout = rng.random(n) * 0.5, prob.a, m
            ref = O.c_transform_f(pot, C64, prob.a, eps)
        else:
            pot, w, nout = rng.random(m) * 0.5, prob.b, n
            ref = O.c_transform_g(pot, C64, prob.b, eps)
        shift = ref + rng.standard_normal(nout) * eps
        dC, dpot, dw, dsh = _dev(prob.C), _dev(pot), _dev(w), _dev(shift)
        outs = []
        for fn in (pkg.eot_ctransform, pkg.eot_ctransform_noalloc):
            out = torch.zeros(nout, dtype=torch.float64, device="cuda")
            lr = torch.zeros(nout, dtype=torch.float64, device="cuda")
            st = fn(side, n, m, dC, dpot, dw, dsh, eps, out, lr)
            assert st == pkg.EOT_OK, pkg.last_error()
            outs.append((out.cpu().numpy(), lr.cpu().numpy()))
        (o1, l1), (o2, l2) = outs
        assert np.abs(o2 - o1).max() <= 1e-5 * eps
        assert np.abs(l2 - l1).max() <= 1e-5
        assert np.abs(o2 - ref).max() <= 1e-5 * eps


@pytest.mark.gpu
@pytest.mark.parametrize("side", ["col", "row"])
def test_noalloc_without_shift(pkg, side):
    """shift = NULL: the call runs two passes (the first one places the
    reference) through the same static array; same results as eot_ctransform
    and as the oracle, on two calls in a row."""
    eps = 2e-3
    n, m = (1500, 1003) if side == "col" else (901, 2052)
    prob = W.random_cost(n, m, seed=21 + n)
    C64 = prob.C.astype(np.float64)
    rng = np.random.default_rng(n)
    s = pkg.EOT_SIDE_COL if side == "col" else pkg.EOT_SIDE_ROW
    if side == "col":
        pot, w, nout = rng.random(n) * 0.5, prob.a, m
        ref = O.c_transform_f(pot, C64, prob.a, eps)
    else:
        pot, w, nout = rng.random(m) * 0.5, prob.b, n
        ref = O.c_transform_g(pot, C64, prob.b, eps)
    dC, dpot, dw = _dev(prob.C), _dev(pot), _dev(w)
    for _ in range(2):
        outs = []
        for fn in (pkg.eot_ctransform, pkg.eot_ctransform_noalloc):
            out = torch.zeros(nout, dtype=torch.float64, device="cuda")
            assert fn(s, n, m, dC, dpot, dw, None, eps, out, None) == pkg.EOT_OK, pkg.last_error()
            outs.append(out.cpu().numpy())
        assert np.abs(outs[1] - outs[0]).max() <= 1e-5 * eps
        assert np.abs(outs[1] - ref).max() <= 1e-5 * eps


@pytest.mark.gpu
def test_noalloc_at_its_size_limit(pkg):
    """n = m = 16384, the largest size the static array serves: the carve-out
    fits on this device and the result equals the allocating transform's; the
    oracle checks a sample of output columns (each column's transform needs
    only that column of the cost)."""
    eps = 5e-3
    n = m = 16384
    prob = W.random_cost(n, m, seed=5)
    rng = np.random.default_rng(6)
    pot = rng.random(n) * 0.5
    dC, dpot, dw = _dev(prob.C), _dev(pot), _dev(prob.a)
    outs = []
    for fn in (pkg.eot_ctransform, pkg.eot_ctransform_noalloc):
        out = torch.zeros(m, dtype=torch.float64, device="cuda")
        st = fn(pkg.EOT_SIDE_COL, n, m, dC, dpot, dw, None, eps, out, None)
        assert st == pkg.EOT_OK, pkg.last_error()
        outs.append(out.cpu().numpy())
    assert np.abs(outs[1] - outs[0]).max() <= 1e-5 * eps
    cols = rng.choice(m, 64, replace=False)
    ref = O.c_transform_f(pot, prob.C[:, cols].astype(np.float64), prob.a, eps)
    assert np.abs(outs[1][cols] - ref).max() <= 1e-5 * eps


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch(pkg):
    C = torch.zeros(1, dtype=torch.float32, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = pkg.eot_ctransform_noalloc(pkg.EOT_SIDE_COL, 20000, 1, C, v, v, None, 1e-2, v)
    assert st == pkg.EOT_EINVAL
    assert "16384" in pkg.last_error()
