"""The bounds-checked build (-DEOT_DEBUG, _lib/libeot_debug.so): the paths of
the library run with every device check compiled in (shared-memory tables of
the small dense kernels, partial-state slots of the passes, mode widths of the
tensor-core products, gang ranks of the batch) and no check fires; the results
agree with the release build's.  Run in a child process that loads the debug
library (EOT_LIBRARY)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import workloads as W
import paper_2506_14780_gb300 as pkg
pkg.load()
out = {"debug": int(pkg.eot.load().eot_debug_build())}
def run(name, prob, **kw):
    f, g, r = pkg.solve(prob, tol=1e-6, max_iter=100000, **kw)
    out[name] = {"status": r["return_status"], "error": r.get("error", ""), "f": f[:64].tolist(),
                 "g": g[:64].tolist(), "iters": r["total_iters"]}
run("plain", W.gaussian_mixture(600, 804, seed=1, eps=1e-2))
run("plain_unaligned", W.gaussian_mixture(500, 803, seed=2, eps=1e-2))
run("sknr", W.gaussian_mixture(512, 640, seed=3, eps=5e-3), ell=20, eps_start=1e-1)
run("sknr_filter", W.gaussian_mixture(400, 300, seed=4, eps=5e-3), ell=10, eps_start=1e-1,
    eig_degree=4, eig_tol=1e-4)
run("fp64", W.uniform_square(128, 160, seed=5, eps=2e-2), prec=pkg.EOT_PREC_FP64, ell=8,
    eps_start=1e-1)
q = W.gaussian_cloud(700, 900, d=16, seed=6, eps=2e-2)
q.normalize_cost = True
run("gram", q, prec=pkg.EOT_PREC_SPLIT_TC)
probs = W.batch_problems(count=12, seed=7, n_lo=40, n_hi=900, eps_lo=0.02, eps_hi=0.1)
keep = []
cp = [pkg.make_problem(p.a, p.b, X=p.X, Y=p.Y, eps=p.eps, normalize_cost=True, keep=keep)
      for p in probs]
for ell in (0, 10):
    fo = [np.zeros(p.a.shape[0]) for p in probs]
    go = [np.zeros(p.b.shape[0]) for p in probs]
    st, rs = pkg.eot_solve_batch(cp, pkg.default_options(tol=1e-6, max_iter=100000, ell=ell,
                                                         eps_start=1e-1), fo, go)
    out[f"batch{ell}"] = {"status": st, "error": pkg.last_error() if st < 0 else "",
                          "f": [f[:16].tolist() for f in fo]}
print("JSON" + json.dumps(out))
"""


def _child(lib_path):
    env = dict(os.environ)
    if lib_path:
        env["EOT_LIBRARY"] = lib_path
    else:
        env.pop("EOT_LIBRARY", None)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("JSON")][-1]
    return json.loads(line[4:])


def test_debug_build_runs_clean_and_agrees():
    from paper_2506_14780_gb300 import build
    path = build.build(debug=True)
    dbg = _child(path)
    rel = _child(None)
    assert dbg["debug"] == 1 and rel["debug"] == 0
    for name in ("plain", "plain_unaligned", "sknr", "sknr_filter", "fp64", "gram"):
        assert dbg[name]["status"] == 0, (name, dbg[name]["error"])
        assert rel[name]["status"] == 0, (name, rel[name]["error"])
        eps = {"plain": 1e-2, "plain_unaligned": 1e-2, "sknr": 5e-3, "sknr_filter": 5e-3,
               "fp64": 2e-2, "gram": 2e-2}[name]
        for side in ("f", "g"):
            d = np.abs(np.array(dbg[name][side]) - np.array(rel[name][side])).max()
            assert d <= 1e-5 * eps, (name, side, d / eps)
    for name in ("batch0", "batch10"):
        assert dbg[name]["status"] == 0, (name, dbg[name]["error"])
        for fd, fr in zip(dbg[name]["f"], rel[name]["f"]):
            assert np.abs(np.array(fd) - np.array(fr)).max() <= 1e-7
