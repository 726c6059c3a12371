"""Write ``sknr_state_4096.npz``: an SK-NR iterate of the benchmark workload at
the target eps = 1e-3, for the element-wise parity test of one device
iteration (tests/test_gpu_sknr_step.py) at the benchmark's size.

Workload: ``workloads.gaussian_mixture(4096, 4096, seed=0)``, squared Euclidean
cost normalised to max 1 and rounded to float32.  The oracle runs the eps
continuation 1e-1 -> 1e-3 (halving, Sec. 5) with SK-NR(30), the D_a Hessian
and modes refreshed at every level by block subspace iteration (block 40,
Ritz residual 1e-2), levels solved to L1 1e-6; at eps = 1e-3 it stops once
the L1 marginal error is below 3e-3 (early in the level, where the Newton
steps are large).  Saved: g_k = f^{C,eps} of the stopping iterate (the input
of the next iteration's line 4) and the modes of that level rounded to
float32, which is how the device stores them.

Calls only ``oracle`` and ``workloads``.  Run from the repository root:
``python tests/golden/make_sknr_state_4096.py`` (a few minutes on one core).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sknr_state_4096.npz")


def main():
    prob = W.gaussian_mixture(4096, 4096, seed=0, eps=1e-3)
    C = O.sq_euclidean_cost(prob.X, prob.Y, normalize=True).astype(np.float32).astype(np.float64)
    a, b = prob.a, prob.b
    levels = O.eps_schedule(1e-1, 1e-3, 0.5)
    f = np.zeros(4096)
    V = None
    for t, e in enumerate(levels):
        last = t == len(levels) - 1
        res = O.sknr(C, a, b, e, V, tol=3e-3 if last else 1e-6, max_iter=100000, f0=f,
                     hessian="diag_alpha")
        f = res.f
        print(f"eps {e:.6g}: {res.iters} iterations", flush=True)
        if not last:
            V, _, _, _ = O.spectral_modes_subspace(res.f, res.g, C, a, b, e, 30, oversample=10,
                                                   tol=1e-2, max_iter=100, seed=t, V0=V)
    g_k = O.c_transform_f(f, C, a, 1e-3)
    np.savez_compressed(OUT, g=g_k, V=V.astype(np.float32), eps=1e-3, seed=0)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
