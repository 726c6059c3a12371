"""ctypes binding of libeot.so (include/eot.h): the same names, argument
marshalling only.  Every computation runs in the CUDA library; there is no
Python or CPU fallback, and loading fails loudly when the library is missing.

Host arrays are NumPy arrays (EOT_MEM_HOST); device arrays are torch CUDA
tensors (EOT_MEM_DEVICE), passed by their data pointers.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# EOT_LIBRARY selects another build of the library (the bounds-checked
# _lib/libeot_debug.so of build.build(debug=True)); the default is the release
LIB_PATH = os.environ.get("EOT_LIBRARY") or os.path.join(_HERE, "_lib", "libeot.so")

# ---- enums (eot.h) ----
EOT_OK, EOT_NOT_CONVERGED, EOT_PENDING = 0, 1, 2
EOT_EINVAL, EOT_ENOMEM, EOT_ENUMERIC, EOT_ETIMEDOUT, EOT_ECUDA, EOT_ENOTFOUND = -1, -2, -3, -4, -5, -6
EOT_MEM_HOST, EOT_MEM_DEVICE = 0, 1
EOT_PREC_FP64, EOT_PREC_FP32, EOT_PREC_SPLIT_TC = 0, 1, 2
EOT_HESS_DIAG_ALPHA, EOT_HESS_EXACT = 0, 1
EOT_SIDE_COL, EOT_SIDE_ROW = 0, 1

STATUS_NAMES = {0: "EOT_OK", 1: "EOT_NOT_CONVERGED", 2: "EOT_PENDING", -1: "EOT_EINVAL",
                -2: "EOT_ENOMEM", -3: "EOT_ENUMERIC", -4: "EOT_ETIMEDOUT", -5: "EOT_ECUDA",
                -6: "EOT_ENOTFOUND"}


class eot_problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("d", C.c_int32),
                ("a", C.c_void_p), ("b", C.c_void_p), ("C", C.c_void_p),
                ("X", C.c_void_p), ("Y", C.c_void_p), ("mem", C.c_int32),
                ("normalize_cost", C.c_int32), ("eps", C.c_double), ("f_init", C.c_void_p),
                ("g_init", C.c_void_p), ("V_init", C.c_void_p), ("V_out", C.c_void_p)]


class eot_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("ell", C.c_int32),
                ("eps_start", C.c_double), ("eps_factor", C.c_double), ("level_tol", C.c_double),
                ("sequential_modes", C.c_int32), ("oversample", C.c_int32),
                ("eig_tol", C.c_double), ("eig_max_iter", C.c_int32), ("prec", C.c_int32),
                ("hessian", C.c_int32), ("poll_every", C.c_int32), ("stream", C.c_void_p),
                ("wait_limit_s", C.c_double), ("stall_window", C.c_int32),
                ("eig_degree", C.c_int32), ("newton_solver", C.c_int32)]


class eot_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("total_iters", C.c_int32),
                ("nr_accepted", C.c_int32), ("nr_rejected", C.c_int32), ("levels", C.c_int32),
                ("eig_iters", C.c_int32), ("l1_marginal", C.c_double), ("row_l1", C.c_double),
                ("col_l1", C.c_double), ("q_dual", C.c_double), ("q_semi", C.c_double),
                ("dual_gap", C.c_double), ("seconds", C.c_double), ("seconds_eig", C.c_double),
                ("seconds_last_level", C.c_double), ("kernel_launches", C.c_int64),
                ("device_t_begin_ns", C.c_int64), ("device_t_end_ns", C.c_int64),
                ("stalled", C.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class eot_sknr_info(C.Structure):
    _fields_ = [("col_l1", C.c_double), ("q_semi", C.c_double), ("dq", C.c_double),
                ("newton_ok", C.c_int32), ("accepted", C.c_int32),
                ("products_in_range", C.c_int32),
                ("stage_seconds", C.c_double * 4)]


_PTR = C.c_void_p
_SIGNATURES = {
    "eot_default_options": (None, [C.POINTER(eot_options)]),
    "eot_solve": (C.c_int, [C.POINTER(eot_problem), C.POINTER(eot_options), _PTR, _PTR,
                            C.POINTER(eot_result)]),
    "eot_solve_batch": (C.c_int, [C.c_int32, C.POINTER(eot_problem), C.POINTER(eot_options),
                                  C.POINTER(_PTR), C.POINTER(_PTR), C.POINTER(eot_result)]),
    "eot_server_create": (C.c_int, [C.POINTER(eot_options), C.c_size_t, C.c_int32,
                                    C.POINTER(_PTR)]),
    "eot_server_submit": (C.c_int, [_PTR, C.POINTER(eot_problem), C.c_uint64,
                                    C.POINTER(C.c_uint64)]),
    "eot_server_poll": (C.c_int, [_PTR, C.c_uint64, _PTR, _PTR, C.POINTER(eot_result)]),
    "eot_server_stats": (C.c_int, [_PTR, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]),
    "eot_server_destroy": (None, [_PTR]),
    "eot_server_submit_opts": (C.c_int, [_PTR, C.POINTER(eot_problem), C.c_uint64,
                                         C.POINTER(eot_options), C.POINTER(C.c_uint64)]),
    "eot_server_status": (C.c_int, [_PTR, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "eot_server_simulate": (C.c_int, [C.c_int32, _PTR, _PTR, _PTR, _PTR, C.c_uint64, C.c_int32,
                                      C.c_double, _PTR, _PTR]),
    "eot_ctransform": (C.c_int, [C.c_int, C.c_int32, C.c_int32, _PTR, _PTR, _PTR, _PTR,
                                 C.c_double, _PTR, _PTR, _PTR]),
    "eot_ctransform_noalloc": (C.c_int, [C.c_int, C.c_int32, C.c_int32, _PTR, _PTR, _PTR, _PTR,
                                         C.c_double, _PTR, _PTR, _PTR]),
    "eot_kapply": (C.c_int, [C.c_int, C.c_int32, C.c_int32, C.c_int32, _PTR, _PTR, _PTR, _PTR,
                             _PTR, C.c_double, _PTR, _PTR, _PTR]),
    "eot_cost": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _PTR, _PTR, C.c_int32, _PTR, _PTR,
                           _PTR]),
    "eot_spectral_modes": (C.c_int, [C.c_int32, C.c_int32, _PTR, _PTR, _PTR, _PTR, _PTR,
                                     C.c_double, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                     C.c_int32, _PTR, _PTR, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double), _PTR]),
    "eot_spectral_modes_filtered": (C.c_int, [C.c_int32, C.c_int32, _PTR, _PTR, _PTR, _PTR,
                                              _PTR, C.c_double, C.c_int32, C.c_int32,
                                              C.c_int32, C.c_double, C.c_int32, C.c_int32, _PTR,
                                              _PTR, C.POINTER(C.c_int32),
                                              C.POINTER(C.c_double), _PTR]),
    "eot_plan": (C.c_int, [C.c_int32, C.c_int32, _PTR, _PTR, _PTR, _PTR, _PTR, C.c_double, _PTR,
                           C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                           _PTR]),
    "eot_marginal_error": (C.c_int, [C.c_int32, C.c_int32, _PTR, _PTR, _PTR, _PTR, _PTR,
                                     C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     _PTR]),
    "eot_batch_plan": (C.c_int, [C.c_int32, _PTR, _PTR, _PTR, _PTR, C.POINTER(eot_options),
                                 C.c_int32, C.c_double, C.c_double, C.c_double, _PTR, _PTR]),
    "eot_exp2": (C.c_int, [C.c_int32, _PTR, _PTR, C.c_int32, _PTR, _PTR]),
    "eot_sknr_step": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _PTR, _PTR, _PTR, C.c_double,
                                _PTR, _PTR, _PTR, _PTR, _PTR, _PTR, _PTR, _PTR, _PTR, _PTR,
                                _PTR, C.POINTER(eot_sknr_info), C.c_int32, _PTR]),
    "eot_solve_traced": (C.c_int, [C.POINTER(eot_problem), C.POINTER(eot_options), _PTR, _PTR,
                                   C.POINTER(eot_result), _PTR, C.c_int32,
                                   C.POINTER(C.c_int64)]),
    "eot_batch_tuning": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), _PTR, _PTR]),
    "eot_debug_build": (C.c_int32, []),
    "eot_last_error": (C.c_char_p, []),
    "eot_version": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libeot.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} not found: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list:
    return list(_SIGNATURES)


# ---------------------------------------------------------------------------
# Marshalling helpers
# ---------------------------------------------------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, keep: list, dtype=None):
    """Data pointer of a NumPy array (made contiguous / cast, kept alive) or a torch tensor."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        keep.append(x)
        return x.data_ptr()
    arr = np.ascontiguousarray(x, dtype=dtype)
    keep.append(arr)
    return arr.ctypes.data


def default_options(**kw) -> eot_options:
    o = eot_options()
    load().eot_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def make_problem(a, b, C=None, X=None, Y=None, eps=1e-2, normalize_cost=False, f_init=None,
                 keep: Optional[list] = None, cost_dtype=np.float32, g_init=None, V_init=None,
                 V_out=None) -> eot_problem:
    """Marshal a problem.  ``cost_dtype`` is float64 for ``EOT_PREC_FP64`` solves
    (the cost matrix is read as double there) and float32 otherwise.  ``V_out``
    (n x ell float64, written by the solve) must be a writable contiguous array
    or tensor: it is passed as is."""
    keep = [] if keep is None else keep
    dev = any(_is_torch(x) for x in (a, b, C, X, Y, f_init, g_init, V_init, V_out)
              if x is not None)
    p = eot_problem()
    p.n = int(a.shape[0])
    p.m = int(b.shape[0])
    p.d = 0 if X is None else int(X.shape[1])
    p.a = _ptr(a, keep, np.float64)
    p.b = _ptr(b, keep, np.float64)
    p.C = _ptr(C, keep, cost_dtype)
    p.X = _ptr(X, keep, np.float32)
    p.Y = _ptr(Y, keep, np.float32)
    p.mem = EOT_MEM_DEVICE if dev else EOT_MEM_HOST
    p.normalize_cost = 1 if normalize_cost else 0
    p.eps = float(eps)
    p.f_init = _ptr(f_init, keep, np.float64)
    p.g_init = _ptr(g_init, keep, np.float64)
    p.V_init = _ptr(V_init, keep, np.float64)
    if V_out is not None and not _is_torch(V_out) and not (
            isinstance(V_out, np.ndarray) and V_out.dtype == np.float64
            and V_out.flags.c_contiguous and V_out.flags.writeable):
        raise ValueError("V_out must be a writable C-contiguous float64 array")
    p.V_out = _ptr(V_out, keep, np.float64)
    return p


def last_error() -> str:
    return load().eot_last_error().decode()


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def eot_solve(problem: eot_problem, options: eot_options, f_out, g_out):
    """Call eot_solve; f_out (n) / g_out (m) are float64 NumPy arrays or torch
    tensors matching problem.mem.  Returns (status, eot_result)."""
    res = eot_result()
    keep = []
    st = load().eot_solve(C.byref(problem), C.byref(options), _ptr(f_out, keep),
                          _ptr(g_out, keep), C.byref(res))
    return st, res


TRACE_DTYPE = np.dtype([("eps", np.float64), ("l1", np.float64), ("q_semi", np.float64),
                        ("dq", np.float64), ("iter", np.int32), ("accepted", np.int32)])


def eot_solve_traced(problem: eot_problem, options: eot_options, f_out, g_out, trace_cap: int):
    """Call eot_solve_traced.  Returns (status, eot_result, records, count):
    records is a NumPy structured array (TRACE_DTYPE) of the last
    min(count, trace_cap) iterations, oldest first."""
    res = eot_result()
    keep = []
    rec = np.zeros(max(1, int(trace_cap)), dtype=TRACE_DTYPE)
    cnt = C.c_int64(0)
    st = load().eot_solve_traced(C.byref(problem), C.byref(options), _ptr(f_out, keep),
                                 _ptr(g_out, keep), C.byref(res), rec.ctypes.data,
                                 int(trace_cap), C.byref(cnt))
    return st, res, rec[: min(cnt.value, int(trace_cap))].copy(), cnt.value


def solve(prob, **opts):
    """Solve a ``workloads.Problem`` (host arrays).  Returns (f, g, result dict).
    Warm starts ``f_init``, ``g_init``, ``V_init`` pass through; with
    ``return_modes=True`` (and ell > 0) the result dict holds the modes of the
    returned pair under "V" (eot_problem.V_out); with ``trace=K`` the solve
    runs through eot_solve_traced and the dict holds the last K iteration
    records under "trace" and their total under "trace_count"."""
    keep = []
    f64 = opts.get("prec", EOT_PREC_FP32) == EOT_PREC_FP64
    want_V = opts.pop("return_modes", False)
    trace_cap = int(opts.pop("trace", 0))
    V = np.zeros((prob.a.shape[0], opts.get("ell", 0))) if want_V else None
    p = make_problem(prob.a, prob.b, C=prob.C, X=prob.X, Y=prob.Y, eps=prob.eps,
                     normalize_cost=prob.normalize_cost, f_init=opts.pop("f_init", None),
                     keep=keep, cost_dtype=np.float64 if f64 else np.float32,
                     g_init=opts.pop("g_init", None), V_init=opts.pop("V_init", None), V_out=V)
    o = default_options(**opts)
    f = np.zeros(p.n)
    g = np.zeros(p.m)
    if trace_cap > 0:
        st, res, rec, cnt = eot_solve_traced(p, o, f, g, trace_cap)
    else:
        st, res = eot_solve(p, o, f, g)
    r = res.as_dict()
    r["return_status"] = st
    if st < 0:
        r["error"] = last_error()
    if trace_cap > 0:
        r["trace"] = rec
        r["trace_count"] = cnt
    if want_V:
        r["V"] = V
    return f, g, r


def eot_solve_batch(problems: list, options: eot_options, f_outs: list, g_outs: list):
    n = len(problems)
    arr = (eot_problem * n)(*problems)
    keep = []
    fp = (C.c_void_p * n)(*[_ptr(x, keep) for x in f_outs])
    gp = (C.c_void_p * n)(*[_ptr(x, keep) for x in g_outs])
    res = (eot_result * n)()
    st = load().eot_solve_batch(n, arr, C.byref(options), fp, gp, res)
    return st, list(res)


def eot_ctransform(side: int, n: int, m: int, Cdev, pot, w, shift, eps: float, out,
                   log_ratio=None, stream=None) -> int:
    return load().eot_ctransform(side, n, m, Cdev.data_ptr(), pot.data_ptr(), w.data_ptr(),
                                 None if shift is None else shift.data_ptr(), float(eps),
                                 out.data_ptr(),
                                 None if log_ratio is None else log_ratio.data_ptr(), stream)


def eot_ctransform_noalloc(side: int, n: int, m: int, Cdev, pot, w, shift, eps: float, out,
                           log_ratio=None, stream=None) -> int:
    return load().eot_ctransform_noalloc(side, n, m, Cdev.data_ptr(), pot.data_ptr(),
                                         w.data_ptr(),
                                         None if shift is None else shift.data_ptr(), float(eps),
                                         out.data_ptr(),
                                         None if log_ratio is None else log_ratio.data_ptr(),
                                         stream)


def eot_kapply(side: int, n: int, m: int, k: int, Cdev, f, g, a, b, eps: float, Z, out,
               stream=None) -> int:
    return load().eot_kapply(side, n, m, k, Cdev.data_ptr(), f.data_ptr(), g.data_ptr(),
                             a.data_ptr(), b.data_ptr(), float(eps), Z.data_ptr(),
                             out.data_ptr(), stream)


def eot_cost(n: int, m: int, d: int, X, Y, normalize: bool, Cout, cmax_out=None,
             stream=None) -> int:
    return load().eot_cost(n, m, d, X.data_ptr(), Y.data_ptr(), 1 if normalize else 0,
                           Cout.data_ptr(), None if cmax_out is None else cmax_out.data_ptr(),
                           stream)


def eot_spectral_modes(n, m, Cdev, f, g, a, b, eps, ell, oversample, tol, max_iter,
                       use_V_as_start, V, rho2=None, stream=None):
    it = C.c_int32(0)
    rs = C.c_double(0.0)
    st = load().eot_spectral_modes(n, m, Cdev.data_ptr(), f.data_ptr(), g.data_ptr(),
                                   a.data_ptr(), b.data_ptr(), float(eps), ell, oversample,
                                   float(tol), max_iter, 1 if use_V_as_start else 0,
                                   V.data_ptr(), None if rho2 is None else rho2.data_ptr(),
                                   C.byref(it), C.byref(rs), stream)
    return st, it.value, rs.value


def eot_spectral_modes_filtered(n, m, Cdev, f, g, a, b, eps, ell, oversample, degree, tol,
                                max_iter, use_V_as_start, V, rho2=None, stream=None):
    it = C.c_int32(0)
    rs = C.c_double(0.0)
    st = load().eot_spectral_modes_filtered(n, m, Cdev.data_ptr(), f.data_ptr(), g.data_ptr(),
                                            a.data_ptr(), b.data_ptr(), float(eps), ell,
                                            oversample, degree, float(tol), max_iter,
                                            1 if use_V_as_start else 0, V.data_ptr(),
                                            None if rho2 is None else rho2.data_ptr(),
                                            C.byref(it), C.byref(rs), stream)
    return st, it.value, rs.value


def eot_batch_plan(n, m, eps, options: eot_options, grid_ctas: int, step_ns: float,
                   fix_ns: float, bar_ns: float, has_f_init=None):
    """Host-only schedule of eot_solve_batch: (status, gangs, transposed) for the
    problem sizes n, m and eps (sequences) under the given cost model."""
    import numpy as np
    n = np.ascontiguousarray(n, dtype=np.int32)
    m = np.ascontiguousarray(m, dtype=np.int32)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    k = int(n.shape[0])
    fi = None if has_f_init is None else np.ascontiguousarray(has_f_init, dtype=np.int32)
    gang = np.zeros(k, dtype=np.int32)
    tr = np.zeros(k, dtype=np.int32)
    st = load().eot_batch_plan(k, n.ctypes.data, m.ctypes.data, eps.ctypes.data,
                               None if fi is None else fi.ctypes.data, C.byref(options),
                               int(grid_ctas), float(step_ns), float(fix_ns), float(bar_ns),
                               gang.ctypes.data, tr.ctypes.data)
    return st, gang, tr


def eot_batch_tuning():
    """The batch kernel's tuning on this device: (status, {"step_ns", "fix_ns",
    "bar_ns", "tiles" (7 size classes of m), "tile_ms" (7 x 4)})."""
    st_ns, fx, br = C.c_double(0), C.c_double(0), C.c_double(0)
    tiles = np.zeros(7, dtype=np.int32)
    tms = np.zeros((7, 4), dtype=np.float32)
    st = load().eot_batch_tuning(C.byref(st_ns), C.byref(fx), C.byref(br), tiles.ctypes.data,
                                 tms.ctypes.data)
    return st, {"step_ns": st_ns.value, "fix_ns": fx.value, "bar_ns": br.value,
                "tiles": tiles, "tile_ms": tms}


def eot_exp2(p, q, variant: int, out, stream=None) -> int:
    """Elementwise 2^(p + q) of the float32 passes (device float32 tensors)."""
    return load().eot_exp2(int(p.numel()), p.data_ptr(), q.data_ptr(), int(variant),
                           out.data_ptr(), stream)


def eot_sknr_step(n, m, ell, Cdev, a, b, eps, g, V, f_k=None, h=None, W=None, grad=None,
                  GV=None, WtDW=None, delta=None, f_trial=None, h_trial=None, stream=None,
                  newton_solver=0):
    """One SK-NR iteration from g with modes V (device tensors; outputs are
    optional device tensors).  Returns (status, info dict)."""
    info = eot_sknr_info()

    def ptr(x):
        return None if x is None else x.data_ptr()

    st = load().eot_sknr_step(n, m, ell, Cdev.data_ptr(), a.data_ptr(), b.data_ptr(),
                              float(eps), g.data_ptr(), V.data_ptr(), ptr(f_k), ptr(h), ptr(W),
                              ptr(grad), ptr(GV), ptr(WtDW), ptr(delta), ptr(f_trial),
                              ptr(h_trial), C.byref(info), int(newton_solver), stream)
    d = {k: getattr(info, k) for k, _ in info._fields_}
    d["stage_seconds"] = list(info.stage_seconds)
    return st, d


def eot_plan(n, m, Cdev, f, g, a, b, eps, P=None, stream=None):
    """The coupling of (f, g) into P (optional n x m float32 device tensor) and
    its transport cost, mass and primal value.  Returns (status, cost, mass, primal)."""
    cost, mass, primal = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
    st = load().eot_plan(n, m, Cdev.data_ptr(), f.data_ptr(), g.data_ptr(), a.data_ptr(),
                         b.data_ptr(), float(eps), None if P is None else P.data_ptr(),
                         C.byref(cost), C.byref(mass), C.byref(primal), stream)
    return st, cost.value, mass.value, primal.value


def eot_marginal_error(n, m, Cdev, f, g, a, b, eps, stream=None):
    r = C.c_double(0.0)
    c = C.c_double(0.0)
    st = load().eot_marginal_error(n, m, Cdev.data_ptr(), f.data_ptr(), g.data_ptr(),
                                   a.data_ptr(), b.data_ptr(), float(eps), C.byref(r),
                                   C.byref(c), stream)
    return st, r.value, c.value


def eot_server_simulate(t_arrive, footprint, work, service_s, budget: int, slots: int,
                        max_wait_s: float = 1.0):
    """Host replay of the server's scheduling policy.  Returns (status,
    t_start, t_done) as NumPy arrays."""
    ta = np.ascontiguousarray(t_arrive, dtype=np.float64)
    fp = np.ascontiguousarray(footprint, dtype=np.uint64)
    wk = np.ascontiguousarray(work, dtype=np.float64)
    sv = np.ascontiguousarray(service_s, dtype=np.float64)
    k = int(ta.shape[0])
    t0 = np.zeros(k)
    t1 = np.zeros(k)
    st = load().eot_server_simulate(k, ta.ctypes.data, fp.ctypes.data, wk.ctypes.data,
                                    sv.ctypes.data, int(budget), int(slots), float(max_wait_s),
                                    t0.ctypes.data, t1.ctypes.data)
    return st, t0, t1


class Server:
    """eot_server_* wrapper (host arrays)."""

    def __init__(self, options: eot_options, hbm_budget_bytes: int, max_slots: int):
        h = C.c_void_p()
        st = load().eot_server_create(C.byref(options), int(hbm_budget_bytes), int(max_slots),
                                      C.byref(h))
        if st != EOT_OK:
            raise RuntimeError(f"eot_server_create: {STATUS_NAMES.get(st)} {last_error()}")
        self.h = h
        self._keep = {}

    def submit(self, prob, cloud_id: int = 0, options: Optional[eot_options] = None) -> int:
        keep = []
        p = make_problem(prob.a, prob.b, C=prob.C, X=prob.X, Y=prob.Y, eps=prob.eps,
                         normalize_cost=prob.normalize_cost, keep=keep)
        t = C.c_uint64(0)
        st = load().eot_server_submit_opts(self.h, C.byref(p), C.c_uint64(cloud_id),
                                           None if options is None else C.byref(options),
                                           C.byref(t))
        if st != EOT_OK:
            raise RuntimeError(f"eot_server_submit: {STATUS_NAMES.get(st)} {last_error()}")
        self._keep[t.value] = (prob.n, prob.m)
        return t.value

    def poll(self, ticket: int):
        n, m = self._keep.get(ticket, (1, 1))
        f = np.zeros(n)
        g = np.zeros(m)
        res = eot_result()
        st = load().eot_server_poll(self.h, C.c_uint64(ticket), f.ctypes.data, g.ctypes.data,
                                    C.byref(res))
        if st != EOT_PENDING:
            self._keep.pop(ticket, None)
        return st, f, g, res.as_dict()

    def stats(self):
        p50, p99, sps = C.c_double(), C.c_double(), C.c_double()
        load().eot_server_stats(self.h, C.byref(p50), C.byref(p99), C.byref(sps))
        return p50.value, p99.value, sps.value

    def status(self) -> dict:
        q, r = C.c_int32(), C.c_int32()
        hb, done = C.c_uint64(), C.c_uint64()
        load().eot_server_status(self.h, C.byref(q), C.byref(r), C.byref(hb), C.byref(done))
        return {"queued": q.value, "running": r.value, "hbm_in_use": hb.value,
                "completed": done.value}

    def close(self):
        if self.h:
            load().eot_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
