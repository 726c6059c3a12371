"""The C-ABI library builds, loads and exports every entry point that
include/eot.h declares (no compute call: CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "eot.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eot_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_14780_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    import paper_2506_14780_gb300 as pkg
    return pkg.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("eot_solve", "eot_solve_batch", "eot_server_submit", "eot_server_poll",
                     "eot_ctransform", "eot_kapply", "eot_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_covers_the_header():
    from paper_2506_14780_gb300 import eot
    assert sorted(eot.exported_symbols()) == _declared()


def test_version_and_error_without_device(lib):
    from paper_2506_14780_gb300 import eot
    assert b"sm_103a" in lib.eot_version()
    o = eot.default_options()
    assert o.tol == 1e-6 and o.eps_factor == 0.5 and o.prec == eot.EOT_PREC_FP32
    # an invalid problem is rejected on the host before any device work
    import numpy as np
    p = eot.make_problem(np.ones(3) / 3, np.ones(2) / 2, C=np.zeros((3, 2), np.float32), eps=-1.0)
    st, _ = eot.eot_solve(p, o, np.zeros(3), np.zeros(2))
    assert st == eot.EOT_EINVAL
    assert "eps" in eot.last_error()


def test_unimplemented_hessian_is_rejected(lib):
    """The device Newton step uses the D_a form of the Hessian (Eq. d2Q_semi
    with D_r replaced by D_a); asking for the exact form fails on the host."""
    import numpy as np
    from paper_2506_14780_gb300 import eot
    o = eot.default_options(ell=2, hessian=eot.EOT_HESS_EXACT)
    p = eot.make_problem(np.ones(5) / 5, np.ones(4) / 4, C=np.zeros((5, 4), np.float32), eps=0.1)
    st, _ = eot.eot_solve(p, o, np.zeros(5), np.zeros(4))
    assert st == eot.EOT_EINVAL
    assert "D_a" in eot.last_error()


def test_debug_build_compiles_with_its_checks(lib):
    """The bounds-checked build (-DEOT_DEBUG) compiles, exports the same
    symbols and reports itself; the release build reports 0 (no device)."""
    import ctypes
    from paper_2506_14780_gb300 import build
    assert lib.eot_debug_build() == 0
    path = build.build(debug=True)
    dbg = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(dbg, name), name
    dbg.eot_debug_build.restype = ctypes.c_int32
    assert dbg.eot_debug_build() == 1


def test_trace_record_layout_matches_the_header():
    """eot_trace_rec (include/eot.h): four doubles then two int32, 40 bytes;
    the binding's NumPy record must read it field by field."""
    from paper_2506_14780_gb300 import eot
    dt = eot.TRACE_DTYPE
    assert dt.itemsize == 40
    assert [dt.fields[k][1] for k in ("eps", "l1", "q_semi", "dq", "iter", "accepted")] == \
        [0, 8, 16, 24, 32, 36]


def test_warm_start_fields_and_output_checks(lib):
    """eot_problem carries g_init, V_init and V_out after f_init; V_out must be
    a writable C-contiguous float64 array (it is written in place)."""
    import numpy as np
    from paper_2506_14780_gb300 import eot
    names = [n for n, _ in eot.eot_problem._fields_]
    assert names[-4:] == ["f_init", "g_init", "V_init", "V_out"]
    a = np.ones(4) / 4
    C = np.zeros((4, 4), np.float32)
    with pytest.raises(ValueError):
        eot.make_problem(a, a, C=C, V_out=np.zeros((4, 2), np.float32))
    with pytest.raises(ValueError):
        eot.make_problem(a, a, C=C, V_out=np.zeros((2, 4)).T)
    p = eot.make_problem(a, a, C=C, V_out=np.zeros((4, 2)), g_init=np.zeros(4))
    assert p.V_out and p.g_init and not p.V_init
    # an option of the Newton solve outside {0, 1} is rejected on the host
    o = eot.default_options(ell=2, newton_solver=3)
    st, _ = eot.eot_solve(eot.make_problem(a, a, C=C, eps=0.1), o, np.zeros(4), np.zeros(4))
    assert st == eot.EOT_EINVAL and "newton_solver" in eot.last_error()
