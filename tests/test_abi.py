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
