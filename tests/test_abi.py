"""The C-ABI library builds, loads without a GPU, and exports every entry point that
include/*.h declares; status strings and option defaults are callable host logic."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(cbg\w*)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libcb():
    import paper_2009_12101_gb300 as cb
    cb.ensure_built()
    return cb.lib()


def test_every_declared_symbol_is_exported(libcb):
    names = _declared_functions()
    assert len(names) >= 15, names
    missing = [n for n in names if not hasattr(libcb, n)]
    assert not missing, missing


def test_status_strings_and_defaults(libcb):
    import paper_2009_12101_gb300 as cb
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        s = libcb.cbgmres_status_string(code)
        assert isinstance(s, bytes) and len(s) > 3
    assert libcb.cbgmres_status_string(12345) == b"unknown status"
    o = cb.Options()
    libcb.cbgmres_options_default(C.byref(o))
    assert o.reorth == 0 and o.precond == 0 and o.arith == 0 and o.check_every == 4 and o.ortho == 0
    assert abs(o.eta - 2 ** -0.5) < 1e-15 and o.breakdown_eps == 2.0 ** -46
    assert [libcb.cbgmres_format_bytes(f) for f in range(7)] == [8, 4, 2, 2, 1, 4, 2]
    assert libcb.cbgmres_format_bytes(9) == 0


def test_options_struct_size_matches_the_binding(libcb):
    """cbgmres_options_default clears the whole C struct: on a buffer filled with a
    pattern it must write exactly the binding's sizeof(Options) bytes (the trailing
    fields default to zero), no fewer and no more."""
    import paper_2009_12101_gb300 as cb
    size = C.sizeof(cb.Options)
    buf = (C.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    libcb.cbgmres_options_default(C.cast(buf, C.POINTER(cb.Options)))
    assert all(b == 0xAB for b in buf[size:])
    assert all(b == 0 for b in buf[size - 8:size])


def test_argument_errors_need_no_gpu(libcb):
    """Entry points reject invalid arguments before touching the device."""
    import paper_2009_12101_gb300 as cb
    h = C.c_void_p()
    assert libcb.cbgmres_create(None, 10, 0, None, C.byref(h)) == -1
    csr = cb.Csr(0, 0, None, None, None, 0, 0)
    assert libcb.cbgmres_create(C.byref(csr), 10, 0, None, C.byref(h)) == -1
    assert libcb.cbgmres_solve(None, None, None, 1e-10, 10, None) == -1
    scale = C.c_double()
    assert libcb.cbg_encode(17, 4, None, 1.0, None, C.byref(scale), None) == -1
    assert libcb.cbg_decode(0, -1, None, 1.0, None, None) == -1


def test_ortho_option_is_checked_before_the_device(libcb):
    """An unknown orthogonalisation is an argument error; the batched solver (CGS only)
    reports MGS as unsupported, and so does the single-system solver for MGS with
    conditional re-orthogonalisation; eta outside (0, 1] is an argument error there. All
    are decided before any device call."""
    import numpy as np
    import paper_2009_12101_gb300 as cb
    rp = np.array([0, 1, 2], np.int32); ci = np.array([0, 1], np.int32); va = np.array([2.0, 3.0])
    csr = cb.Csr(2, 2, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0, 0)
    o = cb.Options()
    libcb.cbgmres_options_default(C.byref(o))
    o.ortho = 7
    h = C.c_void_p()
    assert libcb.cbgmres_create(C.byref(csr), 10, 0, C.byref(o), C.byref(h)) == -1
    o.ortho = cb.ORTHO["mgs"]
    bt = C.c_void_p()
    assert libcb.cbgmres_create_batched(1, C.byref(csr), 10, 1, C.byref(o), C.byref(bt)) == -6
    # conditional re-orthogonalisation: CGS only, eta in (0, 1]
    o.reorth = cb.REORTH["conditional"]
    assert libcb.cbgmres_create(C.byref(csr), 10, 0, C.byref(o), C.byref(h)) == -6
    o.ortho = cb.ORTHO["cgs"]
    for bad_eta in (0.0, -0.5, 1.5, float("nan")):
        o.eta = bad_eta
        assert libcb.cbgmres_create(C.byref(csr), 10, 0, C.byref(o), C.byref(h)) == -1


def test_debug_library_builds_and_exports_every_symbol():
    """The debug variant (-DCBG_DEBUG: guard tails, SpMV index checks) compiles for sm_103a
    and exports the same entry points."""
    from paper_2009_12101_gb300 import build as cbuild
    path = cbuild.build(debug=True)
    assert path.endswith("libcbgmres_debug.so")
    L = C.CDLL(path)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing
