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
    assert o.reorth == 0 and o.precond == 0 and o.arith == 0 and o.check_every == 4
    assert abs(o.eta - 2 ** -0.5) < 1e-15 and o.breakdown_eps == 2.0 ** -46
    assert [libcb.cbgmres_format_bytes(f) for f in range(7)] == [8, 4, 2, 2, 1, 4, 2]
    assert libcb.cbgmres_format_bytes(9) == 0


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
