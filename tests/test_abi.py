"""The C-ABI library builds, loads and exports every symbol include/mcsteklov.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mcsteklov.h")).read()
    return sorted(set(re.findall(r"\b(mcs_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2606_05581_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    lib.mcs_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.mcs_version()


def test_default_params_and_argument_checks_without_gpu():
    import paper_2606_05581_b300 as mcs
    p = mcs.default_params()
    assert p.eps == 1e-3 and p.cap_deg == 2.5 and p.bisect_iters == 10 and p.max_steps == 1024
    # invalid calls are rejected before any launch
    st = mcs.lib().mcs_build_bvh(None, 0, None, 0, None, ctypes.byref(ctypes.c_void_p()))
    assert st == -1 and b"NULL" in mcs.lib().mcs_last_error()
