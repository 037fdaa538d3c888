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


def test_ctypes_structs_match_the_header(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal the C compiler's."""
    import subprocess
    import paper_2606_05581_b300 as mcs
    structs = {"mcs_params": mcs.Params, "mcs_rows": mcs.Rows, "mcs_outputs": mcs.Outputs, "mcs_stats": mcs.Stats,
               "mcs_batch_item": mcs.BatchItem, "mcs_tune_trial": mcs.TuneTrial, "mcs_eig_params": mcs.EigParams,
               "mcs_eig_stats": mcs.EigStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mcsteklov.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
