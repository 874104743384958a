"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry
point that include/dirac.h declares (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "for", "return")))


def test_library_builds_and_exports_header_symbols():
    from paper_1109_2935_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert "solve" in declared and "dirac_apply" in declared and "schwarz_precondition" in declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1109_2935_gb300 import build
    build.build()
    from paper_1109_2935_gb300 import dirac
    assert sorted(dirac.EXPORTED) == _declared()


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the parameter structs have the sizes and field offsets that a C
    compiler gives the declarations in include/dirac.h."""
    import shutil
    import subprocess

    from paper_1109_2935_gb300 import build
    build.build()
    from paper_1109_2935_gb300 import dirac
    structs = {"dirac_params": dirac.DiracParams, "dirac_solver_params": dirac.SolverParams,
               "dirac_solver_stats": dirac.SolverStats, "dirac_ptc_params": dirac.PtcParams,
               "dirac_ptc_train_params": dirac.PtcTrainParams}
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dirac.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)
