"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/celeste.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "celeste.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(celeste_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1801_10277_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_entry_points():
    from paper_1801_10277_gb300 import celeste
    assert set(celeste.EXPORTS) <= set(declared_functions())


def test_fit_option_defaults_without_gpu():
    from paper_1801_10277_gb300 import celeste
    o = celeste.fit_options()
    assert o.max_iter == 50 and o.delta0 == 1.0 and o.eta == 1e-4


def test_header_constants_match_binding():
    src = open(os.path.join(ROOT, "include", "celeste.h")).read()
    from paper_1801_10277_gb300 import celeste
    assert "CELESTE_FP64 = 0" in src and celeste.FP64 == 0
    assert "CELESTE_FP32_ACC64 = 1" in src and celeste.FP32 == 1
    assert "CELESTE_NPARAM = 44" in src and celeste.NPARAM == 44


def test_struct_layouts_match_the_header(tmp_path):
    """Every public struct of include/celeste.h has, as compiled by the host C compiler,
    the size and field offsets that the ctypes binding assumes."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_1801_10277_gb300 import celeste
    structs = [celeste.celeste_image, celeste.celeste_model, celeste.celeste_patch,
               celeste.celeste_fit_options]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "celeste.h"',
             'int main(void) {']
    for s in structs:
        n = s.__name__
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f in s._fields_:
            lines.append(f'printf("{n} {f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    seen = {}
    for line in out.splitlines():
        n, field, v = line.split()
        seen[(n, field)] = int(v)
    for s in structs:
        n = s.__name__
        assert seen[(n, "size")] == ctypes.sizeof(s), n
        for f in s._fields_:
            assert seen[(n, f[0])] == getattr(s, f[0]).offset, (n, f[0])
