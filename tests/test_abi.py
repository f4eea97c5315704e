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


def test_checked_library_builds_and_exports_the_same_symbols():
    """The build with CELESTE_CHECK_BOUNDS (device-side bounds checks that record
    CELESTE_ERR_BOUNDS instead of trapping) compiles and exports every declared entry
    point; the binding loads it when the environment sets CELESTE_CHECK_BOUNDS=1."""
    from paper_1801_10277_gb300 import build, celeste
    path = build.build(checked=True)
    assert path == build.LIB_CHECKED and path != build.LIB
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    old = os.environ.get("CELESTE_CHECK_BOUNDS")
    try:
        os.environ["CELESTE_CHECK_BOUNDS"] = "1"
        assert celeste.lib_path() == build.LIB_CHECKED
        os.environ["CELESTE_CHECK_BOUNDS"] = "0"
        assert celeste.lib_path() == build.LIB
    finally:
        if old is None:
            os.environ.pop("CELESTE_CHECK_BOUNDS", None)
        else:
            os.environ["CELESTE_CHECK_BOUNDS"] = old


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


def _header_enums(tmp_path, names):
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include "celeste.h"', 'int main(void) {']
    lines += [f'printf("{n} %lld\\n", (long long){n});' for n in names]
    lines += ['return 0;', '}']
    src = tmp_path / "enums.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "enums"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (ln.split() for ln in out.splitlines())}


def test_header_enums_match_binding(tmp_path):
    """Status codes, schedules, sizes and the catalog / score column layouts: the values
    the header's enums take when compiled equal the binding's constants and the column
    positions of its field-name lists."""
    from paper_1801_10277_gb300 import celeste as c
    status = {"OK": c.OK, "ERR_ARG": c.ERR_ARG, "ERR_NOT_PD": c.ERR_NOT_PD,
              "ERR_NONFINITE": c.ERR_NONFINITE, "ERR_CUDA": c.ERR_CUDA,
              "ERR_TIMEOUT": c.ERR_TIMEOUT, "ERR_NOMEM": c.ERR_NOMEM, "ERR_BOUNDS": c.ERR_BOUNDS,
              "SCHED_COLOUR": c.SCHED_COLOUR, "SCHED_CYCLADES": c.SCHED_CYCLADES,
              "NPARAM": c.NPARAM, "CAT_NFIELD": c.CAT_NFIELD,
              "SCORE_NFIELD": len(c.SCORE_FIELDS)}
    cat = {"CAT_U0": "u0", "CAT_U1": "u1", "CAT_PSTAR": "p_star", "CAT_IS_STAR": "is_star",
           "CAT_RFLUX_MIX": "rflux_mix", "CAT_RFLUX_MIX_SD": "rflux_mix_sd",
           "CAT_EDEV": "e_dev", "CAT_AXIS": "e_axis", "CAT_ANGLE_DEG": "angle_deg",
           "CAT_SCALE": "scale"}
    within = {"CAT_RMAG": "rmag", "CAT_RMAG_SD": "rmag_sd", "CAT_RFLUX": "rflux",
              "CAT_RFLUX_SD": "rflux_sd", "CAT_COLOR": "color_ug", "CAT_COLOR_SD": "color_ug_sd",
              "CAT_MAG": "mag_u", "CAT_MAG_SD": "mag_u_sd"}
    score = {"SCORE_POSITION": "position", "SCORE_MISSED_GAL": "missed_gal",
             "SCORE_MISSED_STAR": "missed_star", "SCORE_BRIGHTNESS": "brightness",
             "SCORE_COLOR": "color_ug", "SCORE_PROFILE": "profile", "SCORE_AXIS": "axis",
             "SCORE_SCALE": "scale", "SCORE_ANGLE_DEG": "angle_deg", "SCORE_N_GAL": "n_gal",
             "SCORE_N_STAR": "n_star"}
    names = list(status) + list(cat) + list(within) + list(score) + \
        ["CAT_STAR", "CAT_GAL", "CAT_TYPE_NFIELD"]
    v = _header_enums(tmp_path, ["CELESTE_" + n for n in names])
    h = {k[len("CELESTE_"):]: x for k, x in v.items()}
    for n, want in status.items():
        assert h[n] == want, n
    for n, field in cat.items():
        assert c.CAT_FIELDS[h[n]] == field, n
    assert c.CAT_FIELDS[h["CAT_STAR"]] == "star_rmag" and c.CAT_FIELDS[h["CAT_GAL"]] == "gal_rmag"
    assert h["CAT_GAL"] - h["CAT_STAR"] == h["CAT_TYPE_NFIELD"]
    for n, field in within.items():
        assert c.CAT_FIELDS[h["CAT_STAR"] + h[n]] == "star_" + field, n
        assert c.CAT_FIELDS[h["CAT_GAL"] + h[n]] == "gal_" + field, n
    for n, field in score.items():
        assert c.SCORE_FIELDS[h[n]] == field, n
