"""The C-ABI library builds, loads and exports every entry point that
include/dg.h declares, and the binding's struct layouts match the header
(checked by compiling a C probe of sizeof/offsetof with gcc).  No GPU calls."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dg.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:dg_status|const char\*|long long)\s+(\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2002_04222_gb300 import build, _lib
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.LIB_PATH


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ("dg_mesh_create", "dg_residual", "dg_jvp", "dg_precond_build", "dg_precond_apply",
              "dg_gmres", "sdirk_step"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(lib, n), n
    from paper_2002_04222_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()
    lib2 = _lib.load(libpath)
    assert lib2.dg_status_string(0) == b"ok"


def test_struct_layouts_match_header():
    from paper_2002_04222_gb300 import _lib
    structs = {"dg_mesh_desc": _lib.MeshDesc, "dg_physics": _lib.Physics,
               "dg_mesh_info_t": _lib.MeshInfo, "dg_prec_cfg": _lib.PrecCfg,
               "dg_gmres_cfg": _lib.GmresCfg, "dg_gmres_stats": _lib.GmresStats,
               "dg_sdirk_cfg": _lib.SdirkCfg, "dg_step_stats": _lib.StepStats,
               "dg_kernel_time": _lib.KernelTime, "dg_guess_cfg": _lib.GuessCfg,
               "dg_tune_result": _lib.TuneResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "probe.c"), os.path.join(d, "probe")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = dict(l.rsplit(" ", 1) for l in out.strip().splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_noalloc_limit_matches_header():
    from paper_2002_04222_gb300 import _lib
    text = open(HEADER).read()
    val = int(re.search(r"#define DG_GMRES_NOALLOC_MAX_DOUBLES (\d+)", text).group(1))
    assert _lib.NOALLOC_MAX_DOUBLES == val
