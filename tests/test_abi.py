"""The C-ABI library builds, loads without a GPU, exports every function that
include/pb.h declares, and the Python binding's struct layouts match the C
compiler's (no compute calls here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pb.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2502_09323_gb300 import build
    build.build()
    from paper_2502_09323_gb300 import _native
    return _native.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][a-z0-9_ ]*\**\s*\**(pb_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ("pb_build_grid", "pb_assemble_coeffs", "pb_coulomb_terms", "pb_solve", "pb_energy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2502_09323_gb300 import _native
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (pb_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(declared_functions()) == set(_native.SIGNATURES)


def test_version_and_error_without_gpu(lib):
    assert lib.pb_version().startswith(b"pbgpu")
    assert lib.pb_last_error() is not None
    # argument errors are reported before any device work
    rc = lib.pb_build_grid(None, None, 0, 0, None, None)
    assert rc == -1
    assert b"NULL" in lib.pb_last_error()


def test_struct_layouts_match_c(tmp_path):
    from paper_2502_09323_gb300 import _native as N
    structs = {"pb_grid_spec": N.GridSpecC, "pb_params": N.ParamsC, "pb_solve_opts": N.SolveOptsC,
               "pb_solve_stats": N.SolveStatsC, "pb_energy_terms": N.EnergyC,
               "pb_grid_info": N.GridInfoC, "pb_engine_result": N.EngineResultC}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(src)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


def test_oracle_and_library_share_no_code():
    """The CUDA sources include nothing from oracle/, and the oracle nothing
    from the package (they only share the seeded input generator)."""
    csrc = os.path.join(ROOT, "paper_2502_09323_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower().replace("oracles", "")
    for f in ("pb_oracle.c", "oracle.py"):
        txt = open(os.path.join(ROOT, "oracle", f)).read()
        assert "paper_2502_09323_gb300" not in txt and "pb.h" not in txt
