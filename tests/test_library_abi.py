"""The C-ABI library builds for sm_103a, loads, and exports every symbol
that include/ms.h declares (no compute calls: no GPU needed)."""
import re
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_builds_and_exports_header_symbols():
    from paper_2209_04487_gb300 import build
    build.build()
    import ctypes
    lib = ctypes.CDLL(build.LIB)
    hdr = open(os.path.join(ROOT, "include", "ms.h")).read()
    names = set(re.findall(r"\b(ms_[a-z_]+)\s*\(", hdr))
    assert names, "no declarations found"
    for n in sorted(names):
        assert hasattr(lib, n), n
    from paper_2209_04487_gb300 import binding
    assert set(binding.EXPORTED) == names


def test_status_strings():
    from paper_2209_04487_gb300 import binding as B
    codes = (B.MS_OK, B.MS_EINVAL, B.MS_ENOMEM, B.MS_ECUDA, B.MS_ENUMERIC, B.MS_ETIMEOUT,
             B.MS_EUNSUPPORTED, B.MS_EIO)
    texts = [B.LIB.ms_status_string(code) for code in codes]
    assert all(texts) and b"unknown status" not in texts and len(set(texts)) == len(codes)


def test_header_is_c99_and_binding_layouts_match(tmp_path):
    """include/ms.h compiles as plain C99 without warnings, and every
    descriptor struct has the same size and field offsets in C as in the
    ctypes binding (a mismatch would pass garbage across the boundary)."""
    import ctypes
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2209_04487_gb300 import binding as B
    structs = {"ms_grid_desc": B.GridDesc, "ms_materials_desc": B.MaterialsDesc, "ms_species": B.SpeciesDesc,
               "ms_molecules_desc": B.MoleculesDesc, "ms_options": B.Options}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ms.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
