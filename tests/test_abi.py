"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
function include/rossbi.h declares; the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

from paper_2207_04252_gb300 import build, rossbi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "rossbi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rossbi_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(rossbi.EXPORTS) == declared


def test_status_strings_without_gpu():
    build.build()
    assert rossbi.status_string(rossbi.ROSSBI_OK) == "ok"
    assert "Riemann" in rossbi.status_string(rossbi.ROSSBI_ERR_RIEMANN)


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError):
        rossbi._lib_backup = rossbi._lib
        try:
            rossbi._lib = None
            rossbi.load(str(tmp_path / "missing.so"))
        finally:
            rossbi._lib = rossbi._lib_backup


def test_invalid_descriptions_rejected_without_gpu():
    """Argument checks run before any CUDA call."""
    build.build()
    bad = rossbi.make_desc(rossbi.ROSSBI_GEOM_CYL, (8, 8, 8), (0.5, 0, -0.1), (2.0, 6.28, 0.1),
                           (2, 1, 2), (2, 1, 2))  # cylindrical theta must be periodic
    with pytest.raises(rossbi.RossbiError) as e:
        rossbi.rossbi_init_grid(bad)
    assert e.value.code == rossbi.ROSSBI_ERR_ARG
    zero = rossbi.make_desc(rossbi.ROSSBI_GEOM_BOX, (0, 4, 4), (0, 0, 0), (1, 1, 1), (0, 0, 0), (0, 0, 0))
    with pytest.raises(rossbi.RossbiError):
        rossbi.rossbi_init_grid(zero)


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets that a C
    compiler gives the header's structs (gcc, this machine's ABI)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {
        "rossbi_grid_desc": rossbi.rossbi_grid_desc,
        "rossbi_disc_params": rossbi.rossbi_disc_params,
        "rossbi_dust_params": rossbi.rossbi_dust_params,
        "rossbi_damping_params": rossbi.rossbi_damping_params,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rossbi.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = {}
    for line in out:
        if line:
            name, key, val = line.split()
            c[(name, key)] = int(val)
    for name, cls in structs.items():
        assert ctypes.sizeof(cls) == c[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == c[(name, field)], (name, field)
