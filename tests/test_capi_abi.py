"""The C-ABI library builds, loads without a GPU, exports every function
declared in include/lbm.h, and the ctypes binding's struct layouts match the
header (checked against gcc's sizeof/offsetof)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1607_02874_gb300 import build, lbm

    build.build()
    return lbm.library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lbm_step" in names and "lbm_create_geometry" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1607_02874_gb300 import lbm

    missing = [n for n in declared_functions() if n not in lbm.SIGNATURES]
    assert not missing, missing


def test_error_strings_without_gpu(lib):
    assert lib.lbm_error_string(0) == b"ok"
    assert b"argument" in lib.lbm_error_string(-1)
    # argument checks happen before any CUDA call
    rc = lib.lbm_create_geometry(None, None, None, None)
    assert rc == -1
    assert lib.lbm_step(None, 1) == -1


def test_struct_layouts_match_header(tmp_path):
    from paper_1607_02874_gb300 import lbm

    structs = {"lbm_geometry_desc": lbm.lbm_geometry_desc, "lbm_params": lbm.lbm_params, "lbm_obs": lbm.lbm_obs,
               "lbm_allocator": lbm.lbm_allocator}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    for line in out:
        if not line:
            continue
        sname, field, val = line.split()
        cls = structs[sname]
        if field == "size":
            assert ctypes.sizeof(cls) == int(val), sname
        else:
            assert getattr(cls, field).offset == int(val), (sname, field)
