"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/gks.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gks_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_09058_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gks_create", "gks_solve", "gks_sync", "gks_destroy", "gks_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gks_[a-z_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_library_loads_and_binds(libpath):
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(lib, n)
    from paper_2606_09058_gb300 import gks
    assert gks.load() is not None


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2606_09058_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "gks_oracle" not in txt, f


def test_binding_refuses_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("CUDA present")
    from paper_2606_09058_gb300 import gks
    with pytest.raises(RuntimeError):
        gks.Context(0)


def test_python_options_match_the_header_layout(tmp_path):
    """gks_opts as the C compiler lays it out (offset of every field, total size) equals the
    ctypes mirror the binding passes to gks_create."""
    from paper_2606_09058_gb300 import gks
    fields = [f for f, _ in gks._Opts._fields_]
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gks.h"\nint main(void) {\n' +
                    "".join(f'  printf("{f} %zu\\n", offsetof(gks_opts, {f}));\n' for f in fields) +
                    '  printf("sizeof %zu\\n", sizeof(gks_opts));\n  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n") if l)
    for f in fields:
        assert int(got[f]) == getattr(gks._Opts, f).offset, f
    assert int(got["sizeof"]) == ctypes.sizeof(gks._Opts)
