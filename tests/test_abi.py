"""The C-ABI library builds, loads and exports every symbol include/combo.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "combo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(combo_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_13624_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 12
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2204_13624_gb300 import combo

    assert sorted(combo.EXPORTS) == declared_symbols()


def test_struct_layouts_match_header():
    """ctypes mirrors of the public structs have the C sizes (checked by compiling a probe)."""
    import subprocess
    import tempfile

    from paper_2204_13624_gb300 import combo

    probe = r'''
#include <stdio.h>
#include "combo.h"
int main(void){printf("%zu %zu %zu %zu\n", sizeof(combo_problem), sizeof(combo_options), sizeof(combo_result), sizeof(combo_ctx_opts));return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(v) for v in subprocess.check_output([exe]).split()]
    assert sizes == [ctypes.sizeof(combo.ProblemS), ctypes.sizeof(combo.OptionsS), ctypes.sizeof(combo.ResultS),
                     ctypes.sizeof(combo.CtxOpts)]


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2204_13624_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".c", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "combo_oracle" not in txt, f
