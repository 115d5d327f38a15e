"""The C-ABI library builds, loads and exports every entry point that
include/af.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "af.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(af_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libaf():
    from paper_2508_06273_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["af_create", "af_set_state", "af_step", "af_get_state", "af_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(libaf):
    missing = [n for n in declared_functions() if not hasattr(libaf, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2508_06273_gb300 import af

    assert sorted(af.EXPORTS) == declared_functions()


def test_library_is_built_for_sm_103a(libaf):
    from paper_2508_06273_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_oracle_is_independent_of_the_library():
    """The oracle and the CUDA path share no code: neither imports or
    includes the other."""
    osrc = "".join(open(os.path.join(ROOT, "oracle", f)).read() for f in ("afo.c", "afo.h", "afo.py", "__init__.py"))
    assert "paper_2508_06273_gb300" not in osrc and "af_common" not in osrc and "af.h\"" not in osrc
    pkg = os.path.join(ROOT, "paper_2508_06273_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "afo" not in text, f
