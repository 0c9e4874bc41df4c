"""The C-ABI library builds for sm_103a, loads, and exports every function
include/trig.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "trig.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(trig_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1411_3968_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert "trig_create" in names and "trig_batch_run" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib_path):
    from paper_1411_3968_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_binding_struct_sizes_match_header():
    from paper_1411_3968_gb300 import _lib
    assert ctypes.sizeof(_lib.trig_params) == 40
    assert ctypes.sizeof(_lib.trig_slice_dev) == 80
    assert _lib.HIT_DTYPE.itemsize == 16 and _lib.TRIGGER_DTYPE.itemsize == 16
    assert _lib.WINDOW_DTYPE.itemsize == 32 and _lib.STATS_DTYPE.itemsize == 40


def test_oracle_and_generator_build():
    import oracle
    import workload
    assert os.path.exists(oracle.build())
    assert os.path.exists(workload.build())


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1411_3968_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "oracle.h" not in text and "liboracle" not in text, f
