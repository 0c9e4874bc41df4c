"""The C-ABI library builds for sm_103a, loads, and exports every function
include/trig.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(trig_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


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


def _c_layout(structs):
    """sizeof and field offsets of the header's structs, from gcc."""
    import subprocess
    import tempfile
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "trig.h"', '#include "trig_array.h"',
             'int main(void) {']
    for name, fields in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append('return 0; }')
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (ln.split() for ln in out.splitlines())}


def test_binding_struct_sizes_match_header():
    from paper_1411_3968_gb300 import _lib
    ct = {"trig_params": _lib.trig_params, "trig_slice_dev": _lib.trig_slice_dev, "trig_result": _lib.trig_result,
          "trig_slice_events": _lib.trig_slice_events, "trig_tune_result": _lib.trig_tune_result,
          "trig_geometry": _lib.trig_geometry, "trig_array_params": _lib.trig_array_params,
          "trig_array_out": _lib.trig_array_out}
    np_types = {"trig_hit": _lib.HIT_DTYPE, "trig_trigger": _lib.TRIGGER_DTYPE, "trig_window": _lib.WINDOW_DTYPE,
                "trig_slice_stats": _lib.STATS_DTYPE, "trig_array_seed": _lib.ASEED_DTYPE,
                "trig_array_stats": _lib.ASTATS_DTYPE, "trig_trace_rec": _lib.TRACE_DTYPE}
    c_names = {"trig_hit": ["t_ns", "pmt", "charge", "reserved"], "trig_trigger": ["t_ns", "pmt", "charge", "count"],
               "trig_window": ["lo_ns", "hi_ns", "n_hits", "n_triggers"],
               "trig_slice_stats": ["status", "flags", "n_hits", "n_seeds", "n_triggers", "n_windows", "n_events"],
               "trig_array_seed": ["t_ns", "pmt", "tower", "n_towers"],
               "trig_array_stats": ["n_tower_triggers", "n_selected", "n_windows", "n_hits", "flags", "status"],
               "trig_trace_rec": ["slice_id", "batch", "batch_slices", "n_pmt", "n_hits", "status", "continuation",
                                  "t_submit_ns", "t_queued_ns", "t_launch_ns", "t_stats_ns", "t_done_ns", "device_ms",
                                  "copy_wait_us"]}
    lay = _c_layout({**{k: [f for f, _ in v._fields_] for k, v in ct.items()}, **c_names})
    for name, cls in ct.items():
        assert ctypes.sizeof(cls) == lay[name], name
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == lay[f"{name}.{f}"], (name, f)
    for name, dt in np_types.items():
        assert dt.itemsize == lay[name], name
        for (f, _), cf in zip(dt.descr, c_names[name]):
            assert dt.fields[f][1] == lay[f"{name}.{cf}"], (name, f)


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
