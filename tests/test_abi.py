"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/tacauchy.h declares (no compute: runs without a GPU)."""
import os
import re

from paper_2606_20426_gb300 import build as b
from paper_2606_20426_gb300 import tacauchy

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "tacauchy.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z_A-Z0-9]+)\s*\(", src)))


def test_header_matches_binding_list():
    assert declared() == sorted(tacauchy.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    b.build()
    lib = tacauchy.load()
    for name in declared():
        assert hasattr(lib, name), name
    assert lib.tc_status_str(0) == b"ok"
    assert lib.tc_status_str(6) == b"line search found no decrease"


def test_invalid_arguments_rejected_without_gpu_work():
    lib = tacauchy.load()
    import ctypes
    h = ctypes.c_void_p()
    # null mesh -> TC_ERR_INVALID_ARG before any device call
    assert lib.tc_create_scene(None, None, None, 0, None, None, None, None, None, None, ctypes.byref(h)) == 1
    assert lib.tc_step(None, None) == 1
    assert lib.tc_stress_from_F(None, -1, 3e5, 0.45, None, None) == 1


def test_new_entry_points_reject_null_handles_without_gpu_work():
    lib = tacauchy.load()
    assert lib.tc_pressure_map(None, None, None, None) == 1
    assert lib.tc_depth_map(None, None, None, None) == 1
    assert lib.tc_vertex_forces(None, None, None, None, None) == 1
    assert lib.tc_force_pressure_map(None, None, None, None) == 1
    assert lib.tc_extract_batch(None, 0, None, None, None) == 0      # an empty batch is a no-op
    assert lib.tc_extract_batch(None, 2, None, None, None) == 1
    assert lib.tc_extract_batch(None, -1, None, None, None) == 1
