"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function that include/sww.h declares (no compute call is made here)."""
import os
import re

from paper_1404_0405_gb300.buildlib import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "sww.h")).read()
    return sorted(set(re.findall(r"^int (sww_\w+)\(", src, flags=re.M)))


def test_header_declares_the_api():
    names = declared()
    assert "sww_create" in names and "sww_step" in names and "sww_adapt" in names
    assert len(names) >= 14


def test_library_exports_declared_symbols():
    import ctypes
    import paper_1404_0405_gb300 as sww
    path = build()
    lib = ctypes.CDLL(path)
    for name in declared():
        assert hasattr(lib, name), name
    assert sorted(sww.EXPORTS) == declared()


def test_error_path_without_compute():
    """Argument checks happen before any device call."""
    import ctypes
    import paper_1404_0405_gb300 as sww
    lib = sww.load()
    h = ctypes.c_void_p()
    bad = sww.Config(5, 3, 6.371e6, 7.292e-5, 9.80616, 1e4, 8, 0, 0.8, 1e-2)
    assert lib.sww_create(ctypes.byref(bad), None, ctypes.byref(h)) == -1
    buf = ctypes.create_string_buffer(256)
    lib.sww_last_error(buf, 256)
    assert b"jmin" in buf.value
    assert lib.sww_step(None, 1.0, 1, 1) == -1
