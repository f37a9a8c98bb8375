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
    # the allocation-free diagnostics and the barrier fault hook refuse a null
    # handle before touching CUDA
    assert lib.sww_mass_energy_static(None, None, None, None) == -1
    lib.sww_last_error(buf, 256)
    assert b"null handle" in buf.value
    assert lib.sww_barrier_fault(None, 0, -1) == -1
    # the live-node count reads host memory only; a null handle or output is refused
    n = ctypes.c_int64(7)
    assert lib.sww_live_nodes(None, ctypes.byref(n)) == -1 and n.value == 7


def test_config_checks_without_compute():
    """Each configuration field out of its range is refused before any device
    call: the prescribed-velocity flag, the threshold regime, the stage mode,
    a zero mean depth without a prescribed velocity, a negative viscosity, a
    negative eps, a patch side other than 4, 8 or 16."""
    import ctypes
    import paper_1404_0405_gb300 as sww
    lib = sww.load()

    def cfg(**kw):
        c = sww.Config(2, 4, 6.371e6, 7.292e-5, 9.80616, 1e4, 8, 0, 0.8, 1e-2)
        for k, v in kw.items():
            setattr(c, k, v)
        return c

    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(256)
    for kw, word in [({"advect": 2}, b"advect"), ({"regime": 3}, b"regime"), ({"persistent": 4}, b"persistent"),
                     ({"H": 0.0}, b"H"), ({"nu": -1.0}, b"nu"), ({"eps": -1.0}, b"eps"),
                     ({"patch": 2}, b"patch"), ({"patch": 32}, b"patch")]:
        assert lib.sww_create(ctypes.byref(cfg(**kw)), None, ctypes.byref(h)) == -1, kw
        lib.sww_last_error(buf, 256)
        assert word in buf.value, (kw, buf.value)


def test_header_is_plain_c_and_links():
    """include/sww.h compiles as pedantic C99, and a C program using it links
    against the library (no GPU needed to build; examples/step.c)."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc")
    if gcc is None:
        import pytest
        pytest.skip("no C compiler")
    path = build()
    with tempfile.TemporaryDirectory() as d:
        obj, exe = os.path.join(d, "step.o"), os.path.join(d, "step")
        subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), "-c", os.path.join(ROOT, "examples", "step.c"), "-o", obj],
                       check=True)
        subprocess.run([gcc, obj, "-L", os.path.dirname(path), "-lsww", "-lm", "-o", exe], check=True)
