"""CPU-only checks of the boundary: the CUDA library builds for sm_103a, loads without a GPU and exports
every function include/morlet_sft.h declares; the Python binding exposes the same names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "morlet_sft.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2110_11866_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("morlet_plan", "morlet_forward", "morlet_backward", "gauss_smooth", "morlet_plan_destroy",
              "morlet_strerror", "morlet_last_device_error"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(built_lib):
    import paper_2110_11866_gb300 as m
    for n in _declared():
        assert n in m.EXPORTED_SYMBOLS and hasattr(m, n), n


def test_strerror_and_argument_errors_without_gpu(built_lib):
    """Status strings and argument validation need no device."""
    import paper_2110_11866_gb300 as m
    assert m.morlet_strerror(m.MORLET_ERR_TIMEOUT).startswith("a kernel timed out")
    assert m.morlet_strerror(0) == "ok"
    lib = m.lib()
    h = ctypes.c_void_p()
    assert lib.morlet_plan(ctypes.byref(h), None, None) == m.MORLET_ERR_ARG
    assert lib.morlet_forward(None, None, None, None) == m.MORLET_ERR_ARG
    assert lib.gauss_smooth(None, 0, 1.0, 3, 0, 0, None, None) == m.MORLET_ERR_ARG

    assert lib.morlet_plan_set_row_thresholds(None, 128, 4096) == m.MORLET_ERR_ARG
    assert lib.morlet_plan_set_spin_limit(None, 10) == m.MORLET_ERR_ARG
