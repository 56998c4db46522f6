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
    assert lib.gauss_filter_2d(None, 4, 4, 2.0, 3, 0, 0, 0, None, None) == m.MORLET_ERR_ARG
    buf = ctypes.create_string_buffer(64)  # a non-null pointer for the size checks (never read)
    assert lib.gauss_filter_2d(buf, 0, 4, 2.0, 3, 0, 0, 0, buf, None) == m.MORLET_ERR_ARG
    assert lib.gauss_filter_2d(buf, 4, 4, 2.0, 3, 3, 0, 0, buf, None) == m.MORLET_ERR_ARG
    assert lib.gauss_filter_2d(buf, 4, 4, 2.0, 3, 0, 0, 7, buf, None) == m.MORLET_ERR_ARG

    assert lib.morlet_plan_set_row_thresholds(None, 128, 4096) == m.MORLET_ERR_ARG
    assert lib.morlet_plan_set_spin_limit(None, 10) == m.MORLET_ERR_ARG
    assert lib.morlet_plan_set_schedule(None, 16, 32, 0, 0) == m.MORLET_ERR_ARG
    assert lib.morlet_plan_schedule(None, None) == m.MORLET_ERR_ARG
    assert lib.morlet_measure_fp64_rate(None, None) == m.MORLET_ERR_ARG


def test_plan_descriptor_errors_without_gpu(built_lib):
    """Descriptor validation happens before any device call: invalid batches, scales, term counts
    and option combinations are refused with the documented status on a machine without a GPU."""
    import paper_2110_11866_gb300 as m
    bad = [
        (dict(lengths=[], sigmas=[8.0]), m.MORLET_ERR_ARG),                 # no signals
        (dict(lengths=[100, 0], sigmas=[8.0]), m.MORLET_ERR_ARG),           # an empty signal
        (dict(lengths=[100], sigmas=[]), m.MORLET_ERR_ARG),                 # no scales
        (dict(lengths=[100], sigmas=[0.25]), m.MORLET_ERR_ARG),             # sigma below 0.5
        (dict(lengths=[100], sigmas=[float("nan")]), m.MORLET_ERR_ARG),     # NaN sigma
        (dict(lengths=[100], sigmas=[8.0], K=13), m.MORLET_ERR_UNSUPPORTED),  # more terms than built
        (dict(lengths=[100], sigmas=[8.0], K=-1), m.MORLET_ERR_ARG),
        (dict(lengths=[100], sigmas=[8.0], K=0), m.MORLET_ERR_ARG),         # automatic K needs fit_tol
        (dict(lengths=[100], sigmas=[8.0], precision=3), m.MORLET_ERR_ARG),
        (dict(lengths=[100], sigmas=[8.0], transform=m.MORLET_ASFT, precision=m.MORLET_FP64),
         m.MORLET_ERR_UNSUPPORTED),                                         # ASFT is FP32 only
        (dict(lengths=[100], sigmas=[8.0], xi=float("inf")), m.MORLET_ERR_ARG),
        (dict(lengths=[100], sigmas=[8.0], norm=2), m.MORLET_ERR_ARG),
        (dict(lengths=[100], sigmas=[8.0], method=3), m.MORLET_ERR_ARG),
        # multiplication method: only the SFT, FP32, rotating form, 2K - 1 terms (3K - 1 with the
        # kappa terms of norm = 1) <= 12
        (dict(lengths=[100], sigmas=[8.0], method=m.MORLET_MULTIPLY, transform=m.MORLET_ASFT),
         m.MORLET_ERR_UNSUPPORTED),
        (dict(lengths=[100], sigmas=[8.0], method=m.MORLET_MULTIPLY, precision=m.MORLET_FP64),
         m.MORLET_ERR_UNSUPPORTED),
        (dict(lengths=[100], sigmas=[8.0], method=m.MORLET_MULTIPLY, norm=1, K=5), m.MORLET_ERR_UNSUPPORTED),
        (dict(lengths=[100], sigmas=[8.0], method=m.MORLET_MULTIPLY, K=7), m.MORLET_ERR_UNSUPPORTED),
        (dict(lengths=[100], sigmas=[8.0], method=m.MORLET_MULTIPLY, form=m.MORLET_FORM_KERNEL),
         m.MORLET_ERR_UNSUPPORTED),
    ]
    for kw, code in bad:
        with pytest.raises(m.MorletError) as err:
            m.morlet_plan(**kw)
        assert err.value.code == code, (kw, err.value.code)
