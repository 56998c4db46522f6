"""Python binding of the GB300 SFT/ASFT Morlet library (C ABI in include/morlet_sft.h).

Argument marshalling only: every step of the transform runs in the CUDA library
(_build/libmorlet_sft.so). If that library is missing the calls raise; there is no CPU path.
PyTorch, when used, only provides device memory and streams.

Names follow the C ABI: morlet_plan, morlet_forward, morlet_backward, gauss_smooth,
morlet_plan_destroy, morlet_strerror, morlet_last_device_error, morlet_plan_info, morlet_plan_stats.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "MORLET_OK", "MORLET_ERR_ARG", "MORLET_ERR_UNSUPPORTED", "MORLET_ERR_CUDA", "MORLET_ERR_TIMEOUT",
    "MORLET_ERR_NOMEM", "MORLET_DIRECT", "MORLET_GAUSS", "MORLET_MULTIPLY", "MORLET_SFT", "MORLET_ASFT", "MORLET_FP32_PLAIN",
    "MORLET_FP32_COMP", "MORLET_FP64", "MORLET_FORM_AUTO", "MORLET_FORM_KERNEL", "MORLET_FORM_ROTATING",
    "MORLET_FLAG_NO_GRAPH", "MORLET_FLAG_AUTOTUNE", "MORLET_FLAG_NO_HALO", "MORLET_FLAG_EDGE", "MORLET_FLAG_NO_ADJOINT",
    "MorletError", "lib", "lib_path",
    "morlet_plan", "morlet_forward", "morlet_backward", "gauss_smooth", "morlet_plan_destroy",
    "morlet_strerror", "morlet_last_device_error", "morlet_plan_info", "morlet_plan_stats",
    "morlet_plan_set_spin_limit", "morlet_debug_skip_tickets", "EXPORTED_SYMBOLS", "source_hash",
    "morlet_forward_noalloc", "morlet_plan_set_row_thresholds", "gauss_filter_2d",
    "morlet_plan_set_schedule", "morlet_plan_schedule", "morlet_measure_fp64_rate",
]

MORLET_OK, MORLET_ERR_ARG, MORLET_ERR_UNSUPPORTED, MORLET_ERR_CUDA, MORLET_ERR_TIMEOUT, MORLET_ERR_NOMEM = (
    0, -1, -2, -3, -4, -5)
MORLET_DIRECT, MORLET_GAUSS, MORLET_MULTIPLY = 0, 1, 2
MORLET_SFT, MORLET_ASFT = 0, 1
MORLET_FP32_PLAIN, MORLET_FP32_COMP, MORLET_FP64 = 0, 1, 2
MORLET_FORM_AUTO, MORLET_FORM_KERNEL, MORLET_FORM_ROTATING = 0, 1, 2
MORLET_FLAG_NO_GRAPH, MORLET_FLAG_AUTOTUNE, MORLET_FLAG_NO_HALO, MORLET_FLAG_EDGE, MORLET_FLAG_NO_ADJOINT = 1, 2, 4, 8, 16

EXPORTED_SYMBOLS = [
    "morlet_plan", "morlet_forward", "morlet_backward", "gauss_smooth", "morlet_plan_destroy",
    "morlet_strerror", "morlet_last_device_error", "morlet_plan_info", "morlet_plan_stats",
    "morlet_plan_set_spin_limit", "morlet_debug_skip_tickets", "morlet_forward_noalloc",
    "morlet_plan_set_row_thresholds", "gauss_filter_2d", "morlet_plan_set_schedule", "morlet_plan_schedule",
    "morlet_measure_fp64_rate",
]

_HERE = os.path.dirname(os.path.abspath(__file__))


def source_hash() -> str:
    """SHA-1 of the CUDA sources (identifies the kernel a profile was taken on)."""
    import glob
    import hashlib
    h = hashlib.sha1()
    for f in sorted(glob.glob(os.path.join(_HERE, "csrc", "*"))):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def lib_path() -> str:
    return os.path.join(_HERE, "_build", "libmorlet_sft.so")


class MorletError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {morlet_strerror(code)} ({code})")


class _Desc(ctypes.Structure):
    _fields_ = [
        ("n_signals", ctypes.c_int64), ("lengths", ctypes.c_void_p),
        ("n_scales", ctypes.c_int32), ("sigmas", ctypes.c_void_p),
        ("xi", ctypes.c_double), ("K", ctypes.c_int32), ("fit_tol", ctypes.c_double),
        ("method", ctypes.c_int32), ("transform", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("norm", ctypes.c_int32), ("n0", ctypes.c_int32), ("window_mult", ctypes.c_double),
        ("deriv", ctypes.c_int32), ("form", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("spin_limit", ctypes.c_int64),
    ]


_lib = None


def lib():
    """Load the CUDA library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built ({path}); run paper_2110_11866_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.morlet_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Desc), vp]
    L.morlet_forward.argtypes = [vp, vp, vp, vp]
    L.morlet_backward.argtypes = [vp, vp, vp, vp]
    L.gauss_smooth.argtypes = [vp, i64, ctypes.c_double, i32, i32, i32, vp, vp]
    L.morlet_plan_destroy.argtypes = [vp]
    L.morlet_plan_destroy.restype = None
    L.morlet_strerror.argtypes = [ctypes.c_int]
    L.morlet_strerror.restype = ctypes.c_char_p
    L.morlet_last_device_error.argtypes = [vp, vp]
    L.morlet_plan_info.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(i32)]
    L.morlet_plan_stats.argtypes = [vp, ctypes.POINTER(i64)]
    L.morlet_plan_set_spin_limit.argtypes = [vp, i64]
    L.morlet_debug_skip_tickets.argtypes = [vp, i64]
    L.morlet_plan_set_row_thresholds.argtypes = [vp, i64, i64]
    L.gauss_filter_2d.argtypes = [vp, i64, i64, ctypes.c_double, i32, i32, i32, i32, vp, vp]
    L.morlet_forward_noalloc.argtypes = [vp, i64, ctypes.c_double, ctypes.c_double, i32, vp, vp]
    L.morlet_plan_set_schedule.argtypes = [vp, i32, i32, i32, i32]
    L.morlet_plan_schedule.argtypes = [vp, ctypes.POINTER(i64)]
    L.morlet_measure_fp64_rate.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
    for f in ("morlet_plan", "morlet_forward", "morlet_backward", "gauss_smooth", "morlet_last_device_error",
              "morlet_plan_info", "morlet_plan_stats", "morlet_plan_set_spin_limit", "morlet_debug_skip_tickets",
              "morlet_forward_noalloc", "morlet_plan_set_row_thresholds", "gauss_filter_2d",
              "morlet_plan_set_schedule", "morlet_plan_schedule", "morlet_measure_fp64_rate"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _stream(s):
    """A stream as a void*: None -> current torch stream if torch has CUDA, else the default stream."""
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def _ptr(p):
    if hasattr(p, "data_ptr"):
        return ctypes.c_void_p(p.data_ptr())
    return ctypes.c_void_p(int(p))


def _check(code, what):
    if code != MORLET_OK:
        raise MorletError(code, what)


def morlet_strerror(code: int) -> str:
    return lib().morlet_strerror(int(code)).decode()


class Plan:
    """Owns a morlet_plan_t; destroyed with morlet_plan_destroy (or when garbage collected)."""

    def __init__(self, handle, lengths, sigmas, desc):
        self.handle = handle
        self.lengths = list(lengths)
        self.sigmas = list(sigmas)
        self.desc = desc

    @property
    def n_samples(self):
        return sum(self.lengths)

    @property
    def n_outputs(self):
        return sum(self.lengths) * len(self.sigmas)

    def __del__(self):
        try:
            if self.handle:
                morlet_plan_destroy(self)
        except Exception:
            pass


def morlet_plan(lengths, sigmas, xi=6.0, K=4, fit_tol=0.0, method=MORLET_DIRECT, transform=MORLET_SFT,
                precision=MORLET_FP32_COMP, norm=0, n0=0, window_mult=0.0, deriv=0, form=MORLET_FORM_AUTO,
                flags=0, spin_limit=0, stream=None) -> Plan:
    import numpy as np
    lens = np.ascontiguousarray(lengths, dtype=np.int64)
    sig = np.ascontiguousarray(sigmas, dtype=np.float64)
    d = _Desc(len(lens), lens.ctypes.data, len(sig), sig.ctypes.data, float(xi), int(K), float(fit_tol),
              int(method), int(transform), int(precision), int(norm), int(n0), float(window_mult), int(deriv),
              int(form), int(flags), int(spin_limit))
    h = ctypes.c_void_p()
    _check(lib().morlet_plan(ctypes.byref(h), ctypes.byref(d), _stream(stream)), "morlet_plan")
    return Plan(h, lens.tolist(), sig.tolist(), dict(xi=xi, K=K, method=method, transform=transform,
                                                     precision=precision, norm=norm, n0=n0, deriv=deriv,
                                                     form=form, flags=flags))


def morlet_forward(plan: Plan, x, W, stream=None):
    _check(lib().morlet_forward(plan.handle, _ptr(x), _ptr(W), _stream(stream)), "morlet_forward")


def morlet_backward(plan: Plan, gW, gx, stream=None):
    _check(lib().morlet_backward(plan.handle, _ptr(gW), _ptr(gx), _stream(stream)), "morlet_backward")


def gauss_smooth(x, N, sigma, P, deriv, precision, y, stream=None):
    _check(lib().gauss_smooth(_ptr(x), int(N), float(sigma), int(P), int(deriv), int(precision), _ptr(y),
                              _stream(stream)), "gauss_smooth")


def gauss_filter_2d(img, ny, nx, sigma, P, deriv_y, deriv_x, precision, out, stream=None):
    """Separable Gaussian filtering of a [ny][nx] device image (G along y and x, or their
    derivatives): batched 1-D transforms over the rows and the columns."""
    _check(lib().gauss_filter_2d(_ptr(img), int(ny), int(nx), float(sigma), int(P), int(deriv_y), int(deriv_x),
                                 int(precision), _ptr(out), _stream(stream)), "gauss_filter_2d")


def morlet_plan_destroy(plan: Plan):
    if plan.handle:
        lib().morlet_plan_destroy(plan.handle)
        plan.handle = None


def morlet_last_device_error(plan: Plan, stream=None) -> int:
    return int(lib().morlet_last_device_error(plan.handle, _stream(stream)))


def morlet_plan_info(plan: Plan, s: int) -> dict:
    L = ctypes.c_int64()
    p0 = ctypes.c_int32()
    K = ctypes.c_int32()
    n0 = ctypes.c_int32()
    m = (ctypes.c_double * 12)()
    l = (ctypes.c_double * 12)()
    _check(lib().morlet_plan_info(plan.handle, int(s), ctypes.byref(L), ctypes.byref(p0), ctypes.byref(K), m, l,
                                  ctypes.byref(n0)), "morlet_plan_info")
    return dict(L=L.value, p0=p0.value, K=K.value, m=list(m)[:K.value], l=list(l)[:K.value], n0=n0.value)


def morlet_plan_stats(plan: Plan) -> dict:
    o = (ctypes.c_int64 * 15)()
    _check(lib().morlet_plan_stats(plan.handle, o), "morlet_plan_stats")
    keys = ["threads", "items", "ctas", "work_items", "sub_tiles", "rows_lookback", "rows_window", "launches",
            "rows_start_state", "prefix_items", "rows_lane_chunk", "lane_chunk_items", "lane_chunk_max_L",
            "start_state_min_L", "start_state_window_sums"]
    return dict(zip(keys, list(o)))


def morlet_plan_set_spin_limit(plan: Plan, polls: int):
    _check(lib().morlet_plan_set_spin_limit(plan.handle, int(polls)), "morlet_plan_set_spin_limit")


def morlet_plan_set_row_thresholds(plan: Plan, lane_chunk_max_L: int, start_state_min_L: int):
    """Rows with L <= lane_chunk_max_L take the lane-chunk scan, rows with L > start_state_min_L
    start from exact states (0 turns either off); compensated-FP32 rotating-form SFT plans only."""
    _check(lib().morlet_plan_set_row_thresholds(plan.handle, int(lane_chunk_max_L), int(start_state_min_L)),
           "morlet_plan_set_row_thresholds")


def morlet_plan_set_schedule(plan: Plan, seg_mult: int = 16, ss_tiles_max: int = 32, order: int = 0,
                             asft_chains: int = 0):
    """The forward's scheduling knobs (see the C header); none changes the transform."""
    _check(lib().morlet_plan_set_schedule(plan.handle, int(seg_mult), int(ss_tiles_max), int(order),
                                          int(asft_chains)), "morlet_plan_set_schedule")


def morlet_plan_schedule(plan: Plan) -> dict:
    o = (ctypes.c_int64 * 8)()
    _check(lib().morlet_plan_schedule(plan.handle, o), "morlet_plan_schedule")
    keys = ["lane_chunk_max_L", "start_state_min_L", "seg_mult", "ss_tiles_max", "order", "asft_chains",
            "autotuned", "autotune_outputs"]
    return dict(zip(keys, list(o)))


def morlet_measure_fp64_rate(stream=None) -> float:
    """Measured FP64 FMA rate of the current device in flops/s (a timed kernel of FMA chains)."""
    v = ctypes.c_double()
    _check(lib().morlet_measure_fp64_rate(ctypes.byref(v), _stream(stream)), "morlet_measure_fp64_rate")
    return v.value


def morlet_debug_skip_tickets(plan: Plan, skip: int):
    _check(lib().morlet_debug_skip_tickets(plan.handle, int(skip)), "morlet_debug_skip_tickets")


def morlet_forward_noalloc(x, N, sigma, xi, K, W, stream=None):
    """Forward transform of one FP32 signal at one scale using only the library's fixed device
    scratch array (no allocation anywhere); for callers that cannot allocate device memory."""
    _check(lib().morlet_forward_noalloc(_ptr(x), int(N), float(sigma), float(xi), int(K), _ptr(W),
                                        _stream(stream)), "morlet_forward_noalloc")
