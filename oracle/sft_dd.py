"""ctypes wrapper and build step for the double-double C oracle (oracle/sft_dd.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sft_dd.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libsft_dd.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile sft_dd.c with gcc (OpenMP, no FP contraction so TwoSum stays exact)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.oracle_sft_dd.argtypes = [d, i64, i64, i32, i32, d, d, d]
        lib.oracle_sft_dd.restype = ctypes.c_int
        lib.oracle_asft_dd.argtypes = [d, i64, i64, i32, i32, ctypes.c_double, i64, d, d,
                                       ctypes.c_double, ctypes.c_double, d]
        lib.oracle_asft_dd.restype = ctypes.c_int
        lib.oracle_sft_dd_batch.argtypes = [d, d, d, i32, d, d, i32, i32, d, d, d, i32]
        lib.oracle_sft_dd_batch.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def sft_direct_method(x, fit):
    """O-SFT: direct-method Morlet transform by the kernel integral (Sec. II-B, Sec. III-A)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    K = len(fit["m"])
    m = np.ascontiguousarray(fit["m"], np.float64)
    l = np.ascontiguousarray(fit["l"], np.float64)
    W = np.zeros(2 * x.shape[0], np.float64)
    rc = lib.oracle_sft_dd(_ptr(x), x.shape[0], int(fit["L"]), int(fit["p0"]), K, _ptr(m), _ptr(l), _ptr(W))
    if rc != 0:
        raise RuntimeError("oracle_sft_dd failed")
    return W[0::2] + 1j * W[1::2]


def adjoint_sft(g, fit):
    """Adjoint of the direct-method transform (real input, real loss) by the kernel integral.

    With g[n] = dLoss/dRe W[n] + i dLoss/dIm W[n] the gradient is
    dx[t] = sum_k Re(conj(g[t+k]) psi_hat[k]) (the transpose of W = sum_k psi_hat[k] x[n-k]).
    Write g = a + i b. The fitted kernel has an even real part and an odd imaginary part (Sec. III-A:
    cos terms m_p, sin terms l_p), so sum_k psi_hat[k] a[t+k] is the transform of a evaluated with
    the kernel reflected, which conjugates the imaginary part: dx = Re W(a) - Im W(b), where W(.) is
    the O-SFT transform of a real signal. Two O(N K) runs instead of the O(N L) direct transpose
    (morlet.adjoint_direct, which this is pinned against)."""
    g = np.asarray(g, dtype=np.complex128)
    return sft_direct_method(g.real, fit).real - sft_direct_method(g.imag, fit).imag


def sft_gauss(x, gfit):
    """Gaussian smoothing / derivative by the kernel integral: sum_p coef_p c_p (cos) or s_p (sin)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    K = len(gfit["coef"])
    c = np.ascontiguousarray(gfit["coef"], np.float64)
    z = np.zeros(K)
    W = np.zeros(2 * x.shape[0], np.float64)
    if gfit["basis"] == "cos":
        rc = lib.oracle_sft_dd(_ptr(x), x.shape[0], int(gfit["L"]), 0, K, _ptr(c), _ptr(z), _ptr(W))
        out = W[0::2]
    else:
        rc = lib.oracle_sft_dd(_ptr(x), x.shape[0], int(gfit["L"]), 0, K, _ptr(z), _ptr(c), _ptr(W))
        out = W[1::2]
    if rc != 0:
        raise RuntimeError("oracle_sft_dd failed")
    return out.copy()


def asft_direct_method(x, fit, sigma: float, xi: float, n0: int):
    """ASFT direct-method Morlet transform by the attenuated recursion (Sec. II-D, Sec. III-A),
    with the decaying sign reading, output shift n0 and factor E = e^{-alpha^2/(4 gamma)} e^{i omega0 n0}."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    K = len(fit["m"])
    m = np.ascontiguousarray(fit["m"], np.float64)
    l = np.ascontiguousarray(fit["l"], np.float64)
    alpha = float(n0) / (sigma * sigma)
    g = 1.0 / (2.0 * sigma * sigma)
    mag = math.exp(-alpha * alpha / (4.0 * g))
    ph = (xi / sigma) * n0
    W = np.zeros(2 * x.shape[0], np.float64)
    rc = lib.oracle_asft_dd(_ptr(x), x.shape[0], int(fit["L"]), int(fit["p0"]), K, alpha, int(n0),
                            _ptr(m), _ptr(l), mag * math.cos(ph), mag * math.sin(ph), _ptr(W))
    if rc != 0:
        raise RuntimeError("oracle_asft_dd failed")
    return W[0::2] + 1j * W[1::2]


def asft_gauss(x, gf):
    """Gaussian smoothing (or a derivative) by the attenuated recursion (Sec. II-D, eq. GsASFT):
    the damped window sums of the cos part and of the sin part of the fit, shifted by n0 and scaled
    by C = e^{-alpha^2/(4 gamma)} (see morlet.fit_gauss_asft); real output."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    K = len(gf["cos"])
    c = np.ascontiguousarray(gf["cos"], np.float64)
    sn = np.ascontiguousarray(gf["sin"], np.float64)
    sigma, alpha, n0 = gf["sigma"], gf["alpha"], gf["n0"]
    C = math.exp(-alpha * alpha * sigma * sigma / 2.0)
    W = np.zeros(2 * x.shape[0], np.float64)
    rc = lib.oracle_asft_dd(_ptr(x), x.shape[0], int(gf["L"]), 0, K, float(alpha), int(n0), _ptr(c), _ptr(sn),
                            C, 0.0, _ptr(W))
    if rc != 0:
        raise RuntimeError("oracle_asft_dd failed")
    return W[0::2] + W[1::2]


def sft_batch(signals, fits, n_threads: int = 0):
    """All (signal, scale) chains of a ragged batch, OpenMP over chains. Returns (W, threads used).

    W is the scalogram laid out as [signal][scale][n] (complex128)."""
    lib = _load()
    lens = np.array([s.shape[0] for s in signals], np.int64)
    off = np.zeros(len(signals), np.int64)
    off[1:] = np.cumsum(lens)[:-1]
    x = np.ascontiguousarray(np.concatenate(signals).astype(np.float64))
    K = len(fits[0]["m"])
    Ls = np.array([f["L"] for f in fits], np.int64)
    p0 = np.array([f["p0"] for f in fits], np.int32)
    ore = np.ascontiguousarray(np.concatenate([f["m"] for f in fits]), np.float64)
    oim = np.ascontiguousarray(np.concatenate([f["l"] for f in fits]), np.float64)
    S = len(fits)
    W = np.zeros(2 * int(lens.sum()) * S, np.float64)
    used = lib.oracle_sft_dd_batch(_ptr(x), _ptr(off), _ptr(lens), len(signals), _ptr(Ls), _ptr(p0), S, K,
                                   _ptr(ore), _ptr(oim), _ptr(W), int(n_threads))
    if used < 0:
        raise RuntimeError("oracle_sft_dd_batch failed")
    return W[0::2] + 1j * W[1::2], used
