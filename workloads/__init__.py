"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and bench.py.

This module only draws numbers. It holds none of the transform's arithmetic (no fit, no
window, no phase), so the CPU oracle and the CUDA path can both take their inputs from
here without sharing any of the method's code.

The paper (Sec. V-B) times one signal of N = 102400 samples with sigma up to 8192 and does
not say what the signal was; it uses no public dataset. The five workloads below are
synthetic stand-ins with the shapes of those experiments: single long signals, sigma
sweeps up to 8192 and beyond, and a ragged multi-signal scalogram batch. Every recipe is
written out here so that it can be checked by reading.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """One batch: ragged real signals, a list of scales and the transform settings."""
    name: str
    signals: list            # list of 1-D numpy arrays (float32 or float64)
    sigmas: list             # list of float
    K: int                   # number of Fourier terms
    xi: float = 6.0          # centre parameter; omega0 = xi / sigma
    dtype: str = "f32"
    extra: dict = field(default_factory=dict)

    @property
    def lengths(self):
        return [int(s.shape[0]) for s in self.signals]

    @property
    def n_outputs(self):
        return sum(self.lengths) * len(self.sigmas)

    def concat(self):
        return np.concatenate(self.signals) if self.signals else np.zeros(0, np.float32)


def c1_fp64_single(seed: int = 0) -> Workload:
    """N = 4096 i.i.d. N(0,1) samples (float64), sigma = 64, K = 4."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(4096).astype(np.float64)
    return Workload("c1_fp64_N4096_sigma64_K4", [x], [64.0], 4, dtype="f64")


def c2_chirps(seed: int = 1, N: int = 102400):
    """Sum of 3 linear chirps plus N(0, 0.1^2) noise (float32).

    Draw order from default_rng(seed): 6 frequencies U[0.001, 0.2] rad/sample taken as
    (start, end) pairs for chirps 0..2, then 3 initial phases U[0, 2 pi), then N noise samples
    of standard deviation 0.1. Chirp c has phase phi_c + f_s n + (f_e - f_s) n^2 / (2 (N-1)),
    so its instantaneous frequency goes linearly from f_s to f_e, with unit amplitude.
    """
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.001, 0.2, size=6)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=3)
    n = np.arange(N, dtype=np.float64)
    x = np.zeros(N, np.float64)
    for c in range(3):
        fs, fe = f[2 * c], f[2 * c + 1]
        x += np.cos(ph[c] + fs * n + (fe - fs) * n * n / (2.0 * (N - 1)))
    x += rng.normal(0.0, 0.1, size=N)
    return x.astype(np.float32)


C2_SIGMAS = [8.0, 32.0, 128.0, 512.0, 2048.0, 8192.0]
C2_KS = [3, 4, 6]


def c2_workload(sigma: float, K: int, seed: int = 1) -> Workload:
    return Workload(f"c2_chirps_N102400_sigma{int(sigma)}_K{K}", [c2_chirps(seed)], [sigma], K)


def c3_lengths(seed: int = 2, n_signals: int = 256, lo: int = 1024, hi: int = 1048576):
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=n_signals)
    return rng, np.rint(np.exp(u)).astype(np.int64)


C3_SIGMAS = [2.0 ** (3 + j / 3.0) for j in range(32)]


def c3_scalogram(seed: int = 2, n_signals: int = 256, max_len: int | None = None) -> Workload:
    """Ragged batch: 256 float32 signals, lengths log-uniform in [1024, 1048576].

    Draw order from default_rng(seed): the 256 lengths round(exp(U(ln 1024, ln 1048576))),
    then 256 tone frequencies log-uniform in [6/sigma_max, 6/sigma_min], then 256 tone phases
    U[0, 2 pi), then for each signal in turn its N(0,1) noise. Each signal is noise plus
    cos(f n + phi) of unit amplitude. 32 scales sigma_j = 2^(3 + j/3), K = 4.
    `max_len` clips the lengths (for a smaller test batch with the same recipe).
    """
    rng, lengths = c3_lengths(seed, n_signals)
    if max_len is not None:
        lengths = np.minimum(lengths, max_len)
    smin, smax = C3_SIGMAS[0], C3_SIGMAS[-1]
    fr = np.exp(rng.uniform(math.log(6.0 / smax), math.log(6.0 / smin), size=n_signals))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=n_signals)
    sigs = []
    for i in range(n_signals):
        Ni = int(lengths[i])
        n = np.arange(Ni, dtype=np.float64)
        x = rng.standard_normal(Ni) + np.cos(fr[i] * n + ph[i])
        sigs.append(x.astype(np.float32))
    return Workload("c3_scalogram_256sig_32scales_K4", sigs, list(C3_SIGMAS), 4)


C4_SIGMAS = [2.0 ** (4 + j / 2.0) for j in range(16)]


def c4_batch(seed: int = 3, n_signals: int = 64, N: int = 65536) -> Workload:
    """64 float32 signals of N(0,1), N = 65536, 16 scales sigma_j = 2^(4 + j/2), K = 4."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n_signals, N)).astype(np.float32)
    return Workload("c4_grad_64x65536_16scales_K4", [x[i] for i in range(n_signals)],
                    list(C4_SIGMAS), 4)


def c4_loss_weights(seed: int = 4, n_signals: int = 64, n_scales: int = 16, N: int = 65536):
    """Fixed N(0,1) loss weights, one per (signal, scale, n), float32."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_signals, n_scales, N)).astype(np.float32)


C5_SIGMAS = [8192.0, 65536.0, 1048576.0]


def c5_pink(seed: int = 5, N: int = 1 << 24):
    """Pink (1/f power) noise plus a 0.05 rad/sample tone, float32.

    White N(0,1) from default_rng(seed) -> rfft -> bin k >= 1 scaled by 1/sqrt(k), DC bin set
    to 0 -> irfft -> scaled to unit standard deviation; then cos(0.05 n) of amplitude 1 added.
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(N)
    F = np.fft.rfft(w)
    k = np.arange(F.shape[0], dtype=np.float64)
    scale = np.zeros_like(k)
    scale[1:] = 1.0 / np.sqrt(k[1:])
    p = np.fft.irfft(F * scale, n=N)
    p /= p.std()
    p += np.cos(0.05 * np.arange(N, dtype=np.float64))
    return p.astype(np.float32)


def c5_workload(sigma: float, seed: int = 5, N: int = 1 << 24, dtype: str = "f32") -> Workload:
    x = c5_pink(seed, N)
    if dtype == "f64":
        x = x.astype(np.float64)
    return Workload(f"c5_pink_N{N}_sigma{int(sigma)}_K6", [x], [sigma], 6, dtype=dtype)


def white(seed: int, N: int, dtype=np.float32):
    """Plain N(0,1) samples for edge-case tests."""
    return np.random.default_rng(seed).standard_normal(N).astype(dtype)
