"""Helpers for the GPU tests: run the CUDA library through its C ABI on torch device memory, and
run the CPU oracle on the same seeded inputs."""
import numpy as np

import paper_2110_11866_gb300 as m
from oracle import morlet as om
from oracle import sft_dd


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def gpu_forward(signals, sigmas, K=4, precision=m.MORLET_FP32_COMP, form=m.MORLET_FORM_AUTO,
                transform=m.MORLET_SFT, xi=6.0, n0=0, flags=0, norm=0, reps=1):
    """Scalogram of a ragged batch; returns (plan, list over signals of arrays [S, N_i])."""
    import torch
    f64 = precision == m.MORLET_FP64
    rdt = torch.float64 if f64 else torch.float32
    cdt = torch.complex128 if f64 else torch.complex64
    lens = [len(s) for s in signals]
    x = torch.from_numpy(np.concatenate(signals).astype(np.float64 if f64 else np.float32)).cuda()
    plan = m.morlet_plan(lens, sigmas, xi=xi, K=K, precision=precision, form=form, transform=transform,
                         n0=n0, flags=flags, norm=norm)
    W = torch.empty(sum(lens) * len(sigmas), dtype=cdt, device="cuda")
    for _ in range(reps):
        m.morlet_forward(plan, x, W)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    Wh = W.cpu().numpy()
    out, off = [], 0
    S = len(sigmas)
    for n in lens:
        out.append(Wh[S * off:S * (off + n)].reshape(S, n))
        off += n
    return plan, out


def oracle_fit(sigma, K, xi=6.0, norm=0):
    return om.fit_direct(sigma, xi, K, norm=norm)


def oracle_forward(x, sigma, K, transform=m.MORLET_SFT, xi=6.0, n0=None, norm=0):
    fit = oracle_fit(sigma, K, xi, norm)
    x = np.asarray(x, np.float64)
    if transform == m.MORLET_SFT:
        return sft_dd.sft_direct_method(x, fit)
    n0 = om.default_n0(sigma) if not n0 else n0
    return sft_dd.asft_direct_method(x, fit, sigma, xi, n0)
