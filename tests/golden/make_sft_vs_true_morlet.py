"""Writes sft_vs_true_morlet.json: the approximation error of the SFT direct method (Sec. III-A) against
the true Morlet wavelet, per number of terms K, at the workloads' window L = ceil(4 sigma) and
xi = 6, unnormalised Morlet (norm = 0), computed by the oracle alone.

Per (K, sigma):
  - kernel_rmse: relative RMSE of the fitted kernel psi_hat (zero outside [-L, L]) against the true
    Morlet over [-5L, 5L] (the paper's error measure, Sec. IV);
  - kernel_max: max |psi_hat - psi| / max |psi| over [-L, L];
  - transform_max (sigma = 64 only): max |W_sft - W_true| / max |W_true| on the N = 4096 N(0,1) signal of
    the FP64 single-signal workload, W_sft the O-SFT transform and W_true the direct convolution with
    the true Morlet truncated at +-8 sigma.
The GPU paths compute psi_hat's transform exactly (to rounding); this table is the method's own error,
reported beside the parity gates and never gated. Run: python tests/golden/make_sft_vs_true_morlet.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as WL  # noqa: E402
from oracle import morlet as M  # noqa: E402
from oracle import sft_dd as D  # noqa: E402

XI = 6.0
KS = [2, 3, 4, 5, 6, 8]
SIGMAS = [8.0, 64.0, 512.0, 4096.0]


def row(K, sigma, x=None):
    fit = M.fit_direct(sigma, XI, K)
    L = fit["L"]
    hat = M.kernel_direct(fit)
    k = np.arange(-L, L + 1)
    psi = M.morlet(k, sigma, XI, 0)
    r = {"K": K, "sigma": sigma, "L": L, "p_start": fit["p0"],
         "kernel_rmse": M.morlet_relative_rmse(hat, L, sigma, XI, norm=0),
         "kernel_max": float(np.abs(hat - psi).max() / np.abs(psi).max())}
    if x is not None:
        ws = D.sft_direct_method(x, fit)
        wt = M.morlet_true_direct(x, sigma, XI)
        r["transform_max"] = float(np.abs(ws - wt).max() / np.abs(wt).max())
    return r


def main():
    x = WL.c1_fp64_single().signals[0]
    rows = [row(K, s, x if s == 64.0 else None) for K in KS for s in SIGMAS]
    out = {"source": "arXiv:2110.11866, Sec. III-A (direct method) and Sec. IV (relative RMSE over [-5L, 5L]); "
                     "every number is computed by oracle/ through this script",
           "xi": XI, "window": "L = ceil(4 sigma)", "norm": 0, "rows": rows}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sft_vs_true_morlet.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
