"""Writes morlet_approx_sweep.json: the approximation-error experiment of arXiv:2110.11866, Sec. IV
("Approximation error of the Morlet wavelet", Figs. MSE1 and MSE2), computed by the oracle alone.

sigma = 60, xi = 1 .. 20, the normalised Morlet of Sec. III; for every (method, order) the window L is
the one with the smallest relative RMSE over [-5L, 5L] (the paper's choice). Methods: the direct
method with P_D terms (least-residual P_S), the multiplication method with P_M (2 P_M + 1
non-harmonic terms and the kappa terms), and the Morlet truncated to [-3 sigma, 3 sigma]. The paper
prints no values for these figures, so the table is the oracle's; tests pin its shape to what the
text states. Run: python tests/golden/make_morlet_approx_sweep.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import morlet as M  # noqa: E402

SIGMA = 60.0
XIS = [float(x) for x in range(1, 21)]
CASES = [("direct", 3), ("direct", 5), ("direct", 6), ("direct", 7),
         ("multiply", 1), ("multiply", 2), ("multiply", 3), ("truncated", 0)]


def main():
    rows = []
    for xi in XIS:
        row = {"xi": xi}
        for meth, P in CASES:
            b = M.best_window(meth, SIGMA, xi, P)
            row[f"{meth}_{P}"] = {"rmse": b["rmse"], "L": b["L"], "p_start": b["p0"]}
        rows.append(row)
    out = {
        "source": "arXiv:2110.11866, Sec. IV 'Approximation error of the Morlet wavelet' (Figs. MSE1, MSE2): "
                  "sigma = 60, xi = 1..20, window chosen for the smallest relative RMSE over [-5L, 5L]. "
                  "The figures' values are not printed; every number here is computed by oracle/morlet.py "
                  "(best_window) through this script.",
        "sigma": SIGMA,
        "norm": 1,
        "cases": [f"{m}_{p}" for m, p in CASES],
        "rows": rows,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "morlet_approx_sweep.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
