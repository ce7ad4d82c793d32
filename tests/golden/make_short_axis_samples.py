"""Write stored oracle results for the short-axis kernel's large-grid plans.

Two Henon-Heiles runs (Sec. III.C model, lambda = 0.111803, balanced windows
dq = sqrt(2 pi / n)), one Strang step of dt = 0.02 each, from Gaussians near
q = 2, computed by the FP64 CPU oracle alone:
  - 12^7 (3.6e7 points): the GPU's FP64 plan transforms a strided group of
    three 12-point axes that has a leading index, as the 12^8 plan does;
  - 16^6 (1.7e7 points): the GPU's FP32 plan transforms a strided group of two
    16-point axes with a leading index and a single 16-point axis of stride
    16^5, as the 16^8 plan does.
About 15 minutes of oracle time.  The GPU test is tests/test_gpu_short_large.py.

python tests/golden/make_short_axis_samples.py [12p7|16p6]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from tests.golden import records  # noqa: E402

LAM = 0.111803
CASES = {"12p7": (12, 7, "hh_12p7_strang1.txt", 127), "16p6": (16, 6, "hh_16p6_strang1.txt", 166)}


def initial(n, D):
    dq = np.sqrt(2 * np.pi / n)
    fac = [("gauss", 2.0 + 0.1 * l, 0.2 - 0.1 * l, 1.0) for l in range(D)]
    return (n,) * D, (dq,) * D, fac, [2.0 + 0.1 * l for l in range(D)], [0.2 - 0.1 * l for l in range(D)]


def run(key):
    n, D, fname, seed = CASES[key]
    N, dq, fac, qc, pc = initial(n, D)
    o = oracle.Grid(N, dq)
    o.set_potential(oracle.POT_HENON_HEILES, [LAM])
    o.set_separable(fac, qc, pc)
    t0 = time.time()
    o.propagate(1, 0.02, "strang")
    el = time.time() - t0
    records.write(os.path.join(HERE, fname), o, f"Henon-Heiles {n}^{D}, one Strang step, dt = 0.02", el, seed)
    print(f"{fname}: {el:.0f} s")


if __name__ == "__main__":
    for key in (sys.argv[1:] or list(CASES)):
        run(key)
