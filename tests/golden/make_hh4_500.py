"""Write the stored oracle results of the 500-step Henon-Heiles runs on 4D
grids.

The Henon-Heiles model of Sec. III.C (lambda = 0.111803, m = hbar = 1) on 12^4
and 16^4 grids with balanced windows (dq = sqrt(2 pi / n)), Gaussians of unit
width at q = 2, fourth-order Suzuki composition, dt = 0.01, 500 steps (the
length of the 8D workload), computed by the FP64 CPU oracle alone.  Read by
tests/test_gpu_8d.py.

python tests/golden/make_hh4_500.py   (writes the .txt files beside it)
"""
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from tests.golden import records  # noqa: E402

STEPS, DT, SCHEME, LAM = 500, 0.01, "suzuki4", 0.111803
SAMPLE_SEED = 500


def main():
    for n in (12, 16):
        D = 4
        dq = math.sqrt(2 * math.pi / n)
        o = oracle.Grid((n,) * D, (dq,) * D)
        o.set_potential(oracle.POT_HENON_HEILES, [LAM])
        o.set_separable([("gauss", 2.0, 0.0, 1.0)] * D, [2.0] * D, [0.0] * D)
        t0 = time.time()
        o.propagate(STEPS, DT, SCHEME)
        el = time.time() - t0
        out = os.path.join(HERE, f"hh_{n}p4_suzuki4_500.txt")
        records.write(out, o, f"Henon-Heiles {n}^4, suzuki4, dt = 0.01, 500 steps", el, SAMPLE_SEED)
        print(f"wrote {out} in {el:.0f} s")


if __name__ == "__main__":
    main()
