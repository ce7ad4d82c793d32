"""Write the stored oracle result of the Sec. III.A adaptive-vs-fixed comparison.

The Duschinsky-rotated 3D harmonic model (Table I) propagated by the FP64 CPU
oracle on the adaptive 32^3 grid (dq = 0.4375, centred at the origin) and on
the fixed 128^3 grid with twice its position and momentum ranges (dq =
0.21875, centred at the excited-state minimum q0), fourth-order triple jump,
dt = 50/512, 64 steps.  Stored: the distance of the two final states
(tests/grid_distance.py: the sparser state carried onto the denser grid by
trigonometric interpolation), the distance of their mean positions, and the
adaptive grid's final centres.  About seven minutes of oracle time; read by
tests/test_gpu_adaptive_vs_fixed.py.

python tests/golden/make_adaptive_vs_fixed.py   (writes the .txt beside it)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from tests import grid_distance as gd  # noqa: E402
from tests import inputs  # noqa: E402

OUT = os.path.join(HERE, "adaptive_vs_fixed_duschinsky_yoshida4_64.txt")
STEPS, DT, SCHEME = 64, 50.0 / 512, "yoshida4"
ADAPTIVE = ((32,) * 3, (0.4375,) * 3)
FIXED = ((128,) * 3, (0.21875,) * 3)


def make(N, dq, centre):
    P = inputs.DUSCHINSKY3D
    o = oracle.Grid(N, dq, minv=P["omega"])
    o.set_potential(oracle.POT_HARMONIC, list(np.array(P["K"]).ravel()) + list(P["q0"]))
    o.set_separable([("gauss", 0.0, 0.0, 1.0)] * 3, list(centre), [0.0] * 3)
    return o


def state(o, N, dq):
    psi, q, p, _ = o.get_state()
    return psi, {"N": list(N), "dq": list(dq), "q": list(q), "p": list(p)}


def main():
    t0 = time.time()
    oa = make(*ADAPTIVE, (0.0,) * 3)
    of = make(*FIXED, inputs.DUSCHINSKY3D["q0"])
    oa.propagate(STEPS, DT, SCHEME, oracle.SPLIT_TVT, oracle.GRID_ADAPTIVE)
    of.propagate(STEPS, DT, SCHEME, oracle.SPLIT_TVT, oracle.GRID_FIXED)
    pa, sa = state(oa, *ADAPTIVE)
    pf, sf = state(of, *FIXED)
    d = gd.distance(pa, sa, pf, sf)
    dq_mean = float(np.abs(gd.mean_q(pa, sa) - gd.mean_q(pf, sf)).max())
    el = time.time() - t0
    with open(OUT, "w") as f:
        f.write("# FP64 oracle: Sec. III.A adaptive 32^3 vs fixed 128^3, Table I model, "
                f"{SCHEME}, dt = 50/512, {STEPS} steps\n")
        f.write(f"# written by tests/golden/{os.path.basename(sys.argv[0])} ({el:.0f} s of oracle time)\n")
        f.write(f"distance = {d!r}\n")
        f.write(f"mean_q_distance = {dq_mean!r}\n")
        f.write("q = " + " ".join(repr(float(v)) for v in sa["q"]) + "\n")
        f.write("p = " + " ".join(repr(float(v)) for v in sa["p"]) + "\n")
    print(f"wrote {OUT} in {el:.0f} s: distance {d:.6e}")


if __name__ == "__main__":
    main()
