"""Write the stored oracle result of the full-length atom-diatom run.

The collinear atom-diatom model of Sec. III.B on the 256 x 256 moving grid,
fourth-order triple jump, dt = 1 a.u., 2000 steps (t = 2000 a.u.), computed
by the FP64 CPU oracle alone (about ten minutes on one core).  The GPU test
(tests/test_gpu_long.py) compares the library's run with this record instead
of repeating the oracle run on every GPU test session.

Stored (tests/golden/records.py): the grid centres q, p and the time t; the
norm and energy; the discrete L2 norm of psi; and psi at 1024 grid points:
the 512 of largest modulus and 512 drawn from a seeded generator.

python tests/golden/make_atom_diatom_t2000.py   (writes the .txt beside it)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from tests import inputs  # noqa: E402
from tests.golden import records  # noqa: E402

OUT = os.path.join(HERE, "atom_diatom_256x256_yoshida4_t2000.txt")
STEPS, DT, SCHEME = 2000, 1.0, "yoshida4"
SAMPLE_SEED = 2000


def setup():
    P = inputs.ATOM_DIATOM
    minv = (1 / P["mu"][0], 1 / P["mu"][1])
    pot = [P["Dm"], P["a"], P["re"], P["A"], P["beta"]]
    o = oracle.Grid(P["N"], P["dq"], minv=minv)
    o.set_potential(oracle.POT_ATOM_DIATOM, pot)
    rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
    fac = [("gauss", P["R0"], P["P0"], P["sigma"]), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])]
    o.set_separable(fac, [P["R0"], rbar], [P["P0"], 0.0])
    return o


def main():
    o = setup()
    t0 = time.time()
    o.propagate(STEPS, DT, SCHEME)
    el = time.time() - t0
    records.write(OUT, o, "atom-diatom 256x256 moving grid, yoshida4, dt = 1 a.u., 2000 steps", el, SAMPLE_SEED)
    print(f"wrote {OUT} in {el:.0f} s")


if __name__ == "__main__":
    main()
