"""The atom-diatom workload at its full length: the 256 x 256 moving grid
(Sec. III.B model) propagated to t = 2000 a.u. with the fourth-order triple
jump at dt = 1 a.u. (2000 steps, 6001 kinetic and 6000 potential substeps),
against the FP64 oracle's result of the same run, stored by
tests/golden/make_atom_diatom_t2000.py (about ten minutes of oracle time, too
long to repeat in every GPU session).

Compared: the grid centres (1e-12 relative), the time, the norm and energy,
and psi at the 1024 stored grid points (the 512 of largest modulus and 512
seeded ones), each within 1e-12 of the discrete L2 norm of psi: a relative
L2 distance <= 1e-12 over the whole grid implies that bound at every point.
"""
import numpy as np
import pytest

from tests import inputs
from tests.golden import records

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as m

    m.lib()
    return m


def test_atom_diatom_256x256_yoshida4_to_t2000(mg):
    rec = records.read("atom_diatom_256x256_yoshida4_t2000.txt")
    P = inputs.ATOM_DIATOM
    g = mg.Propagator(P["N"], P["dq"], minv=(1 / P["mu"][0], 1 / P["mu"][1]))
    g.set_potential(mg.MG_POT_ATOM_DIATOM, [P["Dm"], P["a"], P["re"], P["A"], P["beta"]])
    rbar = mg.mg_morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
    g.set_separable([("gauss", P["R0"], P["P0"], P["sigma"]), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])],
                    [P["R0"], rbar], [P["P0"], 0.0])
    g.propagate(2000, 1.0, "yoshida4")
    psi, q, p, t = g.get_state()
    n, E, _, _ = g.observables()
    err = {"q": np.abs(q - rec["q"]).max() / max(1.0, np.abs(rec["q"]).max()),
           "p": np.abs(p - rec["p"]).max() / max(1.0, np.abs(rec["p"]).max()),
           "norm": abs(n - rec["norm"]), "energy": abs(E - rec["energy"]) / abs(rec["energy"]),
           "psi": np.abs(psi.ravel()[rec["idx"]] - rec["psi"]).max() / rec["psi_l2"]}
    assert abs(t - rec["t"]) < 1e-9
    assert all(v < TOL for v in err.values()), err
