"""mg_propagate_noalloc: the propagation for callers that cannot allocate
device memory (a host application or framework that owns all device memory
through its own pool, or a loop where an allocation's device synchronisation
is not acceptable).  Its scratch is a fixed array inside the library, shared
by every call, so these tests also check that leftover contents of a previous
call (another grid, another potential) do not leak into the next one.

This file sorts last so that a run stopping at its first failure has already
run every other test.
"""
import numpy as np
import pytest

from tests import inputs

TOL = 1e-12


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    # sum of axis lengths 4224 > 4096: refused before any device work
    from paper_1909_06412_gb300 import _build, capi
    import ctypes, os

    if not os.path.exists(capi.LIB_PATH):
        _build.build()
    fn = capi.lib().mg_propagate_noalloc
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    fn.argtypes = [i32, vp, vp, vp, d, i32, vp, i32, vp, vp, vp, i64, d, ctypes.c_char_p, i32, i32, vp]
    fn.restype = i32
    N = np.array([1024, 1024, 1024, 1024, 128], dtype=np.int64)
    dq = np.full(5, 0.1)
    minv = np.eye(5).ravel()
    pot = np.array([0.1])
    q, p = np.zeros(5), np.zeros(5)
    P = lambda a: a.ctypes.data_as(vp)
    rc = fn(5, P(N), P(dq), P(minv), 1.0, capi.MG_POT_HENON_HEILES, P(pot), 1, vp(256), P(q), P(p),
            1, 0.1, b"strang", 0, 0, None)
    assert rc == capi.MG_ERR_UNSUPPORTED


@pytest.mark.gpu
def test_noalloc_matches_the_context_entry_point_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as mg

    def case_atom_diatom():
        P = inputs.ATOM_DIATOM
        N, dq = (64, 48), (0.32, 0.2)
        minv = (1 / P["mu"][0], 1 / P["mu"][1])
        pot = [P["Dm"], P["a"], P["re"], P["A"], P["beta"]]
        rbar = mg.mg_morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
        fac = [("gauss", P["R0"], P["P0"], P["sigma"]), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])]
        return N, dq, minv, mg.MG_POT_ATOM_DIATOM, pot, fac, [P["R0"], rbar], [P["P0"], 0.0], 2.0

    def case_harmonic():
        P = inputs.HARMONIC3D
        om = np.array(P["omega"])
        pot = list(np.diag(om ** 2).ravel()) + [0.0, 0.0, 0.0]
        fac = [("gauss", P["q0"][l], P["p0"][l], om[l] ** -0.5) for l in range(3)]
        return (16, 12, 24), (0.6, 0.7, 0.45), (1.0, 1.0, 1.0), mg.MG_POT_HARMONIC, pot, fac, P["q0"], P["p0"], 0.05

    # two different grids in a row, then the first again: each call must match
    # the context-based entry point (mg_create ... mg_propagate) on the same input
    for case, split, scheme in [(case_atom_diatom, mg.MG_TVT, "yoshida4"),
                                (case_harmonic, mg.MG_VTV, "suzuki4"),
                                (case_atom_diatom, mg.MG_TVT, "yoshida4")]:
        N, dq, minv, kind, pot, fac, qc, pc, dt = case()
        g = mg.Propagator(N, dq, minv=minv)
        g.set_potential(kind, pot)
        g.set_separable(fac, qc, pc)
        u0 = g.psi.clone()
        _, q0, p0, _ = g.get_state(want_psi=False)
        g.propagate(12, dt, scheme, split)
        _, q_ref, p_ref, _ = g.get_state(want_psi=False)
        u_ref = g.psi.double().cpu().numpy()

        d_psi = u0.clone()
        q, p = q0.copy(), p0.copy()
        mg.mg_propagate_noalloc(N, dq, minv, 1.0, kind, pot, d_psi, q, p, 12, dt, scheme, split,
                                stream=g.stream)
        u = d_psi.cpu().numpy()
        assert rel(u, u_ref) < TOL
        assert np.abs(q - q_ref).max() < TOL * max(1.0, np.abs(q_ref).max())
        assert np.abs(p - p_ref).max() < TOL * max(1.0, np.abs(p_ref).max())
