"""The full-size 8D short-axis plans compared point by point with the FP64
oracle, through separability.

With a diagonal harmonic potential, V = sum_a k_a (x_a - c_a)^2 / 2, a
diagonal mass and a product initial state, every substep of the moving-grid
integrator acts on each axis alone: the kinetic and potential factors are
products of per-axis factors (eq:U_T_tensor, eq:U_V_tensor), and the Ehrenfest
reductions <p_a> and <dV/dq_a> of a product state depend only on its a-th
factor.  The 8D state after n steps is then the product of eight 1D oracle
runs, and its grid centres are theirs.  This holds on the 12^8 FP64 grid
(4.3e8 points, the plan {5,6,7}, {2,3,4}, {0,1}) and on the 16^8 FP32 grid
(4.3e9 points), where a full oracle run is out of reach, so the kernels'
full-size passes are checked element by element at sampled points: the
points of largest modulus and seeded random ones."""
import numpy as np
import pytest

import oracle
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 8
STEPS, DT, SCHEME = 3, 0.05, "suzuki4"


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as m

    m.lib()
    return m


def axis_setup(a):
    """Force constant, potential centre and initial Gaussian of axis a."""
    omega = 1.0 + 0.05 * a
    return omega ** 2, 0.2 - 0.05 * a, ("gauss", 0.5 + 0.1 * a, 0.3 - 0.05 * a, omega ** -0.5)


def oracle_axes(n, dq):
    """The eight 1D oracle runs: scaled states u_a and final centres."""
    us, qs, ps = [], [], []
    for a in range(D):
        k, c, fac = axis_setup(a)
        o = oracle.Grid((n,), (dq,))
        o.set_potential(oracle.POT_HARMONIC, [k, c])
        o.set_separable([fac], [fac[1]], [fac[2]])
        o.propagate(STEPS, DT, SCHEME)
        _, q, p, _ = o.get_state()
        us.append(o.get_u())
        qs.append(q[0])
        ps.append(p[0])
    return us, np.array(qs), np.array(ps)


def sample_points(us, n, count, seed):
    """Flat indices of the product's largest entries (per-axis argmax and its
    neighbours) and of seeded random points, with the product's values."""
    rng = inputs.rng(seed)
    rand = rng.integers(0, n, size=(count, D))
    top = np.array([[int(np.argmax(np.abs(u))) for u in us]])
    near = top + rng.integers(-1, 2, size=(count // 4, D))
    J = np.concatenate([top, np.clip(near, 0, n - 1), rand])
    flat = np.zeros(len(J), dtype=np.int64)
    vals = np.ones(len(J), dtype=np.complex128)
    for a in range(D):
        flat = flat * n + J[:, a]
        vals = vals * us[a][J[:, a]]
    return flat, vals


@pytest.mark.parametrize("n,prec,tol", [(12, 0, 1e-12), (16, 1, 5e-5)])
def test_full_size_8d_matches_product_of_1d_oracle_runs(mg, n, prec, tol):
    dq = float(np.sqrt(2 * np.pi / n))
    K = np.zeros((D, D))
    ctr, facs = [], []
    for a in range(D):
        k, c, fac = axis_setup(a)
        K[a, a] = k
        ctr.append(c)
        facs.append(fac)
    g = mg.Propagator((n,) * D, (dq,) * D, precision=prec)
    g.set_potential(mg.MG_POT_HARMONIC, list(K.ravel()) + ctr)
    g.set_separable(facs, [f[1] for f in facs], [f[2] for f in facs])
    assert g.path == (2 if prec == 1 else 1)
    g.propagate(STEPS, DT, SCHEME)
    _, q, p, _ = g.get_state(want_psi=False)

    us, q1, p1 = oracle_axes(n, dq)
    ct = max(tol, 1e-12)
    assert np.abs(q - q1).max() < ct, (q, q1)
    assert np.abs(p - p1).max() < ct, (p, p1)
    flat, want = sample_points(us, n, 4096, 20190913)
    u = g.psi.view(torch.complex128 if prec == 0 else torch.complex64)
    got = u[torch.from_numpy(flat).to(u.device)].to(torch.complex128).cpu().numpy()
    # the product state has unit L2 norm, so tol bounds each point's error
    # by tol times the norm of the whole state
    err = np.abs(got - want).max()
    assert err < tol, err
    g.close()
    torch.cuda.empty_cache()
