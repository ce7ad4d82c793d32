"""The device arithmetic the kernels rely on, checked directly.

- The table-driven e^{i theta} of the kernels (Tang's method: a three-word
  Cody-Waite reduction by pi/128, a 256-entry table, short Taylor series)
  against the host's sin and cos over the argument range the phase factors
  reach (|theta| up to 1e5 rad at the grid edges of the atom-diatom model),
  with a stated bound: at most 2 ulp of 1.0 (4.4e-16) absolute.
- The FMA rate probe that the benchmark's FP64 roofline is stated against.
"""
import numpy as np
import pytest

from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as m

    m.lib()
    return m


def test_table_sincos_against_host(mg):
    g = inputs.rng(77)
    th = np.concatenate([
        g.uniform(-1e5, 1e5, 400000), g.uniform(-10.0, 10.0, 400000), g.uniform(-1e-3, 1e-3, 50000),
        np.arange(-512, 513) * (np.pi / 128),  # table nodes and their neighbours
        np.nextafter(np.arange(-512, 513) * (np.pi / 128), np.inf),
        np.arange(-600, 601) * (np.pi / 256),  # midpoints between nodes (largest |r|)
        [0.0, -0.0, 1e-300, 3.0e7, -4.0e8],
    ])
    s, c = mg.mg_probe_expi(torch.from_numpy(th).cuda())
    s, c = s.cpu().numpy(), c.cpu().numpy()
    err = max(np.abs(s - np.sin(th)).max(), np.abs(c - np.cos(th)).max())
    assert err <= 2.0 ** -51, err
    assert np.abs(s * s + c * c - 1).max() < 1e-15


def test_fma_rate_probe(mg):
    r64 = mg.mg_probe_fma_rate(mg.MG_FP64)
    r32 = mg.mg_probe_fma_rate(mg.MG_FP32_MIXED)
    assert r64 > 0 and r32 > r64


@pytest.mark.parametrize("split", [0, 1, 2])
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("nlines", [1, 256, 1000, 40000])
def test_tensor_core_dft16_against_fp64(mg, split, inverse, nlines):
    # the dense 16-point DFT with diagonal multipliers as split-product GEMMs
    # on the tensor cores, element by element against the FP64 product
    g = inputs.rng(1000 + nlines)
    x = (g.standard_normal((nlines, 16)) + 1j * g.standard_normal((nlines, 16))).astype(np.complex64)
    pre = np.exp(1j * g.uniform(-np.pi, np.pi, 16)) / 16
    post = np.exp(1j * g.uniform(-np.pi, np.pi, 16))
    y = mg.mg_probe_tc_dft16(torch.from_numpy(x).cuda(), pre, post, split, inverse).cpu().numpy()
    j = np.arange(16)
    F = np.exp((2j if inverse else -2j) * np.pi * np.outer(j, j) / 16)
    # the multipliers as the device holds them (FP32)
    M = post.astype(np.complex64).astype(np.complex128)[:, None] * F * pre.astype(np.complex64).astype(np.complex128)[None, :]
    ref = x.astype(np.complex128) @ M.T
    err = np.abs(y - ref).max() / np.abs(ref).max()
    # FP32-level: the split products keep 21-24 significant bits per operand
    assert err < 2e-6, err


@pytest.mark.parametrize("split", [0, 1, 2])
@pytest.mark.parametrize("sign", [-1, 1])
def test_tensor_core_dft16_is_the_oracles_transform(mg, split, sign):
    # eq:fourier_pos_to_mom_b on a 16-point axis: f_KJ = N^-1/2 e^{-2 pi i kj/N}
    # e^{-i t_KJ/hbar}, with t_KJ of eq:t_definition separating into a J part,
    # a K part and a constant; the inverse (sign +1) is its adjoint.  The lines
    # through the tensor-core (or register) 16-point DFT with those diagonal
    # factors, element by element against the oracle's transform of each line.
    import oracle

    n, dq, hbar = 16, 0.37, 1.0
    q, p = 0.83, -1.9
    dp = 2 * np.pi * hbar / (n * dq)
    j = np.arange(n)
    c0 = (p - dp * n / 2) * (q - dq * n / 2)
    jpart = np.exp(-1j * (p * dq - np.pi * hbar) * j / hbar)
    kpart = np.exp(-1j * ((q * dp - np.pi * hbar) * j + c0) / hbar)
    if sign == -1:
        pre, post = jpart / np.sqrt(n), kpart
    else:
        pre, post = np.conj(kpart) / np.sqrt(n), np.conj(jpart)
    g = inputs.rng(5150 + split)
    nl = 300
    x = (g.standard_normal((nl, n)) + 1j * g.standard_normal((nl, n))).astype(np.complex64)
    y = mg.mg_probe_tc_dft16(torch.from_numpy(x).cuda(), pre, post, split, sign == 1).cpu().numpy()
    o = oracle.Grid((n,), (dq,), hbar=hbar)
    ref = np.stack([o.apply_f([q], [p], x[i].astype(np.complex128), sign) for i in range(nl)])
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err
