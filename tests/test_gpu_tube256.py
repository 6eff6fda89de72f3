"""Parity on the 256 x 256 x 96 nanotube grid (h ~ 0.18 bohr, the paper's
300 Ry mesh of the double-wall tube section), through the C ABI.

This grid runs compile-time line transforms of lengths 256 (x and y) and 96
(z) that no smaller case reaches, so it is checked against independent FP64
results:

* the library's spectral gradient of a seeded field against numpy's FFT
  (both directions of every line transform at lengths 256 and 96, including
  the rotated radix-16 first pass of length 256);
* E_c^nl and v_nl of the tube against the FP64 oracle, within the path's
  tolerances |Delta E| <= 1e-6 Ha and max|Delta v| <= 1e-5 max|v|;
* the autograd Function (theta recomputed in the backward) against the same
  oracle potential.

grad n is D n (the spectral derivative with the Nyquist components removed),
evaluated in FP64 and rounded to FP32; both sides get the same FP32 inputs.
"""
import numpy as np
import pytest

import oracle as O
from paper_0812_0244_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

SHAPE = (96, 256, 256)
E_TOL = 1e-6
V_REL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def tube():
    d = S.tube_density(3, shape=SHAPE)
    n32 = d["n"].astype(np.float32)
    g32 = O.spectral_gradient(n32.astype(np.float64), d["L"]).astype(np.float32)
    return n32, g32, d["L"]


def test_spectral_gradient_256_96_against_numpy(torch_cuda, tube):
    """Line transforms of lengths 256 and 96 (forward and inverse) through
    vdw_spectral_gradient, against numpy's FFT in FP64."""
    torch = torch_cuda
    from paper_0812_0244_gb300 import vdwnl
    _, _, L = tube
    rng = np.random.default_rng(256)
    # white noise plus a smooth part: every frequency of every axis is present
    f = rng.standard_normal(SHAPE)
    z, y, x = np.meshgrid(*(np.arange(m) / m for m in SHAPE), indexing="ij")
    f += 3.0 * np.sin(2 * np.pi * (x + 2 * y)) * np.cos(2 * np.pi * 3 * z)
    f32 = f.astype(np.float32)
    ref = O.spectral_gradient(f32.astype(np.float64), L)
    ctx = vdwnl.VdwNL(vdwnl.Params()).plan(SHAPE, L)
    got = ctx.spectral_gradient(torch.tensor(f32, device="cuda")).cpu().numpy().astype(np.float64)
    for c in range(3):
        err = got[c] - ref[c]
        scale = np.abs(ref[c]).max()
        assert np.abs(err).max() <= 1e-5 * scale, (c, np.abs(err).max() / scale)
        assert np.sqrt(np.mean(err ** 2)) <= 2e-6 * np.sqrt(np.mean(ref[c] ** 2)), c


@pytest.mark.slow
def test_tube_256_energy_potential_and_autograd_match_oracle(torch_cuda, tube, table):
    torch = torch_cuda
    from paper_0812_0244_gb300 import vdwnl
    from paper_0812_0244_gb300.autograd import vdw_energy
    n32, g32, L = tube
    ref = O.energy_potential(n32.astype(np.float64), g32.astype(np.float64), L, table)
    vmax = np.abs(ref["v"]).max()
    ctx = vdwnl.VdwNL(vdwnl.Params()).plan(SHAPE, L)
    nt = torch.tensor(n32, device="cuda")
    gt = torch.tensor(g32, device="cuda")
    E, v, _ = ctx.compute(nt, gt)
    torch.cuda.synchronize()
    E = E.cpu().numpy()
    assert abs(E[0] - ref["E"]) <= E_TOL, (E, ref["E"])
    assert abs(E[1] - ref["E_soft"]) <= E_TOL
    assert abs(E[2] - ref["dE"]) <= E_TOL
    v = v.cpu().numpy().astype(np.float64)
    assert np.abs(v - ref["v"]).max() <= V_REL * vmax, np.abs(v - ref["v"]).max() / vmax
    del v

    # autograd: forward E, backward with theta recomputed; grad n enters as a
    # leaf with the oracle's gradient, so dE/dn + D^T dE/dgrad is v dOmega
    n = nt.clone().requires_grad_(True)
    g = gt.clone().requires_grad_(True)
    Ea = vdw_energy(n, g, ctx)
    Ea.backward()
    assert abs(float(Ea.detach()) - ref["E"]) <= E_TOL
    vloc = n.grad.double().cpu().numpy() / ctx.dOmega
    w = g.grad.double().cpu().numpy() / ctx.dOmega
    assert np.abs(vloc - ref["v_loc"]).max() <= V_REL * np.abs(ref["v_loc"]).max()
    assert np.abs(w - ref["w"]).max() <= V_REL * np.abs(ref["w"]).max()
    v_chain = vloc - O.spectral_divergence(w, L)
    assert np.abs(v_chain - ref["v"]).max() <= V_REL * vmax
