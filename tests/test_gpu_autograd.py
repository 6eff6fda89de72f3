"""The torch.autograd.Function on the CUDA library (hand-written backward).

* 48^3 two-atom cell: E(n) with grad n = D n built by a differentiable torch
  spectral derivative (Nyquist removed, the library's convention); autograd's
  dE/dn against the FP64 oracle's v dOmega, and against central finite
  differences of the GPU energy at 20 seeded points.
* 256 x 256 x 96 nanotube cell (the paper's 300 Ry mesh): backward recomputes
  theta; autograd's dE/dn through torch's D equals dOmega times the library's
  own full potential (spectral divergence inside the library).
"""
import numpy as np
import pytest

import oracle as O
from paper_0812_0244_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def torch_spectral_gradient(torch, n, L):
    """grad n = IFFT(i G FFT(n)) with the Nyquist component of each even axis removed."""
    N3, N2, N1 = n.shape
    dev = n.device

    def k(N, Ld):
        m = torch.fft.fftfreq(N, d=1.0 / N, device=dev, dtype=torch.float64)
        if N % 2 == 0:
            m[N // 2] = 0.0
        return 2 * np.pi * m / Ld

    nh = torch.fft.fftn(n.to(torch.float64))
    gx = k(N1, L[0])[None, None, :]
    gy = k(N2, L[1])[None, :, None]
    gz = k(N3, L[2])[:, None, None]
    out = [torch.fft.ifftn(1j * gc * nh).real for gc in (gx, gy, gz)]
    return torch.stack(out).to(torch.float32)


def test_autograd_gradient_matches_oracle_and_fd(torch_cuda, table):
    torch = torch_cuda
    from paper_0812_0244_gb300 import vdwnl
    from paper_0812_0244_gb300.autograd import vdw_energy
    d = S.two_atom_density(7, shape=(48, 48, 48))
    L = d["L"]
    ctx = vdwnl.VdwNL(vdwnl.Params()).plan((48, 48, 48), L)
    n = torch.tensor(d["n"].astype(np.float32), device="cuda", requires_grad=True)
    E = vdw_energy(n, torch_spectral_gradient(torch, n, L), ctx)
    E.backward()
    gE = n.grad.double().cpu().numpy()
    n64 = d["n"].astype(np.float32).astype(np.float64)
    ref = O.energy_potential(n64, O.spectral_gradient(n64, L), L, table)
    vref = ref["v"] * ctx.dOmega
    assert abs(float(E.detach()) - ref["E"]) < 1e-6
    assert np.max(np.abs(gE - vref)) <= 1e-5 * np.abs(vref).max()
    # directional derivatives along smooth seeded perturbations: E moves by
    # ~1e-3 relative, so the check is tight
    E_of = lambda m: float(vdw_energy(m, torch_spectral_gradient(torch, m, L), ctx))
    rng = np.random.default_rng(11)
    with torch.no_grad():
        base = n.detach().clone()
        z, y, x = np.meshgrid(*(np.arange(48) / 48.0 for _ in range(3)), indexing="ij")
        for k in range(4):
            ph = rng.uniform(0, 2 * np.pi, 3)
            dirn = n64 * (1.0 + 0.5 * np.sin(2 * np.pi * x + ph[0]) * np.cos(2 * np.pi * y + ph[1])
                          * np.sin(2 * np.pi * z + ph[2]))
            d_t = torch.tensor(dirn.astype(np.float32), device="cuda")
            h = 1e-3
            fd = (E_of(base + h * d_t) - E_of(base - h * d_t)) / (2 * h)
            an = float(np.sum(gE * dirn.astype(np.float32)))
            assert abs(fd - an) <= 1e-3 * abs(an), (k, fd, an)


def stencil_gradient(torch, n, L):
    """grad n by second-order central differences on the periodic grid (the
    finite-difference gradient the paper uses), differentiable in torch."""
    N3, N2, N1 = n.shape
    h = (L[0] / N1, L[1] / N2, L[2] / N3)
    gx = (torch.roll(n, -1, 2) - torch.roll(n, 1, 2)) / (2 * h[0])
    gy = (torch.roll(n, -1, 1) - torch.roll(n, 1, 1)) / (2 * h[1])
    gz = (torch.roll(n, -1, 0) - torch.roll(n, 1, 0)) / (2 * h[2])
    return torch.stack([gx, gy, gz]).contiguous()


def test_autograd_finite_differences_20_points(torch_cuda):
    """FD at 20 seeded grid points of a 48^3 two-atom cell, with grad n from a
    local stencil: a change of one n_i then moves grad n only at its six
    neighbours.  (With the spectral derivative it moves grad n everywhere,
    including floor-density points where s ~ |grad n|/n^(4/3) makes E far
    from linear at any representable step.)  FP32 rounding of E bounds the
    comparison at a few per cent."""
    torch = torch_cuda
    from paper_0812_0244_gb300 import vdwnl
    from paper_0812_0244_gb300.autograd import vdw_energy
    d = S.two_atom_density(7, shape=(48, 48, 48))
    L = d["L"]
    ctx = vdwnl.VdwNL(vdwnl.Params()).plan((48, 48, 48), L)
    n = torch.tensor(d["n"].astype(np.float32), device="cuda", requires_grad=True)
    E = vdw_energy(n, stencil_gradient(torch, n, L), ctx)
    E.backward()
    gE = n.grad.double().cpu().numpy()
    n64 = d["n"].astype(np.float64)
    E_of = lambda m: float(vdw_energy(m, stencil_gradient(torch, m, L), ctx))
    rng = np.random.default_rng(12)
    cand = np.nonzero(n64.ravel() > 0.05 * n64.max())[0]
    with torch.no_grad():
        base = n.detach().clone()
        for i in rng.choice(cand, 20, replace=False):
            pt = np.unravel_index(i, n64.shape)
            h = 1e-2 * float(base[pt])
            m1, m2 = base.clone(), base.clone()
            m1[pt] += h
            m2[pt] -= h
            fd = (E_of(m1) - E_of(m2)) / (2 * h)
            assert abs(fd - gE[pt]) <= 3e-2 * abs(gE[pt]) + 2e-3 * np.abs(gE).max(), (pt, fd, gE[pt])


@pytest.mark.slow
def test_autograd_full_tube_256(torch_cuda):
    torch = torch_cuda
    from paper_0812_0244_gb300 import vdwnl
    from paper_0812_0244_gb300.autograd import vdw_energy
    d = S.tube_density(3, shape=(96, 256, 256))
    L = d["L"]
    ctx = vdwnl.VdwNL(vdwnl.Params()).plan((96, 256, 256), L)
    n = torch.tensor(d["n"].astype(np.float32), device="cuda", requires_grad=True)
    g = torch_spectral_gradient(torch, n, L)
    E = vdw_energy(n, g, ctx)
    E.backward()
    with torch.no_grad():
        Ef, v, _ = ctx.compute(n.detach(), g.detach().contiguous())
    torch.cuda.synchronize()
    assert abs(float(E) - float(Ef[0])) <= 1e-9 * abs(float(Ef[0]))
    a = n.grad.double()
    b = v.double() * ctx.dOmega
    assert float((a - b).abs().max()) <= 1e-5 * float(b.abs().max())
