"""Several densities per call (vdw_energy_potential_batched): one launch per
stage for the whole batch, the kernel table and the |G| order shared.  Each
density's results must be bitwise those of a single call on it, on a small
grid with a ragged pencil tail and on the 180 x 180 x 72 tube; the batch
workspaces are sized by vdw_plan_batch and a larger batch is refused."""
import numpy as np
import pytest

from paper_0812_0244_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def densities(torch, shape, L, seeds, tube):
    ns = []
    for s in seeds:
        if tube:
            n, _, _ = S.tube_density_torch(s, shape=shape, device="cuda", shift_ang=0.3 * s, rot_deg=4.0 * s)
            ns.append(n.to(torch.float32))
        else:
            d = S.two_atom_density(s, shape=shape)
            ns.append(torch.tensor(d["n"].astype(np.float32), device="cuda"))
    return torch.stack(ns).contiguous()


@pytest.mark.parametrize("shape,tube", [((16, 27, 20), False), ((72, 180, 180), True)], ids=["small", "tube_180"])
def test_batch_equals_single_calls(torch_cuda, shape, tube):
    torch = torch_cuda
    from paper_0812_0244_gb300 import vdwnl
    B = 3
    if tube:
        _, L, _ = S.tube_density_torch(0, shape=(8, 8, 8), device="cpu")
    else:
        L = S.two_atom_density(0, shape=shape)["L"]
    ctx = vdwnl.VdwNL(vdwnl.Params()).plan(shape, L)
    n = densities(torch, shape, L, range(B), tube)
    g = torch.stack([ctx.spectral_gradient(n[b]) for b in range(B)]).contiguous()
    ctx.plan_batch(B)
    Eb, vb = ctx.energy_potential_batched(n, g, v=torch.empty_like(n))
    Eo, _ = ctx.energy_potential_batched(n[:2].contiguous(), g[:2].contiguous())  # energy only, B < Bmax
    torch.cuda.synchronize()
    for b in range(B):
        E1, v1, _ = ctx.compute(n[b].contiguous(), g[b].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(Eb[b], E1), (b, Eb[b], E1)
        assert torch.equal(vb[b], v1), b
        if b < 2:
            assert torch.equal(Eo[b], E1)
    with pytest.raises(vdwnl.VdwError) as e:
        ctx.energy_potential_batched(torch.cat([n, n[:1]]).contiguous(), torch.cat([g, g[:1]]).contiguous())
    assert e.value.code == -2
