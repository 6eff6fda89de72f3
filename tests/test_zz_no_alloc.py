"""vdw_delta_energy_noalloc: the Delta E entry point that allocates no device
memory (for callers that must not allocate when they evaluate the energy)
gives the same Delta E as vdw_energy_potential, call after call.

Kept in a file of its own that pytest collects last; it builds its own
context, so it also passes when run alone in a fresh process."""
import numpy as np
import pytest

from paper_0812_0244_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

E_TOL = 1e-6  # Hartree per cell, as in the parity tests


def test_noalloc_delta_energy_matches_energy_potential():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0812_0244_gb300 import vdwnl
    ctx = vdwnl.VdwNL(vdwnl.Params())
    for seed, shape in ((0, (24, 24, 24)), (5, (12, 20, 16))):
        d = S.two_atom_density(seed, shape=shape)
        ctx.plan(shape, d["L"])
        n = torch.tensor(d["n"].astype(np.float32), device="cuda")
        g = torch.tensor(d["grad"].astype(np.float32), device="cuda")
        E, _, _ = ctx.compute(n, g, want_v=False)
        ref = float(E[2].item())
        dE = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        got = []
        for _ in range(2):  # two calls in a row share the scratch
            ctx.delta_energy_noalloc(n, g, dE)
            torch.cuda.synchronize()
            got.append(float(dE.item()))
        for x in got:
            assert abs(x - ref) <= E_TOL, (x, ref)
        assert got[0] == got[1]


def test_noalloc_rejects_more_points_than_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0812_0244_gb300 import vdwnl
    ctx = vdwnl.VdwNL(vdwnl.Params())
    n = torch.ones(8, dtype=torch.float32, device="cuda")
    g = torch.zeros(24, dtype=torch.float32, device="cuda")
    dE = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = vdwnl.lib()
    import ctypes
    rc = lib.vdw_delta_energy_noalloc(ctx._h, ctypes.c_void_p(n.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                      16777216 + 1, 1.0, ctypes.c_void_p(dE.data_ptr()), None)
    assert rc == -2
