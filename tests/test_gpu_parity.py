"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on a GB300.

Tolerances: |Delta E| <= 1e-6 Ha per cell and max|Delta v| <= 1e-5 max|v|
(FP32 FFTs and contraction, FP64 energy accumulation).  Both sides get the
same FP32-rounded inputs; each builds its own kernel table (the oracle in
numpy/C, the library in FP64 CUDA kernels) and the tables are compared too.
"""
import numpy as np
import pytest

import oracle as O
from paper_0812_0244_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

E_TOL = 1e-6
V_REL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def vd(torch_cuda):
    from paper_0812_0244_gb300 import vdwnl
    vdwnl.lib()
    return vdwnl


@pytest.fixture(scope="module")
def ctx(vd):
    return vd.VdwNL(vd.Params())


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def run_gpu(torch, ctx, n, g, L, want_v=True, want_w=False):
    ctx.plan(n.shape, L)
    nt = torch.tensor(np.asarray(n, np.float32), device="cuda")
    gt = torch.tensor(np.asarray(g, np.float32), device="cuda")
    E, v, w = ctx.compute(nt, gt, want_v=want_v, want_w=want_w)
    torch.cuda.synchronize()
    return (E.cpu().numpy(), None if v is None else v.cpu().numpy().astype(np.float64),
            None if w is None else w.cpu().numpy().astype(np.float64))


def test_kernel_table_parity(vd, table):
    t = vd.kernel_table(vd.Params())
    np.testing.assert_allclose(t["q_mesh"], table.qm, rtol=1e-15)
    assert abs(t["phi0"] - table.phi0) < 1e-12 * abs(table.phi0)
    assert abs(t["C_s"] - table.C_s) < 1e-11 * abs(table.C_s)
    scale = np.abs(table.phik).max(axis=2, keepdims=True)
    assert np.max(np.abs(t["phi_k"] - table.phik) / scale) < 1e-10


CASES = [
    # (N3, N2, N1), L (bohr)   -- spans pencil tiles with ragged tails, odd N2
    ((8, 10, 12), (9.0, 8.0, 10.0)),
    ((12, 15, 16), (10.0, 11.0, 12.0)),
    ((16, 27, 20), (11.0, 12.0, 13.0)),
    ((24, 24, 24), None),
]


@pytest.mark.parametrize("shape,L", CASES)
def test_energy_potential_small(torch_cuda, ctx, table, shape, L):
    if L is None:
        d = S.two_atom_density(0, shape=shape)
        n, g, L = d["n"], d["grad"], d["L"]
    else:
        L = np.asarray(L)
        rng = np.random.default_rng(sum(shape))
        n, g = S._gaussian_sum(shape, L, [0.4 * L, 0.6 * L + 0.3], rng.uniform(0.1, 1.0, 2), rng.uniform(0.6, 1.4, 2),
                               1e-5)
    n, g = f32(n), f32(g)
    ref = O.energy_potential(n, g, L, table)
    E, v, _ = run_gpu(torch_cuda, ctx, n, g, L)
    assert abs(E[1] - ref["E_soft"]) <= E_TOL, (E, ref["E_soft"])
    assert abs(E[2] - ref["dE"]) <= E_TOL, (E, ref["dE"])
    assert abs(E[0] - ref["E"]) <= E_TOL
    assert np.max(np.abs(v - ref["v"])) <= V_REL * np.abs(ref["v"]).max()


def test_gradient_outputs_and_energy_only(torch_cuda, ctx, table):
    d = S.two_atom_density(3, shape=(12, 12, 12))
    n, g, L = f32(d["n"]), f32(d["grad"]), d["L"]
    ref = O.energy_potential(n, g, L, table)
    E, vloc, w = run_gpu(torch_cuda, ctx, n, g, L, want_v=True, want_w=True)
    assert np.max(np.abs(vloc - ref["v_loc"])) <= V_REL * np.abs(ref["v_loc"]).max()
    assert np.max(np.abs(w - ref["w"])) <= V_REL * np.abs(ref["w"]).max()
    E2, _, _ = run_gpu(torch_cuda, ctx, n, g, L, want_v=False, want_w=False)
    assert abs(E2[0] - E[0]) <= 1e-12 * abs(E[0])


def test_uniform_density_property_i(torch_cuda, ctx):
    for nval in (0.01, 0.5):
        d = S.uniform_density((8, 8, 8), (10.0, 11.0, 12.0), nval)
        E, v, _ = run_gpu(torch_cuda, ctx, d["n"], d["grad"], d["L"])
        assert abs(E[1] + E[2]) < 2e-2 * E[2]


def test_invalid_points_are_counted_and_zeroed(torch_cuda, ctx, table):
    d = S.two_atom_density(1, shape=(8, 8, 8))
    n = f32(d["n"])
    n[0, 0, 0] = -1.0
    n[1, 2, 3] = np.nan
    g = f32(d["grad"])
    E, v, _ = run_gpu(torch_cuda, ctx, n, g, d["L"])
    assert ctx.invalid_points() == 2
    assert np.isfinite(E).all() and np.isfinite(v).all()
    n0 = n.copy()
    n0[0, 0, 0] = 0.0
    n0[1, 2, 3] = 0.0
    ref = O.energy_potential(n0, g, d["L"], table)
    assert abs(E[0] - ref["E"]) <= E_TOL


def test_host_entry_point_matches_device(torch_cuda, ctx):
    d = S.two_atom_density(2, shape=(12, 12, 12))
    n, g, L = d["n"], d["grad"], d["L"]
    E, v, _ = run_gpu(torch_cuda, ctx, n, g, L)
    Eh, vh = ctx.energy_potential_host(n.astype(np.float32), g.astype(np.float32))
    assert np.array_equal(Eh, E)
    assert np.array_equal(vh.astype(np.float64), v)


def test_plan_rejects_bad_grids(vd, ctx):
    with pytest.raises(vd.VdwError) as e:
        ctx.plan((8, 8, 14), (10.0, 10.0, 10.0))  # N1 = 14 = 2 * 7
    assert e.value.code == -2
    with pytest.raises(vd.VdwError) as e:
        ctx.plan((9, 8, 8), (10.0, 10.0, 10.0))   # N3 odd
    assert e.value.code == -2
    with pytest.raises(vd.VdwError) as e:
        ctx.plan((8, 8, 8), (0.5, 10.0, 10.0))    # |G|max beyond k_max
    assert e.value.code == -2


@pytest.mark.slow
def test_nanotube_cell_full_size(torch_cuda, ctx, table):
    """The 180 x 180 x 72 double-wall tube (the benchmark workload)."""
    d = S.tube_density(0)
    n, g, L = f32(d["n"]), f32(d["grad"]), d["L"]
    E, v, _ = run_gpu(torch_cuda, ctx, n, g, L)
    ref = O.energy_potential(n, g, L, table)
    assert abs(E[0] - ref["E"]) <= E_TOL, (E, ref["E"])
    assert abs(E[1] - ref["E_soft"]) <= E_TOL
    assert np.max(np.abs(v - ref["v"])) <= V_REL * np.abs(ref["v"]).max()


@pytest.mark.parametrize("shape", [(24, 24, 24), (72, 180, 180)], ids=["two_atom_24", "tube_180x180x72"])
def test_finite_difference_gradient_variant(torch_cuda, table, shape):
    """vdw_energy_potential_fd against the oracle with the same central-
    difference gradient; grad = NULL gives the library's own stencil."""
    torch = torch_cuda
    from paper_0812_0244_gb300 import vdwnl
    d = S.two_atom_density(9, shape=shape) if shape[0] == 24 else S.tube_density(4)
    n32 = d["n"].astype(np.float32)
    L = d["L"]
    g = O.stencil_gradient(n32.astype(np.float64), L)
    ctx = vdwnl.VdwNL(vdwnl.Params()).plan(n32.shape, L)
    nt = torch.tensor(n32, device="cuda")
    gt = torch.tensor(g.astype(np.float32), device="cuda")
    v = torch.empty_like(nt)
    E, _ = ctx.energy_potential_fd(nt, gt, v=v)
    ref = O.energy_potential(n32.astype(np.float64), g.astype(np.float32).astype(np.float64), L, table,
                             gradient="stencil")
    assert abs(float(E[0]) - ref["E"]) <= E_TOL
    vv = v.cpu().numpy()
    assert np.abs(vv - ref["v"]).max() <= V_REL * np.abs(ref["v"]).max()
    # the library's own stencil gradient: the same pipeline on its own result
    v2 = torch.empty_like(nt)
    E2, _ = ctx.energy_potential_fd(nt, None, v=v2)
    assert abs(float(E2[0]) - ref["E"]) <= 1e-6


@pytest.mark.parametrize("fd", [False, True], ids=["spectral", "stencil"])
def test_xc_functional_matches_oracle(torch_cuda, table, fd):
    """E_xc = E_x^revPBE + E_c^LDA + E_c^nl (Eq. Exc) and its potential."""
    torch = torch_cuda
    import oracle.semilocal as SL
    from paper_0812_0244_gb300 import vdwnl
    d = S.two_atom_density(10, shape=(24, 24, 24))
    n32 = d["n"].astype(np.float32)
    L = d["L"]
    n64 = n32.astype(np.float64)
    g = (O.stencil_gradient if fd else O.spectral_gradient)(n64, L).astype(np.float32)
    ctx = vdwnl.VdwNL(vdwnl.Params()).plan(n32.shape, L)
    v = torch.empty(n32.shape, dtype=torch.float32, device="cuda")
    E, _ = ctx.xc_energy_potential(torch.tensor(n32, device="cuda"), torch.tensor(g, device="cuda"), v, fd=fd)
    E = E.cpu().numpy()
    ref = SL.xc_energy_potential(n64, g.astype(np.float64), L, table, gradient="stencil" if fd else "spectral")
    assert abs(E[1] - ref["E_nl"]) <= E_TOL
    assert abs(E[2] - ref["E_x"]) <= 1e-6 * abs(ref["E_x"])
    assert abs(E[3] - ref["E_c"]) <= 1e-6 * abs(ref["E_c"])
    assert abs(E[0] - ref["E_xc"]) <= 1e-6 * abs(ref["E_xc"])
    vv = v.cpu().numpy()
    assert np.abs(vv - ref["v"]).max() <= V_REL * np.abs(ref["v"]).max()


def test_two_live_contexts_of_different_grids(torch_cuda, vd, table):
    """The dynamic shared-memory limit of a kernel is process-wide: a context
    planned for a smaller grid after one for a larger grid (both on the
    runtime-length kernels) must not lower the larger one's limit.  Both keep
    working, interleaved, and match the oracle."""
    torch = torch_cuda
    big = S.two_atom_density(5, shape=(30, 36, 40))
    small = S.two_atom_density(6, shape=(8, 10, 12))
    cb = vd.VdwNL(vd.Params()).plan(big["n"].shape, big["L"])
    cs = vd.VdwNL(vd.Params()).plan(small["n"].shape, small["L"])
    for _ in range(2):
        for c, d in ((cb, big), (cs, small)):
            n, g = f32(d["n"]), f32(d["grad"])
            E, v, _ = c.compute(torch.tensor(np.asarray(n, np.float32), device="cuda"),
                                torch.tensor(np.asarray(g, np.float32), device="cuda"))
            torch.cuda.synchronize()
            ref = O.energy_potential(n, g, d["L"], table)
            assert abs(float(E[0]) - ref["E"]) <= E_TOL
            vv = v.cpu().numpy().astype(np.float64)
            assert np.max(np.abs(vv - ref["v"])) <= V_REL * np.abs(ref["v"]).max()


def test_plan_cell_takes_orthorhombic_cells(torch_cuda, vd, table):
    """vdw_plan_cell with a diagonal cell is vdw_plan with its diagonal; a
    skewed cell is refused and leaves the context's plan in place."""
    torch = torch_cuda
    d = S.two_atom_density(11, shape=(12, 12, 12))
    n, g, L = f32(d["n"]), f32(d["grad"]), d["L"]
    c = vd.VdwNL(vd.Params()).plan_cell(n.shape, np.diag(L))
    nt = torch.tensor(np.asarray(n, np.float32), device="cuda")
    gt = torch.tensor(np.asarray(g, np.float32), device="cuda")
    E, v, _ = c.compute(nt, gt)
    torch.cuda.synchronize()
    ref = O.energy_potential(n, g, L, table)
    assert abs(float(E[0]) - ref["E"]) <= E_TOL
    skew = np.diag(L)
    skew[1, 0] = 0.5
    with pytest.raises(vd.VdwError) as e:
        c.plan_cell(n.shape, skew)
    assert e.value.code == -6
    E2, _, _ = c.compute(nt, gt)
    torch.cuda.synchronize()
    assert float(E2[0]) == float(E[0])
