"""Pins of the learned-basis oracle (oracle/learned.py) against things other
than itself: brute-force rounding, torch's Linear/SiLU, exact reproduction of
linear functions by the knot interpolation, the real-space double sum, and
finite differences of the oracle's own energy and loss."""
import numpy as np
import pytest

import oracle as O
import oracle.learned as LO
from paper_0812_0244_gb300 import synthetic as S

ALL_BF16 = None


def _all_bf16():
    """Every finite bfloat16 value, from its bit patterns."""
    global ALL_BF16
    if ALL_BF16 is None:
        bits = (np.arange(65536, dtype=np.uint32) << 16).view(np.float32)
        bits = bits[np.isfinite(bits)].astype(np.float64)
        ALL_BF16 = np.unique(bits)
    return ALL_BF16


def _nearest_bf16_bruteforce(x):
    vals = _all_bf16()
    i = np.searchsorted(vals, x)
    lo, hi = vals[max(i - 1, 0)], vals[min(i, vals.size - 1)]
    dl, dh = abs(x - lo), abs(hi - x)
    if dl < dh:
        return lo
    if dh < dl:
        return hi
    # tie: the one with an even last significand bit
    lb = np.array([lo], np.float32).view(np.uint32)[0] >> 16
    return lo if lb % 2 == 0 else hi


def test_bf16_round_is_nearest_ties_even():
    rng = np.random.default_rng(0)
    xs = list(rng.normal(0, 3, 400)) + list(10.0 ** rng.uniform(-30, 30, 200) * rng.choice([-1, 1], 200))
    # exact ties: midpoints between neighbouring bf16 values
    v = _all_bf16()
    k = rng.integers(1, v.size - 2, 100)
    xs += list(0.5 * (v[k] + v[k + 1]))
    for x in xs:
        assert LO.bf16_round(np.array([x]))[0] == _nearest_bf16_bruteforce(x), x
    assert LO.bf16_round(np.array([0.0]))[0] == 0.0


def test_mlp_forward_matches_torch_linear_silu():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    mdl = LO.random_model(3)
    rng = np.random.default_rng(1)
    x1, x2 = rng.normal(0, 1.5, 300), rng.normal(0, 1.5, 300)
    f = LO.mlp_forward(x1, x2, mdl)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    bf = lambda a: a.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    X = t(np.stack([x1, x2], 1))
    h1 = bf(F.silu(F.linear(X, bf(t(mdl.W1)), t(mdl.b1))))
    h2 = bf(F.silu(F.linear(h1, bf(t(mdl.W2)), t(mdl.b2))))
    w = F.linear(h2, bf(t(mdl.W3)), t(mdl.b3))
    np.testing.assert_allclose(f["w"].T, w.numpy(), rtol=1e-12, atol=1e-12)


def test_knot_interpolation_catmull_rom():
    """The knot interpolation passes through the knots, reproduces quadratics
    away from the ends (Catmull-Rom is exact for polynomials of degree <= 2
    on uniform knots), continues an even function evenly through k = 0 and a
    linear one linearly past the last knot."""
    mdl = LO.random_model(4, M=3, J=32, k_max=10.0)
    kj = np.arange(mdl.J) * mdl.dk
    a0 = np.linspace(-1, 1, mdl.P)
    a1 = np.linspace(0.3, -0.2, mdl.P)
    a2 = np.linspace(0.05, 0.1, mdl.P)
    rng = np.random.default_rng(2)
    # through the knots
    mdl.K = rng.normal(size=(mdl.P, mdl.J))
    Kk = LO.kernel_eval(mdl, kj)
    for p, (m, n) in enumerate(LO.pair_index(mdl.M)):
        np.testing.assert_allclose(Kk[m, n], mdl.K[p], atol=1e-14)
        np.testing.assert_array_equal(Kk[m, n], Kk[n, m])
    # quadratics on the interior intervals
    mdl.K = a0[:, None] + a1[:, None] * kj[None] + a2[:, None] * kj[None] ** 2
    k = rng.uniform(kj[1], kj[-2], 500)
    Kk = LO.kernel_eval(mdl, k)
    for p, (m, n) in enumerate(LO.pair_index(mdl.M)):
        np.testing.assert_allclose(Kk[m, n], a0[p] + a1[p] * k + a2[p] * k ** 2, atol=1e-12)
    # even quadratic through k = 0 (the mirrored knot K_-1 = K_1)
    mdl.K = a0[:, None] + a2[:, None] * kj[None] ** 2
    k = rng.uniform(0.0, kj[1], 200)
    Kk = LO.kernel_eval(mdl, k)
    for p, (m, n) in enumerate(LO.pair_index(mdl.M)):
        np.testing.assert_allclose(Kk[m, n], a0[p] + a2[p] * k ** 2, atol=1e-12)
    # linear past the last interval's far knot
    mdl.K = a0[:, None] + a1[:, None] * kj[None]
    k = rng.uniform(kj[-2], kj[-1], 200)
    Kk = LO.kernel_eval(mdl, k)
    for p, (m, n) in enumerate(LO.pair_index(mdl.M)):
        np.testing.assert_allclose(Kk[m, n], a0[p] + a1[p] * k, atol=1e-12)


def test_learned_energy_equals_real_space_double_sum(table):
    """E_soft and u against 1/2 dOmega^2 sum_ij theta_mi theta_nj K_mn(r_i - r_j)
    with the periodic kernel K(D) = (1/Omega) sum_G K_mn(|G|) exp(i G.D)."""
    shape = (6, 7, 8)
    L = np.array([9.0, 10.0, 11.0])
    d = S.two_atom_density(5, shape=shape, cell_ang=5.5)
    n, g = d["n"], d["grad"]
    mdl = LO.random_model(5, M=3, J=64, k_max=6.0)
    r = LO.energy_potential(n, g, L, mdl, table, want_v=False, want_grad=True)
    N = n.size
    Omega = float(np.prod(L))
    dOmega = Omega / N
    g1, g2, g3 = O.g_vectors(shape, L)
    kmod = np.sqrt(g1 * g1 + g2 * g2 + g3 * g3).ravel()
    Khat = LO.kernel_eval(mdl, kmod).reshape((3, 3) + shape)
    K = np.real(np.fft.ifftn(Khat, axes=(2, 3, 4))) * N / Omega
    E_bf = O.factored_bruteforce_energy(r["theta"], K, dOmega)
    assert abs(r["E_soft"] - E_bf) < 1e-12 * abs(E_bf)
    idx = np.array(np.unravel_index(np.arange(N), shape)).T
    for i in [0, 11, N - 1]:
        disp = (idx[i][None, :] - idx) % np.array(shape)
        Kij = K[:, :, disp[:, 0], disp[:, 1], disp[:, 2]]
        u_ref = dOmega * np.einsum("abj,bj->a", Kij, r["theta"].reshape(3, -1))
        np.testing.assert_allclose(r["u"].reshape(3, -1)[:, i], u_ref, rtol=1e-10,
                                   atol=1e-12 * np.abs(u_ref).max())


def _tiny(seed=7, shape=(10, 8, 12), L=(9.0, 8.0, 10.0)):
    """Two wide Gaussians over a 1e-4 floor: smooth enough on a coarse grid
    that single-point central differences through the spectral gradient
    converge (at sharp features over a 1e-6 floor they do not)."""
    L = np.asarray(L)
    rng = np.random.default_rng(seed)
    centers = [0.5 * L - 1.0, 0.5 * L + 1.2]
    n, _ = S._gaussian_sum(shape, L, centers, rng.uniform(0.1, 0.6, 2), rng.uniform(0.9, 1.5, 2), 1e-4)
    return n, O.spectral_gradient(n, L), L


@pytest.mark.parametrize("base", [(0.0, 0.0), (0.6, 1.45)], ids=["network", "spline_base"])
def test_learned_potential_matches_finite_differences(table, monkeypatch, base):
    """v (exact Jacobian-vector product) = dE/dn_i / dOmega with grad n = D n,
    with and without the spline base.  The activations' bf16 rounding makes E
    piecewise constant in n, so this pin runs with it off; the bf16 product is
    then compared with the exact one."""
    n, g, L = _tiny()
    mdl = LO.random_model(6, base=base)
    rb = LO.energy_potential(n, g, L, mdl, table, jac_bf16=True)
    monkeypatch.setattr(LO, "bf16_round", lambda a: np.asarray(a, np.float64))
    r = LO.energy_potential(n, g, L, mdl, table, jac_bf16=False)
    dOmega = float(np.prod(L)) / n.size
    rng = np.random.default_rng(3)
    vmax = np.abs(r["v"]).max()
    for i in rng.choice(n.size, 6, replace=False):
        pt = np.unravel_index(i, n.shape)
        h = 1e-4 * n[pt]
        m1, m2 = n.copy(), n.copy()
        m1[pt] += h
        m2[pt] -= h
        E1 = LO.energy(m1, O.spectral_gradient(m1, L), L, mdl, table)
        E2 = LO.energy(m2, O.spectral_gradient(m2, L), L, mdl, table)
        fd = (E1 - E2) / (2 * h) / dOmega
        assert abs(fd - r["v"][pt]) < 1e-6 * vmax, (pt, fd, r["v"][pt])
    # the model evaluated with its bf16 roundings stays within their size
    # (2^-9 relative per rounded value)
    assert np.abs(rb["v"] - r["v"]).max() < 5e-2 * vmax


def test_learned_param_grad_matches_finite_differences(table, monkeypatch):
    """dE/dparams against central differences along single parameters and a
    random direction.  The activations' bf16 rounding makes E piecewise
    constant in the weights, so the network pins run with it switched off
    (the backpropagation formulas do not change)."""
    n, g, L = _tiny()
    mdl = LO.random_model(8)
    monkeypatch.setattr(LO, "bf16_round", lambda a: np.asarray(a, np.float64))
    G = LO.energy_grad(n, g, L, mdl, table)
    p0 = mdl.flat()
    sizes = [int(np.prod(s)) for s in LO.LearnedModel.sizes(mdl.M, mdl.J)]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(9)
    picks = [offs[0] + 5, offs[1] + 3, offs[2] + 130, offs[3] + 7, offs[4] + 77, offs[5] + 2,
             offs[6] + 2 * mdl.J + 3, offs[6] + 17 * mdl.J]
    E = lambda p: LO.energy(n, g, L, mdl.with_flat(p), table)
    for k in picks:
        h = 1e-5 * max(1.0, abs(p0[k]))
        e = np.zeros_like(p0)
        e[k] = h
        fd = (E(p0 + e) - E(p0 - e)) / (2 * h)
        assert abs(fd - G[k]) < 1e-6 * np.abs(G).max() + 1e-5 * abs(G[k]), (k, fd, G[k])
    dirn = rng.normal(size=p0.size)
    h = 1e-6
    fd = (E(p0 + h * dirn) - E(p0 - h * dirn)) / (2 * h)
    an = float(G @ dirn)
    assert abs(fd - an) < 1e-6 * abs(an)


def test_learned_loss_grad_matches_finite_differences(table, monkeypatch):
    """The potential term of the loss gradient through the directional
    derivative of dE/dp, against central differences of the loss itself."""
    n, g, L = _tiny(11)
    monkeypatch.setattr(LO, "bf16_round", lambda a: np.asarray(a, np.float64))
    mdl_ref = LO.random_model(12)
    ref = LO.energy_potential(n, g, L, mdl_ref, table, jac_bf16=False)
    mdl = LO.random_model(13)
    a, b = 1e4, 1e2
    G = LO.loss_grad(n, L, mdl, table, ref["E"], ref["v"], 2, a=a, b=b)
    p0 = mdl.flat()
    rng = np.random.default_rng(14)
    Lf = lambda p: LO.loss(n, L, mdl.with_flat(p), table, ref["E"], ref["v"], 2, a=a, b=b)[0]
    for trial in range(2):
        dirn = rng.normal(size=p0.size)
        h = 1e-5
        fd = (Lf(p0 + h * dirn) - Lf(p0 - h * dirn)) / (2 * h)
        an = float(G @ dirn)
        assert abs(fd - an) < 1e-5 * abs(an), (fd, an)
    # the potential term alone is not negligible in this check
    Gv = LO.loss_grad(n, L, mdl, table, ref["E"], ref["v"], 2, a=0.0, b=b)
    assert np.abs(Gv).max() > 1e-2 * np.abs(G).max()


def test_fit_grad_matches_finite_differences(monkeypatch):
    """Regression gradient of the channel weights against central differences."""
    monkeypatch.setattr(LO, "bf16_round", lambda a: np.asarray(a, np.float64))
    n, g, L = _tiny(21)
    mdl = LO.random_model(22)
    rng = np.random.default_rng(23)
    target = rng.normal(0, 0.3, (mdl.M,) + n.shape)
    weight = n / n.sum()
    G = LO.fit_grad(n, g, mdl, target, weight, 1e-12)

    def F(p):
        m = mdl.with_flat(p)
        ft = LO.features(n, g, m, 1e-12)
        w = LO.mlp_forward(ft["x1"].ravel(), ft["x2"].ravel(), m)["w"]
        return float(np.sum(weight.ravel() * np.sum((w - target.reshape(mdl.M, -1)) ** 2, axis=0)))

    p0 = mdl.flat()
    dirn = rng.normal(size=p0.size)
    h = 1e-6
    fd = (F(p0 + h * dirn) - F(p0 - h * dirn)) / (2 * h)
    assert abs(fd - float(G @ dirn)) < 1e-6 * abs(fd)


def test_spline_base_reproduces_plain_method_basis(table):
    """With the network's output switched off (W3 = 0, b3 = 0) and an M-point
    base mesh, the channels are the plain method's cardinal weights on that
    mesh: theta_m = n p_m(q) (Eq. fofx), against the plain oracle's pointwise
    evaluation with an M-point table."""
    n, g, L = _tiny(31)
    mdl = LO.random_model(32, base=(0.6, 1.45))
    mdl.W3[:] = 0.0
    mdl.b3[:] = 0.0
    r = LO.energy_potential(n, g, L, mdl, table, want_v=False)
    p8 = O.Params(Nq=8, q_1=0.6, lam=1.45)
    qm = O.q_mesh(p8)
    T8 = O.KernelTable(p=p8, qm=qm, Mq=O.cardinal_M(qm), phi0=0.0, C_s=table.C_s, k=None, phik=None)
    pw = O.pointwise(n, g, T8)
    np.testing.assert_allclose(r["theta"], pw["theta"], rtol=1e-12, atol=1e-15)


def test_catmull_rom_weights_reproduce_quadratics():
    """The Catmull-Rom weights of nodes -1, 0, 1, 2 at s in [0, 1]: a partition
    of unity whose interpolant and s derivative are exact for polynomials of
    degree up to two, and which passes through nodes 0 and 1."""
    s = np.linspace(0.0, 1.0, 101)
    w, dw = LO.catmull_rom(s)
    np.testing.assert_allclose(w.sum(0), 1.0, atol=1e-14)
    np.testing.assert_allclose(dw.sum(0), 0.0, atol=1e-13)
    nodes = np.array([-1.0, 0.0, 1.0, 2.0])
    for f, df in ((lambda x: 0 * x + 1.0, lambda x: 0 * x), (lambda x: x, lambda x: 0 * x + 1.0),
                  (lambda x: 3 - 2 * x + 0.5 * x * x, lambda x: -2 + x)):
        np.testing.assert_allclose((w * f(nodes)[:, None]).sum(0), f(s), atol=1e-13)
        np.testing.assert_allclose((dw * f(nodes)[:, None]).sum(0), df(s), atol=1e-12)
    np.testing.assert_allclose(w[:, 0], [0, 1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(w[:, -1], [0, 0, 1, 0], atol=1e-15)


def test_network_table_reproduces_quadratics_and_clamps():
    """A table filled from biquadratic functions (one per channel) gives them
    and their gradients back exactly inside [-D, D]; outside, the feature is
    clamped to the edge and the derivative along that axis is zero."""
    T, D, M = 17, 3.0, 3
    xs = -D + (np.arange(T + 2) - 1.0) * (2.0 * D / (T - 1))
    X1, X2 = np.meshgrid(xs, xs, indexing="ij")
    coef = np.array([[0.3, 1.0, -2.0, 0.5, -0.25, 0.7], [-1.0, 0.2, 0.4, -0.3, 0.1, 0.05], [2.0, 0, 0, 1.0, 0, 0]])

    def g(c, a, b):
        return c[0] + c[1] * a + c[2] * b + c[3] * a * b + c[4] * a * a + c[5] * b * b

    def dg(c, a, b):
        return c[1] + c[3] * b + 2 * c[4] * a, c[2] + c[3] * a + 2 * c[5] * b

    tab = LO.NetworkTable(T=T, D=D, vals=np.stack([g(c, X1, X2) for c in coef]))
    rng = np.random.default_rng(5)
    a, b = rng.uniform(-D, D, 200), rng.uniform(-D, D, 200)
    o, J = tab_eval = LO.table_eval(tab, a, b)
    for m, c in enumerate(coef):
        np.testing.assert_allclose(o[m], g(c, a, b), atol=1e-12)
        d1, d2 = dg(c, a, b)
        np.testing.assert_allclose(J[m, 0], d1, atol=1e-11)
        np.testing.assert_allclose(J[m, 1], d2, atol=1e-11)
    o2, J2 = LO.table_eval(tab, np.array([D + 1.0, 0.3]), np.array([0.2, -D - 2.0]))
    for m, c in enumerate(coef):
        np.testing.assert_allclose(o2[m], g(c, np.array([D, 0.3]), np.array([0.2, -D])), atol=1e-12)
        np.testing.assert_allclose(J2[m, 0], [0.0, dg(c, 0.3, -D)[0]], atol=1e-11)
        np.testing.assert_allclose(J2[m, 1], [dg(c, D, 0.2)[1], 0.0], atol=1e-11)


def test_tabulated_potential_matches_finite_differences(table, monkeypatch):
    """With the network tabulated, E is smooth in n even with the bf16
    roundings of the network (the table is fixed): v = dE/dn_i / dOmega by
    central differences at seeded points.  With the roundings off (the network
    then smooth) the tabulated outputs converge to the network's at third
    order in the node spacing h."""
    n, g, L = _tiny()
    mdl = LO.random_model(6, base=(0.6, 1.45))
    tab = LO.network_table(mdl, 129, 8.0)
    r = LO.energy_potential(n, g, L, mdl, table, table=tab)
    dOmega = float(np.prod(L)) / n.size
    rng = np.random.default_rng(4)
    vmax = np.abs(r["v"]).max()
    for i in rng.choice(n.size, 6, replace=False):
        pt = np.unravel_index(i, n.shape)
        h = 1e-4 * n[pt]
        m1, m2 = n.copy(), n.copy()
        m1[pt] += h
        m2[pt] -= h
        E1 = LO.energy_potential(m1, O.spectral_gradient(m1, L), L, mdl, table, want_v=False, table=tab)["E"]
        E2 = LO.energy_potential(m2, O.spectral_gradient(m2, L), L, mdl, table, want_v=False, table=tab)["E"]
        fd = (E1 - E2) / (2 * h) / dOmega
        assert abs(fd - r["v"][pt]) < 1e-6 * vmax, (pt, fd, r["v"][pt])
    monkeypatch.setattr(LO, "bf16_round", lambda a: np.asarray(a, np.float64))
    ft = LO.features(n, g, mdl, 1e-12)
    od = LO.mlp_forward(ft["x1"].ravel(), ft["x2"].ravel(), mdl)["w"]
    errs = []
    for T in (65, 129, 257):
        ot, _ = LO.table_eval(LO.network_table(mdl, T, 8.0), ft["x1"].ravel(), ft["x2"].ravel())
        errs.append(np.abs(ot - od).max())
    assert errs[1] < errs[0] / 5 and errs[2] < errs[1] / 5, errs
    assert errs[2] < 1e-4 * np.abs(od).max(), errs
