"""Pins of the oracle's energy and potential (no GPU).

* FFT path == Eq. (Eofni) summed directly in real space, for any periodic
  grid kernel K_ab(r_i - r_j) (circular convolution theorem); u_a of
  Eq. (epsilon) likewise.
* Property (i) of the paper: a uniform density gives E_soft + Delta E = 0 up
  to the interpolation error (pins phi_ab(k=0), C_s and the sign and factor
  of Delta E, Eqs. DEnl/Depsnl).
* Property (ii) and the paper's check against direct evaluation of Eq. (Enl):
  the interaction of two separated fragments equals the unfactored direct
  double sum within the interpolation error.
* v = (1/dOmega) dE/dn_i (Eq. Vi) against central differences of E.
* E is invariant under translation of the density by a grid vector.
* The spectral gradient is exact for band-limited periodic functions.
* The factorisation of Eq. (phi) against the unfactored grid sum (reported,
  bounded).
"""
import numpy as np
import pytest

import oracle as O
from paper_0812_0244_gb300 import synthetic as S


def small_density(seed=0, shape=(10, 8, 12), L=(9.0, 8.0, 10.0)):
    # two Gaussians in a small orthorhombic cell
    L = np.asarray(L)
    rng = np.random.default_rng(seed)
    centers = [0.5 * L - 1.0, 0.5 * L + 1.2]
    n, g = S._gaussian_sum(shape, L, centers, rng.uniform(0.1, 0.6, 2), rng.uniform(0.9, 1.5, 2), 1e-4)
    return n, g, L


def test_spectral_gradient_exact_for_band_limited():
    shape = (8, 10, 12)
    L = np.array([7.0, 9.0, 11.0])
    z, y, x = np.meshgrid(*(np.arange(N) * Ld / N for N, Ld in zip(shape, L[::-1])), indexing="ij")
    f = np.sin(2 * np.pi * 2 * x / L[0]) + np.cos(2 * np.pi * 3 * y / L[1]) * np.sin(2 * np.pi * z / L[2])
    g = O.spectral_gradient(f, L)
    gx = 2 * np.pi * 2 / L[0] * np.cos(2 * np.pi * 2 * x / L[0])
    gy = -2 * np.pi * 3 / L[1] * np.sin(2 * np.pi * 3 * y / L[1]) * np.sin(2 * np.pi * z / L[2])
    gz = 2 * np.pi / L[2] * np.cos(2 * np.pi * 3 * y / L[1]) * np.cos(2 * np.pi * z / L[2])
    np.testing.assert_allclose(g[0], gx, atol=1e-12)
    np.testing.assert_allclose(g[1], gy, atol=1e-12)
    np.testing.assert_allclose(g[2], gz, atol=1e-12)
    # the derivative is antisymmetric: <a, D b> = -<D a, b>
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=shape), rng.normal(size=shape)
    for c in range(3):
        lhs = np.sum(a * O.spectral_gradient(b, L)[c])
        rhs = -np.sum(O.spectral_gradient(a, L)[c] * b)
        assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_fft_path_equals_real_space_double_sum(table):
    n, g, L = small_density(1, shape=(6, 4, 8), L=(8.0, 7.0, 9.0))
    shape = n.shape
    N = n.size
    dOmega = np.prod(L) / N
    Nq = table.p.Nq
    R = O.min_image_distances(shape, L)
    rng = np.random.default_rng(2)
    c = rng.normal(size=(Nq, Nq))
    c = c + c.T
    s = rng.uniform(1.0, 3.0, size=(Nq, Nq))
    s = 0.5 * (s + s.T)
    K = c[:, :, None, None, None] * np.exp(-R[None, None] ** 2 / (2 * s[:, :, None, None, None] ** 2))
    Khat = dOmega * np.fft.fftn(K, axes=(2, 3, 4))
    Kflat = np.real(Khat).reshape(Nq, Nq, -1)  # K even in the displacement => real
    r = O.energy_potential(n, g, L, table, kernel_hat=lambda a, b: Kflat[:, :, a:b])
    theta = r["theta"]
    E_bf = O.factored_bruteforce_energy(theta, K, dOmega)
    assert abs(r["E_soft"] - E_bf) < 1e-12 * abs(E_bf)
    # Eq. (epsilon): u_ai = dOmega sum_b sum_j theta_bj K_ab(r_i - r_j)
    idx = np.array(np.unravel_index(np.arange(N), shape)).T
    for i in [0, 7, 55, N - 1]:
        disp = (idx[i][None, :] - idx) % np.array(shape)
        Kij = K[:, :, disp[:, 0], disp[:, 1], disp[:, 2]]
        u_ref = dOmega * np.einsum("abj,bj->a", Kij, theta.reshape(Nq, -1))
        np.testing.assert_allclose(r["u"].reshape(Nq, -1)[:, i], u_ref, rtol=1e-10, atol=1e-12 * np.abs(u_ref).max())


@pytest.mark.parametrize("nval", [0.003, 0.05, 0.5, 3.0])
def test_property_i_uniform_density(table, nval):
    d = S.uniform_density((6, 6, 6), (10.0, 11.0, 12.0), nval)
    r = O.energy_potential(d["n"], d["grad"], d["L"], table)
    assert r["dE"] > 0 and r["E_soft"] < 0
    # residual = interpolation error of the q mesh (largest near q_c, ~1%)
    assert abs(r["E_soft"] + r["dE"]) < 2e-2 * r["dE"]


@pytest.mark.slow
def test_property_ii_and_direct_evaluation(table):
    """Separated fragments: FFT method vs unfactored direct sum of Eq. (Enl)."""
    shape, cell = (40, 40, 40), 40.0
    out = []
    for R in (10.0, 14.0):
        A = S.fragments_density(R, shape=shape, cell=cell, which="A", floor=0)
        B = S.fragments_density(R, shape=shape, cell=cell, which="B", floor=0)
        AB = S.fragments_density(R, shape=shape, cell=cell, which="AB", floor=0)
        e = (O.energy(AB["n"], AB["grad"], AB["L"], table) - O.energy(A["n"], A["grad"], A["L"], table)
             - O.energy(B["n"], B["grad"], B["L"], table))
        dct = O.direct_interaction_energy(A["n"], A["grad"], B["n"], B["grad"], A["L"], table, n_cut=1e-7)
        assert e < 0 and dct < 0
        assert abs(e / dct - 1) < 5e-2, (R, e, dct)
        out.append(dct)
    # the direct sum of two compact fragments falls off as R^-6 up to finite-size
    # corrections of relative order sigma^2/R^2
    slope = np.log(out[1] / out[0]) / np.log(14.0 / 10.0)
    assert -7.2 < slope < -6.0


def test_potential_matches_fd_of_energy(table):
    n, _, L = small_density(3, shape=(8, 6, 10), L=(8.0, 7.0, 9.0))
    E0 = lambda m: O.energy(m, O.spectral_gradient(m, L), L, table)
    g = O.spectral_gradient(n, L)
    r = O.energy_potential(n, g, L, table)
    v = r["v"]
    dOmega = np.prod(L) / n.size
    rng = np.random.default_rng(4)
    pts = [np.unravel_index(i, n.shape) for i in rng.choice(n.size, 6, replace=False)]
    pts.append(np.unravel_index(np.argmax(n), n.shape))
    for pt in pts:
        h = 1e-4 * n[pt]
        m1, m2 = n.copy(), n.copy()
        m1[pt] += h
        m2[pt] -= h
        fdv = (E0(m1) - E0(m2)) / (2 * h * dOmega)
        assert abs(fdv - v[pt]) < 1e-6 * np.abs(v).max(), (pt, fdv, v[pt])


def test_translation_invariance(table):
    n, g, L = small_density(4, shape=(8, 6, 10), L=(8.0, 7.0, 9.0))
    E1 = O.energy_potential(n, g, L, table)
    sh = (3, 2, 5)
    E2 = O.energy_potential(np.roll(n, sh, axis=(0, 1, 2)), np.roll(g, sh, axis=(1, 2, 3)), L, table)
    assert abs(E1["E"] - E2["E"]) < 1e-12 * abs(E1["E"])
    np.testing.assert_allclose(np.roll(E1["v"], sh, axis=(0, 1, 2)), E2["v"], atol=1e-12 * np.abs(E1["v"]).max())


@pytest.mark.slow
def test_factorisation_error_is_small(table):
    """Eq. (phi) replaces phi(q_i r, q_j r) by its cubic-spline interpolation in
    (q_i, q_j); compare the factored and unfactored grid double sums with the
    same minimum-image kernel on a tiny grid."""
    n, g, L = small_density(6, shape=(4, 4, 6), L=(6.0, 6.0, 8.0))
    shape = n.shape
    N = n.size
    dOmega = np.prod(L) / N
    Nq = table.p.Nq
    R = O.min_image_distances(shape, L)
    rv, inv = np.unique(R.ravel(), return_inverse=True)
    qm = table.qm
    K = np.zeros((Nq, Nq, rv.size))
    for a in range(Nq):
        for b in range(a, Nq):
            K[a, b] = K[b, a] = O.phi_soft_points(qm[a] * rv, qm[b] * rv, table.p, table.phi0)
    K = K[:, :, inv].reshape((Nq, Nq) + shape)
    theta = O.pointwise(n, g, table)["theta"]
    E_fac = O.factored_bruteforce_energy(theta, K, dOmega)
    E_unf = O.unfactored_bruteforce_energy(n, g, L, table)
    assert abs(E_fac / E_unf - 1) < 2e-2, (E_fac, E_unf)


def test_stencil_potential_matches_fd_of_energy(table):
    """With grad n from central differences, v = v_loc - (stencil divergence
    of w) is the exact derivative of E(n, D_fd n): central differences of E
    at single points agree with it."""
    n, _, L = small_density(5, shape=(8, 6, 10), L=(8.0, 7.0, 9.0))
    E0 = lambda m: O.energy(m, O.stencil_gradient(m, L), L, table)
    r = O.energy_potential(n, O.stencil_gradient(n, L), L, table, gradient="stencil")
    v = r["v"]
    dOmega = np.prod(L) / n.size
    rng = np.random.default_rng(6)
    for i in rng.choice(n.size, 6, replace=False):
        pt = np.unravel_index(i, n.shape)
        h = 1e-4 * n[pt]
        m1, m2 = n.copy(), n.copy()
        m1[pt] += h
        m2[pt] -= h
        fdv = (E0(m1) - E0(m2)) / (2 * h * dOmega)
        assert abs(fdv - v[pt]) < 1e-6 * np.abs(v).max(), (pt, fdv, v[pt])


def test_stencil_gradient_of_a_sine():
    """The central difference of sin(k x) on the periodic grid is, in closed
    form, cos(k x) sin(k h)/h; the other components vanish."""
    shape = (6, 8, 10)
    L = np.array([5.0, 6.0, 7.0])
    z, y, x = np.meshgrid(*(np.arange(N) * Ld / N for N, Ld in zip(shape, L[::-1])), indexing="ij")
    k = 2 * np.pi / L[0]
    f = np.sin(k * x)
    g = O.stencil_gradient(f, L)
    h = L[0] / shape[2]
    np.testing.assert_allclose(g[0], k * np.cos(k * x) * np.sin(k * h) / (k * h), atol=1e-12)
    np.testing.assert_allclose(g[1], 0.0, atol=1e-12)
    np.testing.assert_allclose(g[2], 0.0, atol=1e-12)
