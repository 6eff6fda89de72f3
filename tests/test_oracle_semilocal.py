"""Pins of the semilocal partner terms (oracle/semilocal.py)."""
import numpy as np

import oracle as O
import oracle.semilocal as SL
from paper_0812_0244_gb300 import synthetic as S


def test_uniform_gas_is_dirac_exchange():
    """grad n = 0: F_x = 1, e_x = -(3/4)(3/pi)^(1/3) n^(4/3) (Dirac)."""
    n = np.array([1e-4, 0.01, 0.3, 2.0])
    e, de, _ = SL.exchange_revpbe(n, np.zeros((3, 4)))
    np.testing.assert_allclose(e, -0.75 * (3 / np.pi) ** (1 / 3) * n ** (4 / 3), rtol=1e-14)
    np.testing.assert_allclose(de, -(3 / np.pi) ** (1 / 3) * n ** (1 / 3), rtol=1e-14)


def test_enhancement_factor_limits():
    """F_x -> 1 + mu s^2 for small s and -> 1 + kappa (the revPBE bound) for large s."""
    n = np.full(3, 0.1)
    kF = (3 * np.pi ** 2 * 0.1) ** (1 / 3)
    e0 = -0.75 * (3 / np.pi) ** (1 / 3) * 0.1 ** (4 / 3)
    for s, Fref, tol in [(1e-3, 1 + SL.MU * 1e-6, 1e-12), (1e4, 1 + SL.KAPPA, 1e-6)]:
        g = np.zeros((3, 3))
        g[0] = s * 2 * kF * 0.1
        e, _, _ = SL.exchange_revpbe(n, g)
        np.testing.assert_allclose(e / e0, Fref, rtol=tol)


def test_gradient_coefficient_is_ma_brueckner():
    """mu = beta pi^2 / 3 with beta = 16 (3 pi^2)^(1/3) C_c(0) / pi, the
    high-density gradient coefficient C_c(0) = 4.235e-3 of Ma and Brueckner:
    the small-s slope of the oracle's F_x, read off e_x itself."""
    n = np.full(3, 0.2)
    kF = (3 * np.pi ** 2 * 0.2) ** (1 / 3)
    e0 = -0.75 * (3 / np.pi) ** (1 / 3) * 0.2 ** (4 / 3)
    s = 1e-4
    g = np.zeros((3, 3))
    g[1] = s * 2 * kF * 0.2
    e, _, _ = SL.exchange_revpbe(n, g)
    slope = (e[0] / e0 - 1.0) / s ** 2
    beta = 16.0 * (3 * np.pi ** 2) ** (1 / 3) * 4.235e-3 / np.pi
    assert abs(slope - beta * np.pi ** 2 / 3) < 2e-5


def test_energy_density_derivatives_match_fd():
    rng = np.random.default_rng(0)
    n = 10 ** rng.uniform(-4, 0.5, 20)
    g = rng.normal(0, 0.3, (3, 20)) * n
    e, de, ge = SL.exchange_revpbe(n, g)
    h = 1e-6 * n
    fd = (SL.exchange_revpbe(n + h, g)[0] - SL.exchange_revpbe(n - h, g)[0]) / (2 * h)
    np.testing.assert_allclose(de, fd, rtol=1e-6)
    for c in range(3):
        hg = 1e-6 * (np.abs(g[c]) + n)
        gp, gm = g.copy(), g.copy()
        gp[c] += hg
        gm[c] -= hg
        fdg = (SL.exchange_revpbe(n, gp)[0] - SL.exchange_revpbe(n, gm)[0]) / (2 * hg)
        np.testing.assert_allclose(ge * g[c], fdg, rtol=1e-5, atol=1e-12)
    ec, dec = SL.correlation_lda(n)
    fdc = (SL.correlation_lda(n + h)[0] - SL.correlation_lda(n - h)[0]) / (2 * h)
    np.testing.assert_allclose(dec, fdc, rtol=1e-6)


def test_xc_potential_matches_fd_of_energy(table):
    """v of E_xc (nonlocal + semilocal) is dE_xc/dn_i / dOmega with grad n = D n."""
    L = np.array([8.0, 7.0, 9.0])
    rng = np.random.default_rng(5)
    n, _ = S._gaussian_sum((8, 6, 10), L, [0.5 * L - 1.0, 0.5 * L + 1.2], rng.uniform(0.1, 0.6, 2),
                           rng.uniform(0.9, 1.5, 2), 1e-4)
    for gradient, D in [("spectral", O.spectral_gradient), ("stencil", O.stencil_gradient)]:
        r = SL.xc_energy_potential(n, D(n, L), L, table, gradient=gradient)
        dOmega = np.prod(L) / n.size
        for i in rng.choice(n.size, 4, replace=False):
            pt = np.unravel_index(i, n.shape)
            h = 1e-4 * n[pt]
            m1, m2 = n.copy(), n.copy()
            m1[pt] += h
            m2[pt] -= h
            E1 = SL.xc_energy_potential(m1, D(m1, L), L, table, gradient=gradient)["E_xc"]
            E2 = SL.xc_energy_potential(m2, D(m2, L), L, table, gradient=gradient)["E_xc"]
            fd = (E1 - E2) / (2 * h * dOmega)
            assert abs(fd - r["v"][pt]) < 1e-6 * np.abs(r["v"]).max(), (gradient, pt, fd, r["v"][pt])
