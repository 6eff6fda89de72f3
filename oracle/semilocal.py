"""FP64 oracle of the semilocal partner terms of vdW-DF (Eq. Exc).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper writes the functional as E_xc = E_x^GGA + E_c^LDA + E_c^nl
(Eq. Exc), with Dion et al.'s choices: revPBE exchange (Zhang and Yang,
PRL 80, 890, 1998) and LDA correlation (Perdew and Wang 1992, the eps_c of
the q0 construction).  Per grid point, with k_F = (3 pi^2 n)^(1/3) and
s = |grad n| / (2 k_F n):

  e_x = n eps_x^unif(n) F_x(s),  eps_x^unif = -3 k_F / (4 pi),
  F_x = 1 + kappa - kappa / (1 + mu s^2 / kappa),
  e_c = n eps_c^PW92(r_s),

E_x = dOmega sum_i e_x,i and E_c^LDA = dOmega sum_i e_c,i.  The potential
adds de/dn to v_loc and de/d(grad n) to w, whose divergence enters v through
the same gradient operator as the nonlocal term (Eq. Vi).

Parity unpinned: revPBE's kappa = 1.245 (a fitted value) is restated from
the published paper, which is not at hand.  mu = beta pi^2 / 3 is pinned
through beta's definition by the Ma-Brueckner high-density gradient
coefficient; the uniform-gas limit (the Dirac exchange), the large-gradient
limit F_x -> 1 + kappa and every derivative are pinned.
"""
from __future__ import annotations

import numpy as np

from . import vdw_oracle as V

KAPPA = 1.245
MU = 0.066725 * np.pi ** 2 / 3.0


def exchange_revpbe(n, grad, n_min=1e-12):
    """e_x, de_x/dn and (de_x/d|grad n|)/|grad n| (coefficient of grad n in
    de_x/d(grad n)); zero where n <= n_min."""
    n = np.asarray(n, np.float64)
    ok = np.isfinite(n) & (n > n_min)
    ns = np.where(ok, n, 1.0)
    g2 = np.sum(np.asarray(grad, np.float64) ** 2, axis=0)
    kF = (3.0 * np.pi ** 2 * ns) ** (1.0 / 3.0)
    Ax = -0.75 * (3.0 / np.pi) ** (1.0 / 3.0)          # n eps_x^unif = Ax n^(4/3)
    s2 = g2 / (4.0 * kF * kF * ns * ns)
    den = 1.0 + MU * s2 / KAPPA
    Fx = 1.0 + KAPPA - KAPPA / den
    dF = MU / (den * den)                                # dF_x / d(s^2)
    e0 = Ax * ns ** (4.0 / 3.0)
    e = e0 * Fx
    de_dn = (4.0 / 3.0) * Ax * ns ** (1.0 / 3.0) * Fx + e0 * dF * (-(8.0 / 3.0) * s2 / ns)
    de_dg = e0 * dF * 2.0 / (4.0 * kF * kF * ns * ns)
    z = np.zeros_like(n)
    return np.where(ok, e, z), np.where(ok, de_dn, z), np.where(ok, de_dg, z)


def correlation_lda(n, n_min=1e-12):
    """e_c = n eps_c(r_s) (PW92, unpolarised) and de_c/dn."""
    n = np.asarray(n, np.float64)
    ok = np.isfinite(n) & (n > n_min)
    ns = np.where(ok, n, 1.0)
    rs = (3.0 / (4.0 * np.pi * ns)) ** (1.0 / 3.0)
    eps, deps = V.pw92_eps_c(rs)
    e = ns * eps
    de = eps + ns * deps * (-rs / (3.0 * ns))
    z = np.zeros_like(n)
    return np.where(ok, e, z), np.where(ok, de, z)


def xc_energy_potential(n, grad, cell, T: V.KernelTable, gradient="spectral"):
    """E_xc of Eq. (Exc) and its potential: the nonlocal part from the plain
    oracle plus the semilocal terms, all through one gradient operator."""
    L = V.check_cell(cell)
    dOmega = float(np.prod(L)) / n.size
    r = V.energy_potential(n, grad, L, T, gradient=gradient)
    ex, dex, gex = exchange_revpbe(n, grad, T.p.n_min)
    ec, dec = correlation_lda(n, T.p.n_min)
    w_sl = gex[None] * np.asarray(grad, np.float64)
    div = V.stencil_divergence(w_sl, L) if gradient == "stencil" else V.spectral_divergence(w_sl, L)
    Ex = dOmega * float(np.sum(ex))
    Ec = dOmega * float(np.sum(ec))
    return dict(E_xc=r["E"] + Ex + Ec, E_nl=r["E"], E_x=Ex, E_c=Ec,
                v=r["v"] + dex + dec - div, v_nl=r["v"])
