"""Wall translation and rotation scan of the double-wall tube, and the
energy-map fit of the paper's Eq. (Uofx) to the nonlocal correlation energy.

Eq. (Uofx) expands the energy of the outer wall's position x on its
configuration surface as U(x) = U0 - 1/4 sum_{G != 0} U_G cos(G . x) over the
superlattice wavevectors; keeping the two stars +-G1 (along the axis) and
+-G2 (around it), as the paper does, each star's two vectors give
1/2 U_G cos(G . x):

    U(z, s) = U0 - 1/2 U_z cos(2 pi z / dz) - 1/2 U_phi cos(2 pi s / ds)

with z the axial shift and s = R_out phi the arc length of the rotation of
the outer wall.  For the armchair (5,5)@(10,10) tube the periods are half the
axial period (dz = 1.23 A) and half the outer wall's 36-degree rotational
period (ds = the arc of 18 degrees at R_out).

The energies come from the library (plain Nq = 20 path, and the learned
8-channel path when a trained model is stored); the fit is a linear least
squares in (U0, U_z, U_phi).  Energies per outer-tube atom in meV, the unit
of the paper's Table I.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import learned as LR
from . import synthetic as S
from . import vdwnl

MEV_PER_HA = 27211.386245988
DZ_ANG = 0.5 * S.T_ARM          # axial period of the energy map
DPHI_DEG = 18.0                  # rotational period of the energy map
OUTER_ATOMS = 160                # (10,10) wall, four axial periods


def fit_energy_map(z_ang, phi_deg, E_mev, r_out_ang):
    """Least-squares U0, U_z, U_phi of the two-star form of Eq. (Uofx) and the
    RMS residual (same units as E)."""
    z = np.asarray(z_ang, np.float64).ravel()
    s = np.deg2rad(np.asarray(phi_deg, np.float64).ravel()) * r_out_ang
    ds = np.deg2rad(DPHI_DEG) * r_out_ang
    A = np.stack([np.ones_like(z), -0.5 * np.cos(2 * np.pi * z / DZ_ANG), -0.5 * np.cos(2 * np.pi * s / ds)], axis=1)
    coef, *_ = np.linalg.lstsq(A, np.asarray(E_mev, np.float64).ravel(), rcond=None)
    resid = np.asarray(E_mev, np.float64).ravel() - A @ coef
    return dict(U0=float(coef[0]), U_z=float(coef[1]), U_phi=float(coef[2]),
                rms=float(np.sqrt(np.mean(resid ** 2))))


def run(nz=8, nphi=8, shape=(72, 180, 180), seed=0, learned=True, log=print):
    """Energies on an nz x nphi lattice of outer-wall shifts in [0, 2.46 A)
    and rotations in [0, 36 deg) (one density seed, so the sites move
    rigidly), their energy maps, and the timing."""
    import torch
    z = np.arange(nz) * (2.0 * DZ_ANG) / nz
    phi = np.arange(nphi) * (2.0 * DPHI_DEG) / nphi
    _, L, natoms = S.tube_density_torch(seed, shape=(8, 8, 8), device="cpu")
    ctx = vdwnl.VdwNL(vdwnl.Params()).plan(shape, L)
    mdl = None
    if learned:
        try:
            mdl = LR.load()
            params = torch.tensor(mdl["params"], dtype=torch.float32, device="cuda")
            ctx.learned_load(params, mdl["J"], mdl["k_max"], mdl["feat"], mdl["base"])
        except (OSError, vdwnl.VdwError) as ex:
            log("learned path skipped: %s" % ex)
            mdl = None
    Ep = np.zeros((nz, nphi))
    El = np.zeros((nz, nphi))
    E = torch.empty(3, dtype=torch.float64, device="cuda")
    t0 = time.time()
    for i, zi in enumerate(z):
        for j, pj in enumerate(phi):
            n64, _, _ = S.tube_density_torch(seed, shape=shape, shift_ang=float(zi), rot_deg=float(pj), device="cuda")
            n = n64.to(torch.float32).contiguous()
            g = ctx.spectral_gradient(n)
            ctx.energy_potential(n, g, E)
            Ep[i, j] = float(E[0])
            if mdl is not None:
                ctx.learned_energy_potential(n, g, E)
                El[i, j] = float(E[0])
    torch.cuda.synchronize()
    zz, pp = np.meshgrid(z, phi, indexing="ij")
    r_out = 3.0 * S.A_CC * 10 / (2.0 * np.pi)
    out = dict(nz=nz, nphi=nphi, shape=list(shape), seconds=time.time() - t0,
               plain=fit_energy_map(zz, pp, (Ep - Ep.mean()) * MEV_PER_HA / OUTER_ATOMS, r_out),
               E_plain_ha=Ep.tolist())
    if mdl is not None:
        out["learned"] = fit_energy_map(zz, pp, (El - El.mean()) * MEV_PER_HA / OUTER_ATOMS, r_out)
        out["learned_minus_plain_mev_per_atom"] = float(np.abs(El - Ep).max() * MEV_PER_HA / natoms)
        out["E_learned_ha"] = El.tolist()
    log(json.dumps({k: v for k, v in out.items() if not k.startswith("E_")}))
    return out


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="outer-wall shift/rotation scan and Eq. (Uofx) fit")
    ap.add_argument("--nz", type=int, default=8)
    ap.add_argument("--nphi", type=int, default=8)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run(a.nz, a.nphi)
    if a.out:
        json.dump(res, open(a.out, "w"))
