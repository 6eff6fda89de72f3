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
import math
import time

import numpy as np

from . import learned as LR
from . import synthetic as S
from . import vdwnl

MEV_PER_HA = 27211.386245988
OUTER_ATOMS = 160                # (10,10) wall, four axial periods


def wall_lattice(n, m, a_cc=S.A_CC, axial_scale=1.0):
    """Bravais lattice of the unrolled (n, m) wall: two primitive vectors as
    rows, in (s, z) = (along the circumference, along the axis), Angstrom;
    with the circumference |C| and the axial period |T|.  C = n a1 + m a2 is
    the chiral vector of the graphene lattice (|a1| = |a2| = sqrt(3) a_cc),
    T the shortest lattice vector perpendicular to it; axial_scale stretches
    z (the synthetic armchair walls use an axial period of 2.46 A)."""
    a = np.sqrt(3.0) * a_cc
    a1 = a * np.array([np.sqrt(3.0) / 2.0, 0.5])
    a2 = a * np.array([np.sqrt(3.0) / 2.0, -0.5])
    C = n * a1 + m * a2
    dR = math.gcd(2 * m + n, 2 * n + m)
    T = ((2 * m + n) // dR) * a1 - ((2 * n + m) // dR) * a2
    c, t = C / np.linalg.norm(C), T / np.linalg.norm(T)
    A = np.array([[a1 @ c, axial_scale * (a1 @ t)], [a2 @ c, axial_scale * (a2 @ t)]])
    return A, float(np.linalg.norm(C)), float(axial_scale * np.linalg.norm(T))


def superlattice_periods(inner, outer, a_cc=S.A_CC, axial_scale=1.0, kmax=40):
    """The construction of the energy map (text before Eq. Uofx): the inner
    wall projected onto the outer surface (its circumferential coordinate
    scaled by R_out/R_in = |C_out|/|C_in|), both walls unrolled, and the
    superlattice wavevectors G = those common to both reciprocal lattices.
    Returns the periodicities 2 pi/|G| of the shortest G along the axis
    (dx_z) and along the circumference (dx_phi, measured on the outer
    circumference), both in Angstrom, the angular period dphi_deg, and the
    shortest common G (length, angle from the axis in degrees)."""
    Ai, Li, _ = wall_lattice(*inner, a_cc=a_cc, axial_scale=axial_scale)
    Ao, Lo, _ = wall_lattice(*outer, a_cc=a_cc, axial_scale=axial_scale)
    Ai = Ai * np.array([Lo / Li, 1.0])
    common = []
    for k1 in range(-kmax, kmax + 1):
        for k2 in range(-kmax, kmax + 1):
            if k1 == 0 and k2 == 0:
                continue
            G = 2.0 * np.pi * np.linalg.solve(Ao, np.array([k1, k2], np.float64))  # G . a_j = 2 pi k_j
            ki = Ai @ G / (2.0 * np.pi)
            if np.all(np.abs(ki - np.round(ki)) < 1e-6):
                common.append(G)
    common = np.array(common)
    length = np.linalg.norm(common, axis=1)
    tol = 1e-9 * length.max()
    gz = np.abs(common[np.abs(common[:, 0]) < tol, 1])
    gs = np.abs(common[np.abs(common[:, 1]) < tol, 0])
    dx_z = 2.0 * np.pi / gz.min()
    dx_phi = 2.0 * np.pi / gs.min()
    i = int(np.argmin(length))
    return dict(dx_z=float(dx_z), dx_phi=float(dx_phi), dphi_deg=float(360.0 * dx_phi / Lo),
                shortest=(float(length[i]), float(np.degrees(np.arctan2(abs(common[i, 0]), abs(common[i, 1]))))))


# the scanned (5,5)@(10,10) tube: the walls of synthetic.armchair_sites
_PERIODS = superlattice_periods((5, 5), (10, 10), axial_scale=S.T_ARM / (np.sqrt(3.0) * S.A_CC))
DZ_ANG = _PERIODS["dx_z"]         # axial period of the energy map (1.23 A)
DPHI_DEG = _PERIODS["dphi_deg"]   # rotational period of the energy map (18 degrees)


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


def translations(shape, L, sub):
    """Rigid translations of the whole cell by multiples of 1/sub of the grid
    spacing along each axis (sub^3 of them, bohr)."""
    N3, N2, N1 = shape
    h = np.asarray(L, np.float64) / np.array([N1, N2, N3], np.float64)
    f = np.arange(sub) / sub
    return [(a * h[0], b * h[1], c * h[2]) for a in f for b in f for c in f]


def scan_energies(ctx, shape, z, phi, seed, dr_out, sub, learned, batch):
    """Energies (Hartree) of the nz x nphi wall positions, each averaged over
    the sub^3 rigid translations of the whole cell: the plain path through
    the batched entry point, and the learned path (per density) if loaded.
    Averaging over translations by half a grid spacing cancels the odd
    harmonics of the energy's dependence on the position of the density
    relative to the grid (the "egg-box" term), which a rigid wall scan would
    otherwise read as part of the energy map."""
    import torch
    _, L, _ = S.tube_density_torch(seed, shape=(8, 8, 8), device="cpu")
    shifts = translations(shape, L, sub)
    jobs = [(i, j, t) for i in range(len(z)) for j in range(len(phi)) for t in shifts]
    Ep = np.zeros((len(z), len(phi)))
    El = np.zeros((len(z), len(phi)))
    E1 = torch.empty(3, dtype=torch.float64, device="cuda")
    for b0 in range(0, len(jobs), batch):
        part = jobs[b0:b0 + batch]
        ns = []
        for i, j, t in part:
            n64, _, _ = S.tube_density_torch(seed, shape=shape, shift_ang=float(z[i]), rot_deg=float(phi[j]),
                                             dr_out_ang=dr_out, origin_bohr=t, device="cuda", sites_alike=True)
            ns.append(n64.to(torch.float32))
        n = torch.stack(ns).contiguous()
        g = torch.stack([ctx.spectral_gradient(n[k]) for k in range(len(part))]).contiguous()
        E, _ = ctx.energy_potential_batched(n, g)
        Eh = E.cpu().numpy()
        for k, (i, j, _) in enumerate(part):
            Ep[i, j] += Eh[k, 0] / len(shifts)
            if learned:
                ctx.learned_energy_potential(n[k], g[k], E1)
                El[i, j] += float(E1[0]) / len(shifts)
    return Ep, (El if learned else None)


def run(nz=8, nphi=8, grids=(144, 180, 200), dr_out=(-0.2, 0.0, 0.2), seed=0, learned=True, sub=2, batch=8,
        log=print):
    """The wall scan: for each grid N x N x 72 and each outer-wall radius
    change dr (Angstrom), energies on an nz x nphi lattice of outer-wall
    shifts in [0, 2.46 A) and rotations in [0, 36 deg) (one density seed, so
    the sites move rigidly; all sites of a wall alike, so that each wall has
    its translation, rotation and screw symmetries and the energy depends on
    the wall position through the common superlattice only), averaged over the
    sub^3 half-spacing translations, and their energy maps (Eq. Uofx).  The learned path runs on
    the grids whose largest |G| lies within its knots."""
    import torch
    z = np.arange(nz) * (2.0 * DZ_ANG) / nz
    phi = np.arange(nphi) * (2.0 * DPHI_DEG) / nphi
    zz, pp = np.meshgrid(z, phi, indexing="ij")
    _, L, natoms = S.tube_density_torch(seed, shape=(8, 8, 8), device="cpu")
    mdl = None
    if learned:
        try:
            mdl = LR.load(LR.MIXED_PATH)  # trained with alike-site tubes among its densities
        except OSError as ex:
            log("learned path skipped: %s" % ex)
    t0 = time.time()
    cases = []
    for N in grids:
        shape = (72, N, N)
        ctx = vdwnl.VdwNL(vdwnl.Params()).plan(shape, L)
        ctx.plan_batch(batch)
        use_l = False
        if mdl is not None:
            try:
                params = torch.tensor(mdl["params"], dtype=torch.float32, device="cuda")
                ctx.learned_load(params, mdl["J"], mdl["k_max"], mdl["feat"], mdl["base"])
                ctx.learned_tabulate(LR.TAB_T, LR.TAB_D)
                use_l = True
            except vdwnl.VdwError as ex:
                log("grid %d: learned path skipped (%s)" % (N, ex))
        for dr in dr_out:
            Ep, El = scan_energies(ctx, shape, z, phi, seed, dr, sub, use_l, batch)
            r_out = 3.0 * S.A_CC * 10 / (2.0 * np.pi) + dr
            case = dict(grid=N, dr_out_ang=dr,
                        plain=fit_energy_map(zz, pp, (Ep - Ep.mean()) * MEV_PER_HA / OUTER_ATOMS, r_out),
                        E_plain_ha=Ep.tolist())
            if El is not None:
                case["learned"] = fit_energy_map(zz, pp, (El - El.mean()) * MEV_PER_HA / OUTER_ATOMS, r_out)
                case["learned_minus_plain_mev_per_atom"] = float(np.abs(El - Ep).max() * MEV_PER_HA / natoms)
                case["E_learned_ha"] = El.tolist()
            cases.append(case)
            log(json.dumps({k: v for k, v in case.items() if not k.startswith("E_")}))
        ctx.close()
    torch.cuda.synchronize()
    return dict(nz=nz, nphi=nphi, sub=sub, seconds=time.time() - t0, dx_z_ang=DZ_ANG,
                dx_phi_ang=_PERIODS["dx_phi"], dphi_deg=DPHI_DEG, cases=cases)


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="outer-wall shift/rotation scan and Eq. (Uofx) fit")
    ap.add_argument("--nz", type=int, default=8)
    ap.add_argument("--nphi", type=int, default=8)
    ap.add_argument("--grids", default="144,180,200")
    ap.add_argument("--dr", default="-0.2,0,0.2")
    ap.add_argument("--sub", type=int, default=2)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run(a.nz, a.nphi, grids=tuple(int(x) for x in a.grids.split(",")),
              dr_out=tuple(float(x) for x in a.dr.split(",")), sub=a.sub)
    if a.out:
        json.dump(res, open(a.out, "w"))
