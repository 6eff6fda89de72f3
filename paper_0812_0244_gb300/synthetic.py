"""Seeded synthetic electron densities on periodic grids.

This module only draws inputs: sums of isotropic Gaussians placed at atomic
sites, with their analytic gradients.  It holds none of the method's
arithmetic, so both the CUDA library's tests and the CPU oracle may take their
inputs from it.

The paper's densities come from SIESTA runs of double-wall carbon nanotubes
(Sec. on DWNTs), which are not available; these generators stand in for them:

* ``two_atom_density``: a cubic 10 A cell with two "atoms" 3 A apart along
  (1,1,1)/sqrt(3), each a sum of three Gaussians with amplitudes U(0.05, 2)
  e/bohr^3 and widths U(0.3, 1.5) bohr, plus a 1e-6 floor.
* ``tube_density``: an armchair (5,5)@(10,10) double-wall tube, carbon sites
  on cylinders of radius 3a_cc n/(2 pi) (3.39 A and 6.78 A), four axial
  periods of 2.46 A in a 25 x 25 x 9.84 A cell, each site carrying 4 e as a
  two-Gaussian sum (widths U(0.4, 1.2) bohr), plus a 1e-6 floor.  The outer
  wall can be shifted along the axis, rotated, and both radii varied.

Arrays have shape (N3, N2, N1) with x (axis 1) fastest; cells are
orthorhombic, given as the three edge lengths in bohr.
"""
from __future__ import annotations

import numpy as np

BOHR_PER_ANG = 1.0 / 0.529177210903
A_CC = 1.42  # carbon-carbon distance, Angstrom
T_ARM = 2.46  # axial period of an armchair tube, Angstrom


def _gaussian_sum(shape, L, centers, amps, sigmas, floor, cut=8.0):
    """n(r) = floor + sum_g A_g exp(-|r - c_g|^2 / (2 s_g^2)) summed over periodic
    images, and its analytic gradient.  Each Gaussian is evaluated on the grid
    points within cut*s_g of one of its images."""
    N3, N2, N1 = shape
    L = np.asarray(L, np.float64)
    h = L / np.array([N1, N2, N3], np.float64)
    n = np.full(shape, float(floor))
    g = np.zeros((3,) + tuple(shape))
    for c, A, s in zip(centers, amps, sigmas):
        R = cut * s
        idx = []
        dis = []
        for d, Nd in enumerate((N1, N2, N3)):
            lo = int(np.floor((c[d] - R) / h[d]))
            hi = int(np.ceil((c[d] + R) / h[d]))
            ii = np.arange(lo, hi + 1)
            if ii.size > Nd:  # box wider than the cell: one full period, minimum image
                ii = np.arange(Nd)
                x = ii * h[d] - c[d]
                x = x - L[d] * np.round(x / L[d])
            else:
                x = ii * h[d] - c[d]
            idx.append(np.mod(ii, Nd))
            dis.append(x)
        x, y, z = dis
        r2 = x[None, None, :] ** 2 + y[None, :, None] ** 2 + z[:, None, None] ** 2
        val = A * np.exp(-r2 / (2.0 * s * s))
        ix = np.ix_(idx[2], idx[1], idx[0])
        np.add.at(n, ix, val)
        f = -val / (s * s)
        np.add.at(g[0], ix, f * x[None, None, :])
        np.add.at(g[1], ix, f * y[None, :, None])
        np.add.at(g[2], ix, f * z[:, None, None])
    return n, g


def _gaussian_sum_torch(shape, L, centers, amps, sigmas, floor, device, cut=8.0):
    """Density part of _gaussian_sum evaluated with torch on a device (FP64):
    the same Gaussians, boxes and images.  A Gaussian's box is the tensor
    product of one index range per axis and its value the product of three
    1D profiles, so the whole sum is sum_g A_g pz_g (x) py_g (x) px_g over
    profiles that vanish outside each box: one matrix product."""
    import torch
    N3, N2, N1 = shape
    L = np.asarray(L, np.float64)
    h = L / np.array([N1, N2, N3], np.float64)
    G = len(centers)
    prof = []
    for d, Nd in enumerate((N1, N2, N3)):
        P = np.zeros((G, Nd))
        for k, (c, s) in enumerate(zip(centers, sigmas)):
            R = cut * s
            lo = int(np.floor((c[d] - R) / h[d]))
            hi = int(np.ceil((c[d] + R) / h[d]))
            ii = np.arange(lo, hi + 1)
            if ii.size > Nd:
                ii = np.arange(Nd)
                x = ii * h[d] - c[d]
                x = x - L[d] * np.round(x / L[d])
            else:
                x = ii * h[d] - c[d]
            np.add.at(P[k], np.mod(ii, Nd), np.exp(-x * x / (2.0 * s * s)))
        prof.append(torch.as_tensor(P, dtype=torch.float64, device=device))
    px, py, pz = prof
    A = torch.as_tensor(np.asarray(amps, np.float64), device=device)
    M = (py[:, :, None] * px[:, None, :]).reshape(G, N2 * N1)
    n = ((pz * A[:, None]).transpose(0, 1) @ M).reshape(N3, N2, N1)
    return n + float(floor)


def tube_density_torch(seed=0, shape=(72, 180, 180), inner=5, outer=10, shift_ang=0.0, rot_deg=0.0,
                       dr_in_ang=0.0, dr_out_ang=0.0, cell_ang=(25.0, 25.0, 9.84), floor=1e-6, device="cuda",
                       origin_bohr=(0.0, 0.0, 0.0), sites_alike=False):
    """tube_density's density (same seeded draws) evaluated on a torch device;
    returns (n as an FP64 tensor, L, natoms).  For generating many training
    densities quickly; the gradient is left to the caller.  origin_bohr moves
    the whole tube rigidly (periodic images included); sites_alike as in
    tube_density."""
    rng = np.random.default_rng(seed)
    L = np.asarray(cell_ang, np.float64) * BOHR_PER_ANG
    R_in = 3.0 * A_CC * inner / (2.0 * np.pi) + dr_in_ang
    R_out = 3.0 * A_CC * outer / (2.0 * np.pi) + dr_out_ang
    n_periods = int(round(cell_ang[2] / T_ARM))
    s_in = armchair_sites(inner, R_in, n_periods)
    s_out = armchair_sites(outer, R_out, n_periods, np.deg2rad(rot_deg), shift_ang)
    sites = np.concatenate([s_in, s_out]) * BOHR_PER_ANG
    sites[:, 0] += 0.5 * L[0] + origin_bohr[0]
    sites[:, 1] += 0.5 * L[1] + origin_bohr[1]
    sites[:, 2] = np.mod(sites[:, 2] + origin_bohr[2], L[2])
    centers, amps, sigmas = _site_gaussians(rng, sites, len(s_in), sites_alike)
    n = _gaussian_sum_torch(shape, L, centers, amps, sigmas, floor, device)
    return n, L, len(sites)


def two_atom_density(seed=0, shape=(24, 24, 24), cell_ang=10.0, sep_ang=3.0, floor=1e-6):
    """Two three-Gaussian 'atoms' in a cubic cell (the small plain-method case)."""
    rng = np.random.default_rng(seed)
    Lb = cell_ang * BOHR_PER_ANG
    L = np.array([Lb, Lb, Lb])
    u = np.ones(3) / np.sqrt(3.0)
    half = 0.5 * sep_ang * BOHR_PER_ANG
    centers, amps, sigmas = [], [], []
    for sgn in (-1.0, 1.0):
        c = 0.5 * L + sgn * half * u
        for _ in range(3):
            centers.append(c)
            amps.append(rng.uniform(0.05, 2.0))
            sigmas.append(rng.uniform(0.3, 1.5))
    n, g = _gaussian_sum(shape, L, centers, amps, sigmas, floor)
    return dict(n=n, grad=g, L=L, natoms=2, centers=np.array(centers))


def armchair_sites(nidx, radius_ang, n_periods=4, phase_rad=0.0, z_shift_ang=0.0):
    """Carbon positions of an armchair (n,n) tube (Angstrom, axis along z through
    the origin).  The unrolled sheet repeats, every 3 a_cc around the
    circumference, four atoms at (0,0), (a_cc,0), (1.5 a_cc, T/2),
    (2.5 a_cc, T/2); wrapping n repeats onto radius R gives R = 3 a_cc n/(2 pi)
    unless a radius is given."""
    basis = np.array([[0.0, 0.0], [A_CC, 0.0], [1.5 * A_CC, 0.5 * T_ARM], [2.5 * A_CC, 0.5 * T_ARM]])
    circ = 3.0 * A_CC * nidx
    out = []
    for per in range(n_periods):
        for rep in range(nidx):
            for bx, bz in basis:
                s = rep * 3.0 * A_CC + bx
                phi = 2.0 * np.pi * s / circ + phase_rad
                out.append((radius_ang * np.cos(phi), radius_ang * np.sin(phi),
                            per * T_ARM + bz + z_shift_ang))
    return np.array(out)


def _site_gaussians(rng, sites, n_inner, alike):
    """Two Gaussians per site carrying 4 e: charge split w : 1 - w with
    w ~ U(0.3, 0.7) and widths ~ U(0.4, 1.2) bohr, drawn per site, or once per
    wall when alike (every site of a wall the same, as carbon atoms are)."""
    def draw():
        w = rng.uniform(0.3, 0.7)
        return w, rng.uniform(0.4, 1.2), rng.uniform(0.4, 1.2)

    wall = (draw(), draw()) if alike else None
    centers, amps, sigmas = [], [], []
    for i, c in enumerate(sites):
        w, s1, s2 = wall[0 if i < n_inner else 1] if alike else draw()
        for q, s in ((4.0 * w, s1), (4.0 * (1.0 - w), s2)):
            centers.append(c)
            amps.append(q / ((2.0 * np.pi) ** 1.5 * s ** 3))
            sigmas.append(s)
    return centers, amps, sigmas


def tube_density(seed=0, shape=(72, 180, 180), inner=5, outer=10, shift_ang=0.0, rot_deg=0.0,
                 dr_in_ang=0.0, dr_out_ang=0.0, cell_ang=(25.0, 25.0, 9.84), floor=1e-6, sites_alike=False):
    """Double-wall armchair tube density (4 e per carbon site, two Gaussians
    each).  sites_alike: one set of Gaussian parameters per wall, so that the
    density has the tube's translation, rotation and screw symmetries (the
    wall scan needs them); otherwise independent parameters per site."""
    rng = np.random.default_rng(seed)
    L = np.asarray(cell_ang, np.float64) * BOHR_PER_ANG
    R_in = 3.0 * A_CC * inner / (2.0 * np.pi) + dr_in_ang
    R_out = 3.0 * A_CC * outer / (2.0 * np.pi) + dr_out_ang
    n_periods = int(round(cell_ang[2] / T_ARM))
    s_in = armchair_sites(inner, R_in, n_periods)
    s_out = armchair_sites(outer, R_out, n_periods, np.deg2rad(rot_deg), shift_ang)
    sites = np.concatenate([s_in, s_out]) * BOHR_PER_ANG
    sites[:, 0] += 0.5 * L[0]
    sites[:, 1] += 0.5 * L[1]
    sites[:, 2] = np.mod(sites[:, 2], L[2])
    centers, amps, sigmas = _site_gaussians(rng, sites, len(s_in), sites_alike)
    n, g = _gaussian_sum(shape, L, centers, amps, sigmas, floor)
    return dict(n=n, grad=g, L=L, natoms=len(sites), centers=sites)


def uniform_density(shape, L, value):
    """Constant density with zero gradient."""
    return dict(n=np.full(shape, float(value)), grad=np.zeros((3,) + tuple(shape)),
                L=np.asarray(L, np.float64), natoms=0)


def fragments_density(R, shape=(64, 64, 64), cell=40.0, sigma=1.0, charge=4.0, floor=0.0, which="AB"):
    """Two identical Gaussian fragments a distance R (bohr) apart along x (for the
    r^-6 separation test); which in {'A', 'B', 'AB'} selects the fragments."""
    L = np.array([cell, cell, cell], np.float64)
    c0 = 0.5 * L
    A = charge / ((2.0 * np.pi) ** 1.5 * sigma ** 3)
    centers, amps, sigmas = [], [], []
    if "A" in which:
        centers.append(c0 - np.array([0.5 * R, 0, 0]))
        amps.append(A)
        sigmas.append(sigma)
    if "B" in which:
        centers.append(c0 + np.array([0.5 * R, 0, 0]))
        amps.append(A)
        sigmas.append(sigma)
    n, g = _gaussian_sum(shape, L, centers, amps, sigmas, floor)
    return dict(n=n, grad=g, L=L, natoms=len(centers))
