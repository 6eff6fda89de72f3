"""Plain FP64 oracle of the Roman-Perez--Soler nonlocal-correlation evaluation.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function states
the passage of the paper it follows; where the paper is silent the reading
taken is written beside it.  Arrays on the real-space grid have shape
(N3, N2, N1) in C order, so index x = i1 runs fastest, the layout the CUDA
library uses for its flat buffers.

Paper passages (Roman-Perez & Soler, arXiv:0812.0244):
  Eq. (Enl)     E_c^nl = 1/2 Int Int n1 n2 phi(q1, q2, r12)
  Eq. (phi)     phi(q1,q2,r) ~ sum_ab phi(qa,qb,r) p_a(q1) p_b(q2)
  Eq. (fofx)    cardinal interpolation functions p_a (cubic splines)
  log mesh      (q_{a+1}-q_a) = lambda (q_a - q_{a-1}), lambda > 1
  Eqs. (qsat), (Sat)  saturation q0 -> h(q0, q_c)
  Eq. (PhiSoft) soft kernel phi0 + phi2 d^2 + phi4 d^4 for d < d_s
  Eqs. (DEnl), (Depsnl)  local correction for the softening
  Eq. (Eoffk)   E = 1/2 sum_ab Int d3k theta_a(k) theta_b(k) phi_ab(k)
  Eq. (Eofni)   grid form 1/2 dOmega^2 sum_ab sum_ij theta_ai theta_bj phi_ab(r_ij)
  Eq. (Vi)      v_i = sum_a (u_ai dtheta_ai/dn_i + sum_j u_aj dtheta_aj/dgrad_j dgrad_j/dn_i)
  Eqs. (epsilon), (epsofk)  u_a as a convolution evaluated with FFTs
Definitions the paper takes from Dion et al. (PRL 92, 246401, 2004):
  q0(n, |grad n|), the kernel phi(d1, d2) and, through q0, the LDA
  correlation of Perdew and Wang (PRB 45, 13244, 1992).

Parity unpinned: Dion's gradient coefficient Z_ab in q0 is restated from the
published paper, which is not at hand, and no test fixes its value.  The
Perdew-Wang constants are pinned through the limits their form is built to
reproduce (high- and low-density expansion coefficients) and against the
independent Perdew-Zunger fit; every derivative is pinned by finite
differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field, asdict

import numpy as np

PI = np.pi

# --------------------------------------------------------------------------
# Parameters (every number the paper leaves open is a field here)
# --------------------------------------------------------------------------


@dataclass
class Params:
    """Method parameters.

    Nq, q_c, m_c : interpolation mesh size, saturation cutoff and order
                   (paper: "N_alpha ~ 20", "m_c ~ 12 and q_c ~ 5 a.u.").
    q_1, lam     : first mesh point and ratio of the logarithmic mesh (paper
                   gives only lambda > 1; reading: q_1 = 1e-5, lambda = 1.2).
    d_s          : soft-kernel radius in d = sqrt(d1^2+d2^2) (reading: 1.0);
                   phi0 is derived so that phi4 = 0 on the diagonal ray.
    na, a_max    : Gauss-Legendre nodes in t = atan(a) on [0, atan(a_max)] for
                   the Dion double integral (reading: 256, 64).
    d_asym       : for min(d1, d2) >= d_asym the kernel takes its closed-form
                   large-separation limit -C/(d1^2 d2^2 (d1^2+d2^2)),
                   C = 12 (4 pi/9)^3 (reading: 8).
    r_c, Nr      : radial transform cut at r_c with Simpson's rule on Nr
                   intervals (reading: 100 bohr, 4096).
    k_max, Nk    : uniform k mesh of the radial table, natural cubic spline
                   in k between its Nk points (reading: 40 bohr^-1, 1024).
    n_cs         : Gauss-Legendre nodes for the softening constant C_s.
    n_min        : densities at or below n_min give theta = 0.
    """
    Nq: int = 20
    q_1: float = 1e-5
    q_c: float = 5.0
    lam: float = 1.2
    m_c: int = 12
    d_s: float = 1.0
    na: int = 256
    a_max: float = 64.0
    d_asym: float = 8.0
    r_c: float = 100.0
    Nr: int = 4096
    k_max: float = 40.0
    Nk: int = 1024
    n_cs: int = 64
    n_min: float = 1e-12

    def key(self):
        return tuple(sorted(asdict(self).items()))


# --------------------------------------------------------------------------
# LDA correlation, q0 and saturation
# --------------------------------------------------------------------------

# Perdew-Wang 1992, unpolarised parameter set (the one Dion et al. use).
PW_A, PW_ALPHA1 = 0.031091, 0.21370
PW_BETA = (7.5957, 3.5876, 1.6382, 0.49294)
Z_AB = -0.8491  # Dion et al. gradient coefficient in q0


def pw92_eps_c(rs):
    """eps_c(rs) in Hartree and d eps_c / d rs (Perdew-Wang 1992, p = 1).
    The restated constants are pinned through the limits the form is built
    to reproduce: c0 (exact), c1 and the missing sqrt(rs) term at high
    density, d0 and d1 at low density, and the Perdew-Zunger fit between."""
    rs = np.asarray(rs, dtype=np.float64)
    b1, b2, b3, b4 = PW_BETA
    srs = np.sqrt(rs)
    Q = 2.0 * PW_A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs)
    dQ = 2.0 * PW_A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs)
    L = np.log1p(1.0 / Q)
    eps = -2.0 * PW_A * (1.0 + PW_ALPHA1 * rs) * L
    deps = -2.0 * PW_A * PW_ALPHA1 * L + 2.0 * PW_A * (1.0 + PW_ALPHA1 * rs) * dQ / (Q * Q + Q)
    return eps, deps


def q0_unsaturated(n, gmod):
    """Dion et al. q0 = -(4 pi/3) eps_xc^0 with the gradient-corrected exchange.

    q0 = k_F (1 - (Z_ab/9) s^2) - (4 pi/3) eps_c^LDA(r_s),
    k_F = (3 pi^2 n)^(1/3), s = |grad n| / (2 k_F n), r_s = (3/(4 pi n))^(1/3).
    Returns q0, d q0/d n, and (d q0/d|grad n|) / |grad n| (finite at grad = 0).
    Parity unpinned for Z_ab (restated constant).
    """
    n = np.asarray(n, dtype=np.float64)
    gmod = np.asarray(gmod, dtype=np.float64)
    kF = np.cbrt(3.0 * PI * PI * n)
    rs = np.cbrt(3.0 / (4.0 * PI * n))
    s2 = gmod * gmod / (4.0 * kF * kF * n * n)
    ec, dec = pw92_eps_c(rs)
    q0 = kF * (1.0 - Z_AB / 9.0 * s2) - 4.0 * PI / 3.0 * ec
    # d kF/dn = kF/(3n), d s^2/dn = -8 s^2/(3n), d rs/dn = -rs/(3n)
    dq0_dn = (kF / (3.0 * n)
              - Z_AB / 9.0 * (kF * s2 / (3.0 * n) - kF * 8.0 * s2 / (3.0 * n))
              - 4.0 * PI / 3.0 * dec * (-rs / (3.0 * n)))
    # d q0/d|g| = -kF Z/9 * 2|g|/(4 kF^2 n^2)  =>  divided by |g|:
    dq0_dg_over_g = -Z_AB / (18.0 * kF * n * n)
    return q0, dq0_dn, dq0_dg_over_g


def saturate(x, q_c, m_c):
    """Eq. (Sat): h(x, x_c) = x_c [1 - exp(-sum_{m=1}^{m_c} (x/x_c)^m / m)] and h'(x)."""
    x = np.asarray(x, dtype=np.float64)
    y = x / q_c
    S = np.zeros_like(y)
    dS = np.zeros_like(y)  # d S / d y
    yp = np.ones_like(y)
    for m in range(1, m_c + 1):
        dS += yp
        yp = yp * y
        S += yp / m
    e = np.exp(-S)
    return q_c * (1.0 - e), e * dS


# --------------------------------------------------------------------------
# q mesh and cardinal cubic splines
# --------------------------------------------------------------------------


def q_mesh(p: Params):
    """Logarithmic mesh: (q_{a+1}-q_a) = lambda (q_a-q_{a-1}), q_1 .. q_Nq = q_c."""
    a = np.arange(p.Nq, dtype=np.float64)
    return p.q_1 + (p.q_c - p.q_1) * (p.lam ** a - 1.0) / (p.lam ** (p.Nq - 1) - 1.0)


def natural_spline_M(x, Y):
    """Second derivatives of the natural cubic splines through columns of Y.

    x: (n,) knots; Y: (n, m) data.  Solves the standard tridiagonal system
    h_{i-1} M_{i-1} + 2 (h_{i-1}+h_i) M_i + h_i M_{i+1} = 6 (slope_i - slope_{i-1})
    with M_0 = M_{n-1} = 0, as a dense linear solve (library primitive).
    """
    x = np.asarray(x, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = x.size
    h = np.diff(x)
    A = np.zeros((n, n))
    R = np.zeros((n,) + Y.shape[1:])
    A[0, 0] = A[-1, -1] = 1.0
    for i in range(1, n - 1):
        A[i, i - 1] = h[i - 1]
        A[i, i] = 2.0 * (h[i - 1] + h[i])
        A[i, i + 1] = h[i]
        R[i] = 6.0 * ((Y[i + 1] - Y[i]) / h[i] - (Y[i] - Y[i - 1]) / h[i - 1])
    return np.linalg.solve(A, R)


def cardinal_M(qm):
    """M[a, k]: second derivative at knot k of the cardinal spline p_a (Eq. fofx:
    the spline through the values f_b = delta_ab)."""
    return natural_spline_M(qm, np.eye(qm.size)).T.copy()


def q_interval(qm, q):
    """Interval index k with qm[k] <= q < qm[k+1]; a q on a knot belongs to the
    upper interval, q = q_c to the last one."""
    k = np.searchsorted(qm, q, side="right") - 1
    return np.clip(k, 0, qm.size - 2)


def cardinal_eval(qm, M, q):
    """p_a(q) and dp_a/dq for all a: arrays of shape (Nq,) + q.shape."""
    q = np.asarray(q, dtype=np.float64)
    k = q_interval(qm, q)
    x0, x1 = qm[k], qm[k + 1]
    h = x1 - x0
    A = (x1 - q) / h
    B = 1.0 - A
    Nq = qm.size
    P = np.zeros((Nq,) + q.shape)
    dP = np.zeros((Nq,) + q.shape)
    for a in range(Nq):
        ya = (k == a).astype(np.float64)
        yb = (k + 1 == a).astype(np.float64)
        Ma, Mb = M[a][k], M[a][k + 1]
        P[a] = A * ya + B * yb + ((A ** 3 - A) * Ma + (B ** 3 - B) * Mb) * h * h / 6.0
        dP[a] = (yb - ya) / h - (3.0 * A * A - 1.0) / 6.0 * h * Ma + (3.0 * B * B - 1.0) / 6.0 * h * Mb
    return P, dP


# --------------------------------------------------------------------------
# The Dion kernel (C quadrature) and the soft kernel
# --------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        bdir = os.path.join(_HERE, "_build")
        os.makedirs(bdir, exist_ok=True)
        so = os.path.join(bdir, "liboracle_dion.so")
        src = os.path.join(_HERE, "dion.c")
        def compile_():
            tmp = so + ".%d.tmp" % os.getpid()
            subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
            os.replace(tmp, so)
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            compile_()
        try:
            lib = ctypes.CDLL(so)
        except OSError:  # built for another machine
            compile_()
            lib = ctypes.CDLL(so)
        P = ctypes.POINTER(ctypes.c_double)
        lib.oracle_dion_phi.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P, P]
        lib.oracle_dion_phi.restype = None
        lib.oracle_dion_W.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.oracle_dion_W.restype = ctypes.c_double
        _LIB = lib
    return _LIB


def build_c():
    """Compile the C part of the oracle (idempotent)."""
    _lib()


def dion_nodes(na, a_max):
    """Gauss-Legendre nodes in t on [0, atan(a_max)], a = tan t, weights with da/dt."""
    t, w = np.polynomial.legendre.leggauss(na)
    T = np.arctan(a_max)
    tt = 0.5 * T * (t + 1.0)
    wt = 0.5 * T * w
    a = np.tan(tt)
    return a, wt * (1.0 + a * a)


def dion_W(a, b):
    return _lib().oracle_dion_W(float(a), float(b))


def dion_quadrature(d1, d2, na=256, a_max=64.0, deriv=False):
    """Dion et al. phi(d1, d2) by the double quadrature (no asymptote)."""
    lib = _lib()
    P = ctypes.POINTER(ctypes.c_double)
    a, wa = dion_nodes(na, a_max)
    d1, d2 = np.broadcast_arrays(np.asarray(d1, np.float64), np.asarray(d2, np.float64))
    shape = d1.shape
    d1 = np.ascontiguousarray(d1.ravel())
    d2 = np.ascontiguousarray(d2.ravel())
    out = np.zeros(d1.size)
    dout = np.zeros(d1.size) if deriv else None
    if d1.size:
        lib.oracle_dion_phi(na, a.ctypes.data_as(P), wa.ctypes.data_as(P), d1.size,
                            d1.ctypes.data_as(P), d2.ctypes.data_as(P), out.ctypes.data_as(P),
                            dout.ctypes.data_as(P) if deriv else None)
    if deriv:
        return out.reshape(shape), dout.reshape(shape)
    return out.reshape(shape)


ASYM_C = 12.0 * (4.0 * PI / 9.0) ** 3


def phi_asymptote(d1, d2):
    """Large-separation limit of the Dion kernel, -C/(d1^2 d2^2 (d1^2 + d2^2))."""
    d1 = np.asarray(d1, np.float64)
    d2 = np.asarray(d2, np.float64)
    return -ASYM_C / (d1 * d1 * d2 * d2 * (d1 * d1 + d2 * d2))


def phi_asymptote_dd(d1, d2):
    """Derivative of the asymptote along the ray: phi_asym ~ d^-6 so dphi/dd = -6 phi/d."""
    d = np.hypot(d1, d2)
    return -6.0 * phi_asymptote(d1, d2) / d


def phi_kernel(d1, d2, p: Params, deriv=False):
    """The (hard) kernel: closed-form asymptote when min(d1,d2) >= d_asym,
    otherwise the double quadrature."""
    d1, d2 = np.broadcast_arrays(np.asarray(d1, np.float64), np.asarray(d2, np.float64))
    use_a = np.minimum(d1, d2) >= p.d_asym
    out = np.zeros(d1.shape)
    dout = np.zeros(d1.shape)
    if np.any(use_a):
        out[use_a] = phi_asymptote(d1[use_a], d2[use_a])
        dout[use_a] = phi_asymptote_dd(d1[use_a], d2[use_a])
    q = ~use_a
    if np.any(q):
        r = dion_quadrature(d1[q], d2[q], p.na, p.a_max, deriv=deriv)
        if deriv:
            out[q], dout[q] = r
        else:
            out[q] = r
    return (out, dout) if deriv else out


def soft_phi0(p: Params):
    """phi0 chosen so that phi4 = 0 on the diagonal ray d1 = d2 (reading)."""
    x = p.d_s / np.sqrt(2.0)
    F, dF = phi_kernel(np.array([x]), np.array([x]), p, deriv=True)
    return float(F[0] - dF[0] * p.d_s / 2.0)


def soft_coeffs_ray(cos_psi, sin_psi, phi0, p: Params):
    """Eq. (PhiSoft): phi2, phi4 so that phi_s matches phi in value and slope at
    d = d_s on the ray (d1, d2) = d (cos psi, sin psi)."""
    F, dF = phi_kernel(p.d_s * np.asarray(cos_psi), p.d_s * np.asarray(sin_psi), p, deriv=True)
    ds = p.d_s
    phi4 = (phi0 - F + dF * ds / 2.0) / ds ** 4
    phi2 = dF / (2.0 * ds) - 2.0 * ds * ds * phi4
    return phi2, phi4


def phi_soft_points(d1, d2, p: Params, phi0=None):
    """phi_s at arbitrary points (soft polynomial inside d_s, kernel outside)."""
    d1 = np.atleast_1d(np.asarray(d1, np.float64))
    d2 = np.atleast_1d(np.asarray(d2, np.float64))
    if phi0 is None:
        phi0 = soft_phi0(p)
    d = np.hypot(d1, d2)
    out = np.zeros(d.shape)
    inner = d < p.d_s
    if np.any(~inner):
        out[~inner] = phi_kernel(d1[~inner], d2[~inner], p)
    if np.any(inner):
        di = d[inner]
        c = np.where(di > 0, d1[inner] / np.where(di > 0, di, 1.0), np.sqrt(0.5))
        s = np.where(di > 0, d2[inner] / np.where(di > 0, di, 1.0), np.sqrt(0.5))
        phi2, phi4 = soft_coeffs_ray(c, s, phi0, p)
        out[inner] = phi0 + phi2 * di ** 2 + phi4 * di ** 4
    return out


# --------------------------------------------------------------------------
# Kernel table: phi_ab(r) -> radial transform phi_ab(k), softening constant
# --------------------------------------------------------------------------


def radial_ft(fr, r, k):
    """4 pi Int_0^{r_max} r^2 f(r) j0(k r) dr by Simpson's rule on the uniform r
    mesh (len(r) odd).  fr: (m, len(r)); returns (m, len(k))."""
    nr = r.size
    assert nr % 2 == 1
    dr = r[1] - r[0]
    w = np.ones(nr)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    w *= dr / 3.0
    kr = np.outer(k, r)
    j0 = np.sinc(kr / PI)  # sin(kr)/(kr)
    J = j0 * (4.0 * PI * w * r * r)[None, :]
    return np.asarray(fr) @ J.T


def kernel_r(p: Params, qm=None, phi0=None):
    """phi_s,ab(r) = phi_s(q_a r, q_b r) on the r mesh, for the Nq(Nq+1)/2 pairs a <= b."""
    if qm is None:
        qm = q_mesh(p)
    if phi0 is None:
        phi0 = soft_phi0(p)
    r = np.linspace(0.0, p.r_c, p.Nr + 1)
    pairs = [(a, b) for a in range(p.Nq) for b in range(a, p.Nq)]
    out = np.zeros((len(pairs), r.size))
    for ip, (a, b) in enumerate(pairs):
        qa, qb = qm[a], qm[b]
        qq = np.hypot(qa, qb)
        d = qq * r
        phi2, phi4 = soft_coeffs_ray(qa / qq, qb / qq, phi0, p)
        inner = d < p.d_s
        out[ip, inner] = phi0 + phi2 * d[inner] ** 2 + phi4 * d[inner] ** 4
        out[ip, ~inner] = phi_kernel(qa * r[~inner], qb * r[~inner], p)
    return r, pairs, out


def softening_constant(p: Params, phi0=None):
    """C_s = Int_0^{d_s/sqrt2} 4 pi x^2 [phi(x,x) - phi_s(x,x)] dx (Eq. Depsnl).

    The printed upper limit is d_s with d the diagonal argument; the integrand
    vanishes for x > d_s/sqrt(2) (there phi_s = phi), so the integral is taken
    where it is nonzero, with Gauss-Legendre on n_cs nodes."""
    if phi0 is None:
        phi0 = soft_phi0(p)
    X = p.d_s / np.sqrt(2.0)
    t, w = np.polynomial.legendre.leggauss(p.n_cs)
    x = 0.5 * X * (t + 1.0)
    wx = 0.5 * X * w
    F = phi_kernel(x, x, p)
    phi2, phi4 = soft_coeffs_ray(np.sqrt(0.5), np.sqrt(0.5), phi0, p)
    d2 = 2.0 * x * x
    Fs = phi0 + phi2 * d2 + phi4 * d2 * d2
    return float(np.sum(wx * 4.0 * PI * x * x * (F - Fs)))


@dataclass
class KernelTable:
    p: Params
    qm: np.ndarray           # (Nq,) q mesh
    Mq: np.ndarray           # (Nq, Nq) cardinal-spline second derivatives
    phi0: float
    C_s: float
    k: np.ndarray            # (Nk,) uniform k mesh
    phik: np.ndarray         # (Nq, Nq, Nk) phi_ab(k), symmetric in a, b
    Mk: np.ndarray = field(default=None)  # (Nq, Nq, Nk) second derivatives in k

    @property
    def dk(self):
        return self.k[1] - self.k[0]


def build_kernel_table(p: Params) -> KernelTable:
    """phi_ab(k) = 4 pi Int_0^{r_c} r^2 phi_s(q_a r, q_b r) j0(k r) dr on a uniform
    k mesh (the paper: 'calculated in spherical coordinates, and stored in a
    radial mesh of points k'), plus C_s for Delta E."""
    qm = q_mesh(p)
    phi0 = soft_phi0(p)
    r, pairs, fr = kernel_r(p, qm, phi0)
    k = np.linspace(0.0, p.k_max, p.Nk)
    tab = radial_ft(fr, r, k)
    phik = np.zeros((p.Nq, p.Nq, p.Nk))
    for ip, (a, b) in enumerate(pairs):
        phik[a, b] = tab[ip]
        phik[b, a] = tab[ip]
    T = KernelTable(p=p, qm=qm, Mq=cardinal_M(qm), phi0=phi0, C_s=softening_constant(p, phi0),
                    k=k, phik=phik)
    T.Mk = natural_spline_M(k, phik.reshape(-1, p.Nk).T).T.reshape(p.Nq, p.Nq, p.Nk)
    return T


_TABLE_CACHE = {}


def kernel_table(p: Params | None = None) -> KernelTable:
    """Cached build_kernel_table (in memory, and on disk under oracle/_build)."""
    if p is None:
        p = Params()
    key = p.key()
    if key in _TABLE_CACHE:
        return _TABLE_CACHE[key]
    import hashlib
    import json
    h = hashlib.sha1(json.dumps(key).encode() + open(os.path.join(_HERE, "dion.c"), "rb").read()
                     + open(__file__, "rb").read()).hexdigest()[:16]
    path = os.path.join(_HERE, "_build", "ktable_%s.npz" % h)
    if os.path.exists(path):
        z = np.load(path)
        T = KernelTable(p=p, qm=z["qm"], Mq=z["Mq"], phi0=float(z["phi0"]), C_s=float(z["C_s"]),
                        k=z["k"], phik=z["phik"], Mk=z["Mk"])
    else:
        T = build_kernel_table(p)
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".%d.tmp.npz" % os.getpid()
        np.savez(tmp, qm=T.qm, Mq=T.Mq, phi0=T.phi0, C_s=T.C_s, k=T.k, phik=T.phik, Mk=T.Mk)
        os.replace(tmp, path)
    _TABLE_CACHE[key] = T
    return T


def phik_eval(T: KernelTable, kv):
    """phi_ab(|G|) by the natural cubic spline in k: (Nq, Nq) + kv.shape."""
    kv = np.asarray(kv, np.float64)
    dk = T.dk
    j = np.clip(np.floor(kv / dk).astype(np.int64), 0, T.k.size - 2)
    A = (T.k[j + 1] - kv) / dk
    B = 1.0 - A
    y0, y1 = T.phik[:, :, j], T.phik[:, :, j + 1]
    M0, M1 = T.Mk[:, :, j], T.Mk[:, :, j + 1]
    return A * y0 + B * y1 + ((A ** 3 - A) * M0 + (B ** 3 - B) * M1) * dk * dk / 6.0


# --------------------------------------------------------------------------
# Grid, reciprocal vectors, spectral gradient
# --------------------------------------------------------------------------


def check_cell(cell):
    cell = np.asarray(cell, np.float64)
    if cell.shape == (3,):
        return cell
    assert cell.shape == (3, 3) and np.allclose(cell, np.diag(np.diag(cell)))
    return np.diag(cell).copy()


def g_vectors(shape, L):
    """Cartesian G components broadcastable to shape (N3, N2, N1).

    G_d = 2 pi m_d / L_d with integer frequencies m_d in numpy's FFT order."""
    N3, N2, N1 = shape
    g1 = 2.0 * PI * np.fft.fftfreq(N1, d=1.0 / N1) / L[0]
    g2 = 2.0 * PI * np.fft.fftfreq(N2, d=1.0 / N2) / L[1]
    g3 = 2.0 * PI * np.fft.fftfreq(N3, d=1.0 / N3) / L[2]
    return g1[None, None, :], g2[None, :, None], g3[:, None, None]


def g_vectors_derivative(shape, L):
    """As g_vectors, with the Nyquist frequency of each even axis set to zero so
    that the spectral derivative is a real antisymmetric operator."""
    out = []
    for g, N in zip(g_vectors(shape, L), (shape[2], shape[1], shape[0])):
        g = g.copy()
        if N % 2 == 0:
            m = np.fft.fftfreq(N, d=1.0 / N)
            g.reshape(-1)[np.nonzero(m == -N // 2)[0]] = 0.0
        out.append(g)
    return out


def spectral_gradient(n, L):
    """grad n = IFFT(i G n(G)) with Nyquist components removed; shape (3,) + n.shape."""
    L = check_cell(L)
    nh = np.fft.fftn(n)
    G = g_vectors_derivative(n.shape, L)
    return np.stack([np.real(np.fft.ifftn(1j * g * nh)) for g in G])


def spectral_divergence(w, L):
    """sum_c D_c w_c with the same derivative operator as spectral_gradient."""
    L = check_cell(L)
    G = g_vectors_derivative(w.shape[1:], L)
    acc = np.zeros(w.shape[1:], dtype=np.complex128)
    for c in range(3):
        acc += 1j * G[c] * np.fft.fftn(w[c])
    return np.real(np.fft.ifftn(acc))


def stencil_gradient(n, L):
    """grad n by second-order central differences on the periodic grid, the
    finite-difference gradient the paper's implementation uses (text before
    Eq. Vi): (f(r + h_c e_c) - f(r - h_c e_c)) / (2 h_c)."""
    L = check_cell(L)
    N3, N2, N1 = n.shape
    h = (L[0] / N1, L[1] / N2, L[2] / N3)
    return np.stack([(np.roll(n, -1, axis=2) - np.roll(n, 1, axis=2)) / (2 * h[0]),
                     (np.roll(n, -1, axis=1) - np.roll(n, 1, axis=1)) / (2 * h[1]),
                     (np.roll(n, -1, axis=0) - np.roll(n, 1, axis=0)) / (2 * h[2])])


def stencil_divergence(w, L):
    """sum_c D_c w_c with the central-difference operator of stencil_gradient.
    That operator is antisymmetric, so the chain term of Eq. (Vi),
    sum_j w_j . dgrad_j/dn_i = (D^T w)_i, equals minus this divergence."""
    return sum(stencil_gradient(w[c], L)[c] for c in range(3))


# --------------------------------------------------------------------------
# Pointwise part: q, theta_a and their derivatives
# --------------------------------------------------------------------------


def pointwise(n, grad, T: KernelTable):
    """theta_a = n p_a(q), q = h(q0(n, |grad n|), q_c), and the derivatives the
    potential needs.  Points with n <= n_min (or n not finite) carry theta = 0
    and zero derivatives."""
    p = T.p
    n = np.asarray(n, np.float64)
    grad = np.asarray(grad, np.float64)
    ok = np.isfinite(n) & (n > p.n_min)
    ns = np.where(ok, n, 1.0)
    gmod = np.sqrt(np.sum(grad * grad, axis=0))
    gmod = np.where(ok, gmod, 0.0)
    q0, dq0_dn, dq0_dg = q0_unsaturated(ns, gmod)
    q, hp = saturate(q0, p.q_c, p.m_c)
    qcl = np.clip(q, T.qm[0], T.qm[-1])
    P, dP = cardinal_eval(T.qm, T.Mq, qcl)
    okf = ok.astype(np.float64)
    theta = ns * P * okf
    # q below the mesh is clamped to q_1: the clamped q does not vary there
    inside = (q >= T.qm[0]).astype(np.float64)
    dq_dn = hp * dq0_dn * inside
    dq_dg = hp * dq0_dg * inside  # (dq/d|g|)/|g|
    return dict(ok=ok, n=ns * okf, q=qcl, P=P * okf, dP=dP * okf, theta=theta,
                dq_dn=dq_dn * okf, dq_dg=dq_dg * okf)


# --------------------------------------------------------------------------
# Energy and potential (the hot path, stated plainly)
# --------------------------------------------------------------------------


def contract(theta_hat, Khat):
    """u_hat_a(G) = sum_b K_ab(G) theta_hat_b(G) and the energy sum
    sum_G sum_ab conj(theta_a) K_ab theta_b, for a per-G kernel Khat
    given as a callable(indices) -> (Nq, Nq, m) or an array (Nq, Nq, ...)."""
    Nq = theta_hat.shape[0]
    flat = theta_hat.reshape(Nq, -1)
    u = np.zeros_like(flat)
    esum = 0.0
    m = flat.shape[1]
    chunk = 32768
    for s in range(0, m, chunk):
        e = min(m, s + chunk)
        K = Khat(s, e)
        uc = np.einsum("abm,bm->am", K, flat[:, s:e])
        u[:, s:e] = uc
        esum += float(np.real(np.sum(np.conj(flat[:, s:e]) * uc)))
    return u.reshape(theta_hat.shape), esum


def energy_potential(n, grad, cell, T: KernelTable, kernel_hat=None, want_v=True, gradient="spectral"):
    """E_c^nl and v_nl on the periodic grid.

    Steps in the paper's order: theta_a = n p_a(q0) (after Eq. Eoffk);
    theta_a(G) by FFT; E = 1/2 Omega sum_G sum_ab theta_a(G)* phi_ab(|G|)
    theta_b(G) (Eq. Eoffk with the discrete normalisation below);
    u_a(r_i) = sum_G exp(i G r_i) sum_b phi_ab(|G|) theta_b(G) (Eqs. epsilon,
    epsofk); v_i from Eq. (Vi) with grad n_j = sum_i D_ji n_i the spectral
    derivative, whose transpose is -D; plus the Delta E correction of Eqs.
    (DEnl), (Depsnl) and its potential.

    Discrete conventions (reading): theta(G) = (1/N) sum_i theta_i
    exp(-i G.r_i), G = 2 pi m / L per axis, m in numpy's FFT order.

    gradient: "spectral" (grad n = D n with the spectral D) or "stencil"
    (grad n from central differences, stencil_gradient); v is the exact
    derivative of E under that operator.

    kernel_hat: optional callable (s, e) -> (Nq, Nq, e-s) replacing
    phi_ab(|G|) on the flattened G index range [s, e) (used by the identity
    tests with a grid-sampled kernel).

    Returns dict with E (= E_soft + dE), E_soft, dE, v, v_loc, w, u, theta.
    """
    L = check_cell(cell)
    p = T.p
    shape = n.shape
    N = n.size
    Omega = float(np.prod(L))
    dOmega = Omega / N
    pw = pointwise(n, grad, T)
    theta = pw["theta"]
    th_hat = np.fft.fftn(theta, axes=(1, 2, 3)) / N
    if kernel_hat is None:
        g1, g2, g3 = g_vectors(shape, L)
        gmod = np.sqrt(g1 * g1 + g2 * g2 + g3 * g3).ravel()

        def kernel_hat(s, e):
            return phik_eval(T, gmod[s:e])
    u_hat, esum = contract(th_hat, kernel_hat)
    E_soft = 0.5 * Omega * esum
    nn, q = pw["n"], pw["q"]
    dE_pt = np.where(pw["ok"], dOmega * T.C_s * nn * nn / (2.0 * q ** 3), 0.0)
    dE = float(np.sum(dE_pt))
    out = dict(E=E_soft + dE, E_soft=E_soft, dE=dE, theta=theta)
    if not want_v:
        return out
    u = np.real(np.fft.ifftn(u_hat, axes=(1, 2, 3))) * N
    P, dP = pw["P"], pw["dP"]
    # d theta_a/dn = p_a + n p_a' dq/dn ; d theta_a/d grad = n p_a' (dq/d|g|)/|g| grad
    S0 = np.sum(u * P, axis=0)
    S1 = np.sum(u * dP, axis=0)
    q4 = np.where(pw["ok"], q ** 4, 1.0)
    # Delta E per point: dOmega C_s n^2/(2 q^3); its derivatives / dOmega
    dE_n = T.C_s * (nn / q ** 3 - 1.5 * nn * nn / q4 * pw["dq_dn"])
    dE_g = -1.5 * T.C_s * nn * nn / q4 * pw["dq_dg"]
    v_loc = S0 + nn * S1 * pw["dq_dn"] + dE_n
    v_loc = np.where(pw["ok"], v_loc, 0.0)
    g = nn * S1 * pw["dq_dg"] + dE_g
    w = np.where(pw["ok"], g, 0.0)[None] * np.asarray(grad, np.float64)
    # the chain term of Eq. (Vi) under the gradient operator the caller used
    div = stencil_divergence(w, L) if gradient == "stencil" else spectral_divergence(w, L)
    v = v_loc - div
    out.update(v=v, v_loc=v_loc, w=w, u=u)
    return out


def energy(n, grad, cell, T, **kw):
    return energy_potential(n, grad, cell, T, want_v=False, **kw)["E"]


# --------------------------------------------------------------------------
# Brute-force references used by the pins
# --------------------------------------------------------------------------


def min_image_distances(shape, L):
    """|r_i - r_j| under the minimum-image convention for every grid displacement
    (shape (N3, N2, N1), indexed by the displacement)."""
    N3, N2, N1 = shape
    out = []
    for N, Ld in ((N1, L[0]), (N2, L[1]), (N3, L[2])):
        m = np.arange(N)
        m = np.where(m > N // 2, m - N, m)
        out.append(m * Ld / N)
    x, y, z = out
    return np.sqrt(x[None, None, :] ** 2 + y[None, :, None] ** 2 + z[:, None, None] ** 2)


def factored_bruteforce_energy(theta, K, dOmega):
    """Eq. (Eofni): 1/2 dOmega^2 sum_ab sum_ij theta_ai theta_bj K_ab(r_i - r_j),
    K a periodic grid kernel indexed by displacement, (Nq, Nq, N3, N2, N1).
    Explicit loop over i, vectorised over j (small grids only)."""
    Nq = theta.shape[0]
    shape = theta.shape[1:]
    N3, N2, N1 = shape
    tot = 0.0
    for i3 in range(N3):
        for i2 in range(N2):
            for i1 in range(N1):
                # displacement index (i - j) mod N for all j
                Kd = np.roll(np.roll(np.roll(K[:, :, ::-1, ::-1, ::-1], i3 + 1, axis=2), i2 + 1, axis=3),
                             i1 + 1, axis=4)
                tot += float(np.einsum("a,abj,bj->", theta[:, i3, i2, i1],
                                       Kd.reshape(Nq, Nq, -1), theta.reshape(Nq, -1)))
    return 0.5 * dOmega * dOmega * tot


def unfactored_bruteforce_energy(n, grad, cell, T: KernelTable):
    """Eq. (Enl) on the grid without the factorisation of Eq. (phi):
    1/2 dOmega^2 sum_ij n_i n_j phi_s(q_i r_ij, q_j r_ij), minimum image.
    Tiny grids only: one kernel evaluation per pair of points."""
    L = check_cell(cell)
    pw = pointwise(n, grad, T)
    nn = pw["n"].ravel()
    q = pw["q"].ravel()
    N = nn.size
    dOmega = float(np.prod(L)) / N
    R = min_image_distances(n.shape, L)
    idx = np.array(np.unravel_index(np.arange(N), n.shape)).T
    i_list, j_list, r_list = [], [], []
    for i in range(N):
        dd = (idx[i][None, :] - idx) % np.array(n.shape)
        r = R[dd[:, 0], dd[:, 1], dd[:, 2]]
        i_list.append(np.full(N, i))
        j_list.append(np.arange(N))
        r_list.append(r)
    ii = np.concatenate(i_list)
    jj = np.concatenate(j_list)
    rr = np.concatenate(r_list)
    vals = phi_soft_points(q[ii] * rr, q[jj] * rr, T.p, T.phi0)
    return 0.5 * dOmega * dOmega * float(np.sum(nn[ii] * nn[jj] * vals))


def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def direct_interaction_energy(nA, gA, nB, gB, cell, T: KernelTable, n_cut=1e-8, images=1):
    """Interaction of two separated fragments by Eq. (Enl) evaluated directly on
    the grid, without the factorisation: dOmega^2 sum_{i in A} sum_{j in B}
    n_i n_j phi(q_i r_ij, q_j r_ij), each q from that fragment's own density,
    summed over periodic images of B (|m_d| <= images).  Points with
    n <= n_cut are dropped.  Valid while no pair comes within the soft radius."""
    L = check_cell(cell)
    shape = nA.shape
    N = nA.size
    dOmega = float(np.prod(L)) / N
    pa = pointwise(nA, gA, T)
    pb = pointwise(nB, gB, T)
    N3, N2, N1 = shape
    z, y, x = np.meshgrid(np.arange(N3) * L[2] / N3, np.arange(N2) * L[1] / N2,
                          np.arange(N1) * L[0] / N1, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    ia = np.nonzero(nA.ravel() > n_cut)[0]
    ib = np.nonzero(nB.ravel() > n_cut)[0]
    tot = 0.0
    rng = range(-images, images + 1)
    for m1 in rng:
        for m2 in rng:
            for m3 in rng:
                shift = np.array([m1 * L[0], m2 * L[1], m3 * L[2]])
                for s in range(0, ia.size, 512):
                    ii = ia[s:s + 512]
                    r = np.linalg.norm(pos[ii][:, None, :] - pos[ib][None, :, :] - shift, axis=2)
                    d1 = pa["q"].ravel()[ii][:, None] * r
                    d2 = pb["q"].ravel()[ib][None, :] * r
                    ph = phi_kernel(d1, d2, T.p)
                    tot += float(np.sum(pa["n"].ravel()[ii][:, None] * pb["n"].ravel()[ib][None, :] * ph))
    return dOmega * dOmega * tot
