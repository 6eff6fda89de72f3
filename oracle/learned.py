"""FP64 oracle of the learned reduced basis (no counterpart in the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper evaluates E_c^nl with Nq cardinal-spline channels theta_a = n p_a(q)
and a radial kernel table phi_ab(k) (Eqs. Eoffk, Vi).  The learned reduced
basis keeps that structure with fewer channels whose weights come from a
small network instead of the splines:

  features   f1 = ln n,  s2 = |grad n|^2 n^(-8/3),  f2 = 1/2 ln(s2 + eps^2)
             x = ((f1 - mu1)/sig1, (f2 - mu2)/sig2)
             (a smooth form of ln(|grad n|/n^(4/3)); s2 keeps the map
             differentiable at grad n = 0)
  network    z1 = W1 x + b1, h1 = bf16(silu(z1))
             z2 = W2 h1 + b2, h2 = bf16(silu(z2))
             w  = W3 h2 + b3                         (M outputs)
             weights W1, W2, W3 take bf16 values; biases and sums are wider
  base       optional: w_m = p_m(q) + (network output m), with p_m the
             cardinal cubic splines (Eq. fofx) on an M-point logarithmic
             mesh (q_1, lambda, q_c) and q = h(q0) of Eq. (Sat) clamped to
             that mesh (its derivative is zero where the clamp acts); the
             network then learns a correction to the plain method's basis
  channels   theta_m = n w_m (zero where n <= n_min or n is not finite)
  kernel     K_mn(k) on J uniform knots k_j = j dk, interpolated by
             Catmull-Rom cubics (value at k in [k_j, k_j+1] from the knots
             j-1 .. j+2; K is even in k, so K_-1 = K_1, and the knot past
             the last is the linear extrapolation 2 K_J-1 - K_J-2);
             symmetric, stored as the M(M+1)/2 pairs m <= n (row-major)
  energy     E = 1/2 Omega sum_G sum_mn theta_m(G)* K_mn(|G|) theta_n(G)
                 + Delta E   (the paper's local softening correction, Eqs.
                 DEnl/Depsnl, unchanged: it does not depend on the network)
  potential  v = dE/dn_i / dOmega with grad n = D n (spectral D), assembled
             as in Eq. (Vi): v = v_loc - D.w.

Flat parameter vector (the order the CUDA library uses too):
  W1 [H][2], b1 [H], W2 [H][H], b2 [H], W3 [M][H], b3 [M], K [P][J]
with H = 64 hidden units and P = M(M+1)/2 pairs.

Precision mirrored from the CUDA path: weights and the two hidden activations
are rounded to bf16 (round to nearest, ties to even) before they enter a
product, exactly where the tensor-core operands are bf16.  The potential
needs the network's Jacobian dw/dx, formed by forward mode beside the
forward pass; its tangents are rounded to bf16 where they enter a
tensor-core product unless ``jac_bf16=False``, which gives the exact
derivative of the model (used by the finite-difference pins).
Parameter gradients are exact derivatives of the mirrored forward, treating
each rounding as the identity (straight-through).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import vdw_oracle as V

H = 64


def bf16_round(x):
    """Round to the nearest bfloat16 value (8 significant bits), ties to even.

    Works on the binary significand directly: x = m 2^e with m in [0.5, 1),
    so m 2^8 rounded to an integer (np.rint rounds half to even) keeps 8 bits.
    Normal range only (|x| between 2^-126 and 2^127), which covers every value
    the model produces; zero stays zero."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_prime(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


@dataclass
class LearnedModel:
    """Parameters of the learned basis (FP64 copies of the trained values)."""

    M: int
    W1: np.ndarray  # (H, 2)
    b1: np.ndarray  # (H,)
    W2: np.ndarray  # (H, H)
    b2: np.ndarray  # (H,)
    W3: np.ndarray  # (M, H)
    b3: np.ndarray  # (M,)
    K: np.ndarray   # (P, J) knot values of the pair kernels
    dk: float       # knot spacing (bohr^-1)
    mu1: float
    sig1: float
    mu2: float
    sig2: float
    eps: float      # s2 regulariser (same units as |grad n| / n^(4/3))
    base_q1: float = 0.0    # base mesh (0: no base)
    base_lam: float = 0.0

    @property
    def P(self):
        return self.M * (self.M + 1) // 2

    @property
    def J(self):
        return self.K.shape[1]

    def flat(self):
        return np.concatenate([a.ravel() for a in (self.W1, self.b1, self.W2, self.b2, self.W3, self.b3, self.K)])

    @staticmethod
    def sizes(M, J):
        P = M * (M + 1) // 2
        return [(H, 2), (H,), (H, H), (H,), (M, H), (M,), (P, J)]

    def with_flat(self, v):
        v = np.asarray(v, np.float64)
        out, o = [], 0
        for s in self.sizes(self.M, self.J):
            k = int(np.prod(s))
            out.append(v[o:o + k].reshape(s).copy())
            o += k
        assert o == v.size
        return LearnedModel(self.M, *out, dk=self.dk, mu1=self.mu1, sig1=self.sig1, mu2=self.mu2,
                            sig2=self.sig2, eps=self.eps, base_q1=self.base_q1, base_lam=self.base_lam)


def pair_index(M):
    """(m, n) for every pair p, m <= n, row-major."""
    return [(m, n) for m in range(M) for n in range(m, M)]


def random_model(seed, M=8, J=256, k_max=30.0, mu=(-4.0, 1.0), sig=(3.0, 2.0), eps=0.1, kscale=1.0, base=(0.0, 0.0)):
    """Seeded model with He-style weights and smooth random pair kernels;
    base = (q_1, lambda) of an optional spline base mesh."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, np.sqrt(2.0 / 2), (H, 2))
    W2 = rng.normal(0.0, np.sqrt(2.0 / H), (H, H))
    W3 = rng.normal(0.0, np.sqrt(1.0 / H), (M, H))
    b1 = rng.normal(0.0, 0.1, H)
    b2 = rng.normal(0.0, 0.1, H)
    b3 = rng.normal(0.0, 0.1, M) + 1.0 / M
    dk = k_max / (J - 1)
    k = np.arange(J) * dk
    P = M * (M + 1) // 2
    K = np.zeros((P, J))
    for p in range(P):
        a, w = rng.uniform(-1.0, 1.0), rng.uniform(0.5, 3.0)
        K[p] = kscale * a * np.exp(-(k / w) ** 2)
    return LearnedModel(M, W1, b1, W2, b2, W3, b3, K, dk, mu[0], sig[0], mu[1], sig[1], eps, base[0], base[1])


# --------------------------------------------------------------------------
# pointwise part
# --------------------------------------------------------------------------


def features(n, grad, mdl: LearnedModel, n_min):
    """x1, x2 and their derivatives: dx1/dn, dx2/dn and dx2/dgrad_c = gx2 grad_c."""
    n = np.asarray(n, np.float64)
    ok = np.isfinite(n) & (n > n_min)
    ns = np.where(ok, n, 1.0)
    g2 = np.sum(np.asarray(grad, np.float64) ** 2, axis=0)
    s2 = g2 * ns ** (-8.0 / 3.0)
    den = s2 + mdl.eps ** 2
    x1 = (np.log(ns) - mdl.mu1) / mdl.sig1
    x2 = (0.5 * np.log(den) - mdl.mu2) / mdl.sig2
    dx1_dn = 1.0 / (mdl.sig1 * ns)
    dx2_dn = -(4.0 / 3.0) * s2 / (ns * den * mdl.sig2)
    gx2 = ns ** (-8.0 / 3.0) / (den * mdl.sig2)
    return dict(ok=ok, n=np.where(ok, ns, 0.0), x1=x1, x2=x2, dx1_dn=dx1_dn, dx2_dn=dx2_dn, gx2=gx2)


def base_basis(n, grad, mdl: LearnedModel, T: V.KernelTable):
    """p_m(q), dp_m/dq on the base mesh and dq/dn, (dq/d|grad n|)/|grad n| with
    the clamp's zero derivative; zeros everywhere when the model has no base."""
    shape = np.shape(n)
    if not mdl.base_q1 > 0:
        z = np.zeros((mdl.M,) + shape)
        return z, z.copy(), np.zeros(shape), np.zeros(shape)
    p = T.p
    qb = V.q_mesh(V.Params(Nq=mdl.M, q_1=mdl.base_q1, lam=mdl.base_lam, q_c=p.q_c))
    Mb = V.cardinal_M(qb)
    n = np.asarray(n, np.float64)
    ok = np.isfinite(n) & (n > p.n_min)
    ns = np.where(ok, n, 1.0)
    gmod = np.where(ok, np.sqrt(np.sum(np.asarray(grad, np.float64) ** 2, axis=0)), 0.0)
    q0, dq0_dn, dq0_dg = V.q0_unsaturated(ns, gmod)
    q, hp = V.saturate(q0, p.q_c, p.m_c)
    inside = (q >= qb[0]) & (q <= qb[-1])
    P, dP = V.cardinal_eval(qb, Mb, np.clip(q, qb[0], qb[-1]))
    okf = ok.astype(np.float64)
    return P * okf, dP * okf, hp * dq0_dn * inside * okf, hp * dq0_dg * inside * okf


def mlp_forward(x1, x2, mdl: LearnedModel):
    """Network outputs w (M, m) and the intermediate values, for points given as
    flat arrays x1, x2 of length m."""
    W1, W2, W3 = bf16_round(mdl.W1), bf16_round(mdl.W2), bf16_round(mdl.W3)
    X = np.stack([x1, x2])                       # (2, m)
    z1 = W1 @ X + mdl.b1[:, None]                # (H, m)
    h1 = bf16_round(silu(z1))
    z2 = W2 @ h1 + mdl.b2[:, None]
    h2 = bf16_round(silu(z2))
    w = W3 @ h2 + mdl.b3[:, None]                # (M, m)
    return dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, w=w, W1=W1, W2=W2, W3=W3)


def mlp_jacobian(f, jac_bf16=True):
    """J[m, j, point] = d w_m / d x_j by forward mode: tangents
    dz1_j = W1[:, j], dh1_j = silu'(z1) dz1_j, dz2_j = W2 dh1_j,
    dh2_j = silu'(z2) dz2_j, dw_j = W3 dh2_j.  With jac_bf16 the tangents that
    enter a tensor-core product (dh1_j, dh2_j) are rounded to bf16 as the CUDA
    path does; the activations' own bf16 rounding counts as the identity."""
    r = bf16_round if jac_bf16 else (lambda a: a)
    s1 = silu_prime(f["z1"])
    s2 = silu_prime(f["z2"])
    out = []
    for j in range(2):
        dh1 = r(s1 * f["W1"][:, j][:, None])
        dh2 = r(s2 * (f["W2"] @ dh1))
        out.append(f["W3"] @ dh2)
    return np.stack(out, axis=1)  # (M, 2, m)


# --------------------------------------------------------------------------
# the network tabulated on a node grid of the two features
# --------------------------------------------------------------------------
# The network's output depends on the point only through (x1, x2).  The
# tabulated form evaluates it once on the nodes x = -D + (i - 1) h, i = 0 ..
# T + 1, h = 2 D / (T - 1) (T nodes on [-D, D] and one padding node on each
# side), and a point's outputs are the tensor product of Catmull-Rom cubics
# in x1 and x2 through the 4 x 4 nodes around it.  That interpolant is C1 and
# reproduces quadratics; its x derivatives are the Jacobian the potential
# uses, so v stays the exact derivative of the tabulated E.  Features outside
# [-D, D] are clamped to it (zero derivative along a clamped axis).


@dataclass
class NetworkTable:
    T: int
    D: float
    vals: np.ndarray  # (M, T + 2, T + 2): vals[m, i1, i2] at (x1, x2) node (i1, i2)

    @property
    def h(self):
        return 2.0 * self.D / (self.T - 1)

    def nodes(self):
        return -self.D + (np.arange(self.T + 2) - 1.0) * self.h


def network_table(mdl: LearnedModel, T, D):
    """The network (mlp_forward, bf16 roundings mirrored) on the (T+2)^2 nodes."""
    xs = -D + (np.arange(T + 2) - 1.0) * (2.0 * D / (T - 1))
    X1, X2 = np.meshgrid(xs, xs, indexing="ij")
    w = mlp_forward(X1.ravel(), X2.ravel(), mdl)["w"]
    return NetworkTable(T=T, D=float(D), vals=w.reshape(mdl.M, T + 2, T + 2))


def catmull_rom(s):
    """Weights of the nodes i-1, i, i+1, i+2 at local position s in [0, 1] of
    interval i, and their s derivatives: arrays (4,) + s.shape."""
    s = np.asarray(s, np.float64)
    w = np.stack([0.5 * (-s ** 3 + 2 * s ** 2 - s), 0.5 * (3 * s ** 3 - 5 * s ** 2 + 2),
                  0.5 * (-3 * s ** 3 + 4 * s ** 2 + s), 0.5 * (s ** 3 - s ** 2)])
    dw = np.stack([0.5 * (-3 * s ** 2 + 4 * s - 1), 0.5 * (9 * s ** 2 - 10 * s),
                   0.5 * (-9 * s ** 2 + 8 * s + 1), 0.5 * (3 * s ** 2 - 2 * s)])
    return w, dw


def table_eval(tab: NetworkTable, x1, x2):
    """Outputs o (M, m) and Jacobian J (M, 2, m) at flat feature arrays."""
    x1 = np.asarray(x1, np.float64)
    x2 = np.asarray(x2, np.float64)
    h = tab.h
    out_c = []
    for x in (x1, x2):
        xc = np.clip(x, -tab.D, tab.D)
        u = (xc + tab.D) / h                      # node index of the interval start, in [0, T-1]
        i = np.minimum(np.floor(u).astype(np.int64), tab.T - 2)
        s = u - i
        w, dw = catmull_rom(s)
        inside = (x >= -tab.D) & (x <= tab.D)
        out_c.append((i, w, dw * (inside / h)[None]))
    (i1, a, da), (i2, b, db) = out_c
    M = tab.vals.shape[0]
    o = np.zeros((M, x1.size))
    j1 = np.zeros((M, x1.size))
    j2 = np.zeros((M, x1.size))
    for k in range(4):
        for l in range(4):
            v = tab.vals[:, i1 + k, i2 + l]       # padded index: interval i starts at node i + 1
            o += a[k] * b[l] * v
            j1 += da[k] * b[l] * v
            j2 += a[k] * db[l] * v
    return o, np.stack([j1, j2], axis=1)


# --------------------------------------------------------------------------
# learned kernel
# --------------------------------------------------------------------------


def knot_weights(kmod, dk, J):
    """Catmull-Rom interpolation on knots j dk: for each k the four knot
    indices (j-1 .. j+2, j the interval clamped to the last one) and weights,
    with the index -1 folded onto knot 1 (K even in k) and the index J
    expressed through knots J-1 and J-2 (linear extrapolation).  Returns
    (idx, wts), each of shape (6, m): some entries carry zero weight."""
    s = np.asarray(kmod, np.float64) / dk
    j = np.minimum(np.floor(s).astype(np.int64), J - 2)
    t = s - j
    w = [(-t ** 3 + 2 * t ** 2 - t) / 2, (3 * t ** 3 - 5 * t ** 2 + 2) / 2,
         (-3 * t ** 3 + 4 * t ** 2 + t) / 2, (t ** 3 - t ** 2) / 2]
    idx, wts = [], []
    for i, wi in zip(range(-1, 3), w):
        k = j + i
        lo = k < 0
        hi = k > J - 1
        idx.append(np.where(lo, 1, np.where(hi, J - 1, k)))
        wts.append(np.where(hi, 2.0 * wi, wi))
        idx.append(np.where(hi, J - 2, 0))
        wts.append(np.where(hi, -wi, 0.0))
    idx = np.array(idx)
    wts = np.array(wts)
    keep = np.array([0, 2, 4, 6, 7, 1])  # the six slots: 4 knots + the extrapolation's second term
    return idx[keep], wts[keep]


def kernel_eval(mdl: LearnedModel, kmod):
    """K_mn(|G|) for flat |G| values: array (M, M, m)."""
    idx, wts = knot_weights(kmod, mdl.dk, mdl.J)
    vals = np.zeros((mdl.P, idx.shape[1]))
    for r in range(idx.shape[0]):
        vals += wts[r][None, :] * mdl.K[:, idx[r]]
    out = np.empty((mdl.M, mdl.M, vals.shape[1]))
    for p, (m, n) in enumerate(pair_index(mdl.M)):
        out[m, n] = vals[p]
        out[n, m] = vals[p]
    return out


# --------------------------------------------------------------------------
# energy, potential, parameter gradients
# --------------------------------------------------------------------------


def energy_potential(n, grad, cell, mdl: LearnedModel, T: V.KernelTable, want_v=True, jac_bf16=True,
                     want_grad=False, table: NetworkTable | None = None):
    """E (= E_soft + Delta E), and optionally v and dE/dparams of the learned
    basis on the periodic grid (conventions of the plain oracle: theta(G) =
    (1/N) sum_i theta_i exp(-i G.r_i)).  T supplies the plain method's Delta E
    (C_s and q0 with its saturation).  With a network table the outputs and
    their Jacobian come from its interpolation (table_eval) instead of the
    network at each point."""
    L = V.check_cell(cell)
    shape = n.shape
    N = n.size
    Omega = float(np.prod(L))
    dOmega = Omega / N
    ft = features(n, grad, mdl, T.p.n_min)
    ok = ft["ok"]
    nn = ft["n"]
    if table is None:
        f = mlp_forward(ft["x1"].ravel(), ft["x2"].ravel(), mdl)
        o = f["w"]
    else:
        assert not want_grad, "parameter gradients are those of the network itself"
        o, Jt = table_eval(table, ft["x1"].ravel(), ft["x2"].ravel())
    Pb, dPb, dq_dn_b, dq_dg_b = base_basis(n, grad, mdl, T)
    w = (o.reshape((mdl.M,) + shape) + Pb) * ok[None]
    theta = nn[None] * w
    th_hat = np.fft.fftn(theta, axes=(1, 2, 3)) / N
    g1, g2, g3 = V.g_vectors(shape, L)
    kmod = np.sqrt(g1 * g1 + g2 * g2 + g3 * g3).ravel()
    u_hat, esum = V.contract(th_hat, lambda s, e: kernel_eval(mdl, kmod[s:e]))
    E_soft = 0.5 * Omega * esum
    pw = V.pointwise(n, grad, T)
    q = pw["q"]
    dE_pt = np.where(pw["ok"], dOmega * T.C_s * pw["n"] ** 2 / (2.0 * q ** 3), 0.0)
    dE = float(np.sum(dE_pt))
    out = dict(E=E_soft + dE, E_soft=E_soft, dE=dE, theta=theta, w_ch=w)
    if not (want_v or want_grad):
        return out
    u = np.real(np.fft.ifftn(u_hat, axes=(1, 2, 3))) * N
    out["u"] = u
    if want_v:
        Jm = mlp_jacobian(f, jac_bf16) if table is None else Jt
        c = np.einsum("mjp,mp->jp", Jm, u.reshape(mdl.M, -1)).reshape((2,) + shape)
        S0 = np.sum(u * w, axis=0)
        q4 = np.where(pw["ok"], q ** 4, 1.0)
        dE_n = T.C_s * (pw["n"] / q ** 3 - 1.5 * pw["n"] ** 2 / q4 * pw["dq_dn"])
        dE_g = -1.5 * T.C_s * pw["n"] ** 2 / q4 * pw["dq_dg"]
        S1b = np.sum(u * dPb, axis=0)
        v_loc = S0 + nn * (c[0] * ft["dx1_dn"] + c[1] * ft["dx2_dn"] + S1b * dq_dn_b) + dE_n
        v_loc = np.where(ok, v_loc, 0.0)
        gg = np.where(ok, nn * (c[1] * ft["gx2"] + S1b * dq_dg_b) + dE_g, 0.0)
        wv = gg[None] * np.asarray(grad, np.float64)
        out.update(v=v_loc - V.spectral_divergence(wv, L), v_loc=v_loc, w=wv)
    if want_grad:
        out["grad"] = param_grad(f, th_hat, kmod, u, nn, ok, mdl, Omega, dOmega)
    return out


def param_grad(f, th_hat, kmod, u, nn, ok, mdl: LearnedModel, Omega, dOmega):
    """dE/dparams (flat, in the library's order) by backpropagation."""
    M = mdl.M
    # kernel knots: dE/dK_p[j] = 1/2 Omega sum_G w_j(|G|) (2 - delta_mn) Re(conj th_m th_n)
    idx, wts = knot_weights(kmod, mdl.dk, mdl.J)
    th = th_hat.reshape(M, -1)
    gK = np.zeros_like(mdl.K)
    for p, (m, n) in enumerate(pair_index(M)):
        r = np.real(np.conj(th[m]) * th[n]) * (1.0 if m == n else 2.0) * 0.5 * Omega
        for q in range(idx.shape[0]):
            gK[p] += np.bincount(idx[q], weights=wts[q] * r, minlength=mdl.J)
    # network: cotangent of the outputs w_m at each point is dOmega n u_m
    do = (dOmega * nn * ok)[None] * u
    do = do.reshape(M, -1)
    gb3 = do.sum(axis=1)
    gW3 = do @ f["h2"].T
    dz2 = (f["W3"].T @ do) * silu_prime(f["z2"])
    gb2 = dz2.sum(axis=1)
    gW2 = dz2 @ f["h1"].T
    dz1 = (f["W2"].T @ dz2) * silu_prime(f["z1"])
    gb1 = dz1.sum(axis=1)
    gW1 = dz1 @ f["X"].T
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, gK.ravel()])


def energy(n, grad, cell, mdl, T):
    return energy_potential(n, grad, cell, mdl, T, want_v=False)["E"]


def energy_grad(n, grad, cell, mdl, T):
    return energy_potential(n, grad, cell, mdl, T, want_v=False, want_grad=True)["grad"]


# --------------------------------------------------------------------------
# training loss
# --------------------------------------------------------------------------


def loss(n, cell, mdl, T, E_ref, v_ref, natoms, a=1.0, b=1.0, jac_bf16=False):
    """L = a ((E - E_ref)/natoms)^2 + b sum_i n_i (v_i - v_ref_i)^2 / sum_i n_i,
    with grad n = D n (spectral)."""
    L_ = V.check_cell(cell)
    grad = V.spectral_gradient(n, L_)
    r = energy_potential(n, grad, L_, mdl, T, want_v=True, jac_bf16=jac_bf16)
    dv = r["v"] - v_ref
    return a * ((r["E"] - E_ref) / natoms) ** 2 + b * float(np.sum(n * dv * dv) / np.sum(n)), r


def loss_grad(n, cell, mdl, T, E_ref, v_ref, natoms, a=1.0, b=1.0, rel_step=1e-3):
    """dL/dparams.  The energy term is 2a (E - E_ref)/natoms^2 dE/dp.  The
    potential term needs sum_i lam_i dv_i/dp with lam_i = n_i (v_i - v_ref_i):
    since v_i = dE/dn_i / dOmega with grad n = D n, that sum equals
    (1/dOmega) d/de [dE/dp (n + e lam)] at e = 0, evaluated here by central
    differences with one Richardson step (error O(e^4)); the step makes the
    largest relative change of n equal to rel_step."""
    L_ = V.check_cell(cell)
    N = n.size
    dOmega = float(np.prod(L_)) / N
    grad = V.spectral_gradient(n, L_)
    r = energy_potential(n, grad, L_, mdl, T, want_v=True, jac_bf16=False, want_grad=True)
    lam = n * (r["v"] - v_ref)
    rel = np.max(np.abs(lam / n))
    eps = rel_step / rel if rel > 0 else 0.0

    def gE(e):
        m = n + e * lam
        return energy_grad(m, V.spectral_gradient(m, L_), L_, mdl, T)

    if eps > 0:
        d1 = (gE(eps) - gE(-eps)) / (2 * eps)
        d2 = (gE(eps / 2) - gE(-eps / 2)) / eps
        dd = (4.0 * d2 - d1) / 3.0
    else:
        dd = np.zeros_like(r["grad"])
    g = 2.0 * a * (r["E"] - E_ref) / natoms ** 2 * r["grad"] + (2.0 * b / np.sum(n)) * dd / dOmega
    return g


def fit_grad(n, grad, mdl: LearnedModel, target, weight, n_min):
    """d/dparams of sum_i weight_i sum_m (w_m(x_i) - target_m,i)^2 over the
    points with n > n_min (network part of the flat vector; knots get zero)."""
    ft = features(n, grad, mdl, n_min)
    ok = ft["ok"].ravel()
    f = mlp_forward(ft["x1"].ravel(), ft["x2"].ravel(), mdl)
    M = mdl.M
    do = 2.0 * (np.asarray(weight, np.float64).ravel() * ok)[None] * (f["w"] - np.asarray(target).reshape(M, -1))
    gb3 = do.sum(axis=1)
    gW3 = do @ f["h2"].T
    dz2 = (f["W3"].T @ do) * silu_prime(f["z2"])
    gb2 = dz2.sum(axis=1)
    gW2 = dz2 @ f["h1"].T
    dz1 = (f["W2"].T @ dz2) * silu_prime(f["z1"])
    gb1 = dz1.sum(axis=1)
    gW1 = dz1 @ f["X"].T
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, np.zeros(mdl.K.size)])
