/*
 * vdwnl: the nonlocal van der Waals correlation energy E_c^nl and potential
 * v_nl of Dion et al. on a periodic real-space grid, evaluated with the
 * kernel factorisation and FFT method of Roman-Perez and Soler
 * (arXiv:0812.0244), on one NVIDIA GB300 (sm_103a).
 *
 * The boundary follows the paper's statement that the implementation accepts
 * n(r_i) on a uniform real-space grid and returns the energy and the
 * potential on the same grid (text after Eq. epsofk).  Every entry point
 * returns VDW_OK (0) or a negative error code; no C++ exception crosses it.
 *
 * Conventions shared by all entry points
 *   - Grid N1 x N2 x N3 (x = axis 1 fastest): flat index i = i1 + N1 (i2 + N2 i3),
 *     N = N1 N2 N3.  The cell is orthorhombic with edge lengths L[3] (bohr).
 *     r_i = (i1 L1/N1, i2 L2/N2, i3 L3/N3).
 *   - All densities and potentials are in atomic units (bohr, Hartree).
 *   - "device" pointers are CUDA device (or managed) memory, FP32 unless noted,
 *     caller-owned.  "host" pointers are ordinary (preferably pinned) memory.
 *   - stream is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls taking a stream only enqueue work on it and return,
 *     except where a host read-back is documented.
 *   - Fourier convention: theta(G) = (1/N) sum_i theta_i exp(-i G.r_i),
 *     G = 2 pi (m1/L1, m2/L2, m3/L3).
 */
#ifndef VDWNL_H
#define VDWNL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define VDW_OK 0
#define VDW_ERR_ARG (-1)     /* null pointer, non-positive size, bad parameter */
#define VDW_ERR_SIZE (-2)    /* grid not {2,3,5}-smooth, odd N1 or N3, too large
                                for on-chip staging, or |G|max > k_max         */
#define VDW_ERR_CUDA (-3)    /* a CUDA runtime call failed                      */
#define VDW_ERR_OOM (-4)     /* device allocation failed                         */
#define VDW_ERR_STATE (-5)   /* call made before vdw_plan                        */
#define VDW_ERR_UNSUPPORTED (-6) /* Nq not compiled in; non-orthorhombic cell     */
#define VDW_ERR_TIMEOUT (-7) /* a kernel of an earlier call gave up a bounded
                                wait (see vdw_wait_status); that call's
                                results may be wrong                        */

/* ---- method parameters --------------------------------------------------
 * Nq, q_c, m_c   interpolation mesh size (paper: "N_alpha ~ 20"), saturation
 *                cutoff and order of Eq. (Sat) ("m_c ~ 12 and q_c ~ 5 a.u.");
 *                m_c <= 32.
 * q_1, lambda    first point and ratio of the logarithmic mesh
 *                (q_{a+1}-q_a) = lambda (q_a - q_{a-1}), q_Nq = q_c.
 * d_s            radius of the soft kernel of Eq. (PhiSoft) in
 *                d = sqrt(d1^2 + d2^2); phi0 is set so that phi4 = 0 on the
 *                diagonal ray d1 = d2.
 * na, a_max      Gauss-Legendre nodes in t = atan(a), t in [0, atan(a_max)],
 *                for the Dion et al. double integral defining phi(d1, d2).
 * d_asym         phi takes its closed-form large-separation limit
 *                -12 (4 pi/9)^3 / (d1^2 d2^2 (d1^2 + d2^2)) when
 *                min(d1, d2) >= d_asym.
 * r_c, Nr        radial transform of phi_ab(r) cut at r_c, Simpson's rule on
 *                Nr (even) intervals.
 * k_max, Nk      uniform k mesh of the radial table, natural cubic spline in k.
 * n_cs           Gauss-Legendre nodes for the softening constant C_s of
 *                Eq. (Depsnl).
 * n_min          points with n <= n_min (or n not finite) carry theta = 0.   */
typedef struct vdw_params {
    int Nq;
    double q_1, q_c, lambda;
    int m_c;
    double d_s;
    int na;
    double a_max, d_asym;
    double r_c;
    int Nr;
    double k_max;
    int Nk;
    int n_cs;
    double n_min;
} vdw_params;

/* Fill p with the defaults: Nq 20, q_1 1e-5, q_c 5, lambda 1.2, m_c 12,
 * d_s 1, na 256, a_max 64, d_asym 8, r_c 100, Nr 4096, k_max 40, Nk 1024,
 * n_cs 64, n_min 1e-12. */
int vdw_params_default(vdw_params* p);

/* ---- kernel table (init, FP64 on the GPU) -------------------------------
 * The radial Fourier transform of the factorised kernel
 *   phi_ab(k) = 4 pi Int_0^{r_c} r^2 phi_s(q_a r, q_b r) j0(k r) dr
 * (the paper: phi_ab(k) "can be calculated in spherical coordinates, and
 * stored in a radial mesh of points k", text after Eq. Eoffk), the soft
 * kernel of Eq. (PhiSoft), and the softening constant
 *   C_s = Int_0^{d_s/sqrt2} 4 pi x^2 [phi(x,x) - phi_s(x,x)] dx
 * of Eq. (Depsnl), all computed in FP64 by kernels on the current device.
 * Outputs (host, caller-owned, any may be NULL): q_mesh[Nq];
 * phi_k[Nq*Nq*Nk] with phi_k[(a*Nq + b)*Nk + m] = phi_ab(m k_max/(Nk-1));
 * phi0; C_s.  Synchronous. */
int vdw_kernel_table(const vdw_params* p, double* q_mesh, double* phi_k,
                     double* phi0, double* C_s);

/* ---- context ------------------------------------------------------------ */
typedef struct vdw_ctx* vdw_handle;

/* Create a context on the current device.  If phi_k (host, FP64, layout as
 * in vdw_kernel_table) is NULL the table is generated on the GPU by
 * vdw_kernel_table and C_s is ignored; otherwise phi_k and C_s are used as
 * given.  The context owns its tables and (after vdw_plan) its workspace.
 * Synchronous. */
int vdw_create(vdw_handle* h, const vdw_params* p, const double* phi_k, double C_s);

/* Fix the grid N1 x N2 x N3 and the orthorhombic cell L[3] (bohr) and
 * allocate the workspace (about (Nq + 3) (N1/2+1) N2 N3 complex FP32 values
 * plus 5 N bytes).  Requirements: each N_d is {2,3,5}-smooth, 4 <= N_d <= 256,
 * N1 and N3 even, the largest |G| of the grid <= k_max.  May be called again
 * to re-plan.  Synchronous. */
int vdw_plan(vdw_handle h, int n1, int n2, int n3, const double L[3]);

/* vdw_plan with the cell given as its three lattice vectors (the form the
 * method's reciprocal-space sums take for any cell: the wavevectors G of the
 * grid and their lengths |G| come from the cell), cell[9] row-major, row i =
 * lattice vector a_i (bohr) along which grid axis i (N1, N2, N3) runs.  This
 * implementation takes orthorhombic cells: a cell whose off-diagonal entries
 * are not zero (beyond 1e-12 of its largest diagonal entry) returns
 * VDW_ERR_UNSUPPORTED and leaves the context as it was; otherwise it is
 * vdw_plan with L = the diagonal (VDW_ERR_ARG if a diagonal entry is not
 * positive).  Synchronous. */
int vdw_plan_cell(vdw_handle h, int n1, int n2, int n3, const double cell[9]);

/* E_c^nl and, on request, its potential (device pointers, caller-owned).
 *   n        [N]    density (FP32)
 *   grad     [3][N] its gradient, components x, y, z (FP32), or NULL: the
 *                   library then computes grad n = D n with its spectral
 *                   derivative (vdw_spectral_gradient) into a context-owned
 *                   buffer (allocated on first use)
 *   E        [3]    FP64 device output {E_c^nl, E_soft, Delta E} (Hartree);
 *                   E_soft is Eq. (Eoffk) with the soft kernel, Delta E the
 *                   local correction of Eqs. (DEnl, Depsnl); may be NULL.
 *   v        [N]    output or NULL.
 *   w        [3][N] output or NULL.
 * With v != NULL and w == NULL, v is v_nl of Eq. (Vi): (1/dOmega) dE/dn_i
 * with grad n_j = sum_i D_ji n_i and D the spectral derivative with the
 * Nyquist components removed, i.e. v = v_loc - sum_c D_c w_c.
 * With w != NULL, v (if given) receives only v_loc = (1/dOmega) dE/dn_i at
 * fixed gradient and w receives (1/dOmega) dE/d(grad_c n)_i, leaving the
 * chain through the gradient to the caller (a finite-difference stencil, or
 * autograd).
 * With v == NULL and w == NULL only the energy is computed.
 * Asynchronous on stream. */
int vdw_energy_potential(vdw_handle h, const float* n, const float* grad,
                         double* E, float* v, float* w, void* stream);

/* ---- several densities per call ------------------------------------------
 * The per-SCF-step cost of the method is its Nq forward and Nq inverse FFTs
 * (text after Eq. Eoffk); a training set or an energy-map scan evaluates many
 * densities of one grid.  vdw_plan_batch sizes the context's per-density
 * workspaces for Bmax densities (about (Nq + 3) (N1/2+1) N2 N3 complex FP32
 * values, twice over, plus 25 N bytes, per density); the kernel table, the
 * twiddles and the |G| order stay shared.  It synchronises the device, and
 * replaces the workspaces of earlier calls; vdw_plan resets Bmax to 1.
 * Returns VDW_ERR_OOM if they do not fit (the context must then be planned
 * again).  Synchronous. */
int vdw_plan_batch(vdw_handle h, int Bmax);

/* E_c^nl and v_nl of B <= Bmax densities of the planned grid in one call,
 * each stage one kernel launch over all of them (device pointers,
 * caller-owned, contiguous per density):
 *   n [B][N], grad [B][3][N] (required), E [B][3] FP64 ({E_c^nl, E_soft,
 *   Delta E} per density), v [B][N] or NULL (energy only).
 * Density b's results are bitwise those of vdw_energy_potential on n[b],
 * grad[b].  Asynchronous on stream. */
int vdw_energy_potential_batched(vdw_handle h, int B, const float* n, const float* grad, double* E, float* v,
                                 void* stream);

/* The same energy with the finite-difference gradient of the paper's own
 * implementation: grad n by second-order central differences on the periodic
 * grid, (f(r + h_c e_c) - f(r - h_c e_c)) / (2 h_c).  grad (device [3][N])
 * must hold that gradient, or be NULL for the library to compute it.  v (or
 * NULL for the energy alone) is v_nl of Eq. (Vi) under this operator:
 * v = v_loc - sum_c D_c w_c with D the same stencil (it is antisymmetric), so
 * v is the exact derivative of E(n, D n); the chain term costs one stencil
 * pass instead of the three spectral transforms of vdw_energy_potential.
 * Asynchronous on stream. */
int vdw_energy_potential_fd(vdw_handle h, const float* n, const float* grad, double* E, float* v, void* stream);

/* The whole exchange-correlation functional of Eq. (Exc),
 * E_xc = E_x^GGA + E_c^LDA + E_c^nl, with Dion et al.'s partners: revPBE
 * exchange (kappa = 1.245, mu = 0.066725 pi^2/3) and the Perdew-Wang LDA
 * correlation.  E (device FP64 [4]) receives {E_xc, E_c^nl, E_x, E_c^LDA};
 * v (device [N] or NULL) the potential of E_xc.  fd = 0: grad n is the
 * spectral gradient (as vdw_energy_potential), fd = 1: central differences
 * (as vdw_energy_potential_fd); grad may be NULL for the library to compute
 * it.  Asynchronous on stream. */
int vdw_xc_energy_potential(vdw_handle h, const float* n, const float* grad, double* E, float* v, int fd,
                            void* stream);

/* The same computation on host buffers (n[N], grad[3N] in; E[3], v[N] out):
 * copies the inputs to context-owned device buffers (allocated on first use),
 * runs vdw_energy_potential with the full potential, copies E and v back and
 * synchronises stream before returning.  The inputs go up in up to four z
 * slabs on a context-owned copy stream, and the pointwise pass processes each
 * slab as soon as it has arrived; the results are bitwise those of
 * vdw_energy_potential.  Host buffers should be page-locked for the copies to
 * overlap. */
int vdw_energy_potential_host(vdw_handle h, const float* n, const float* grad,
                              double* E, float* v, void* stream);

/* Number of points of the last completed call whose density was negative or
 * not finite (they were treated as n = 0).  Synchronises the device. */
int vdw_last_invalid_points(vdw_handle h, long long* count);

/* Per-stage timing, for measurement.  While enabled, vdw_energy_potential
 * (and the learned and finite-difference variants) record a CUDA event on
 * the stream before the first kernel and after each stage:
 *   0 pointwise (q, interval, theta, Delta E)   1 forward plane FFTs (x, z)
 *   2 forward y FFTs into |G| order             3 contraction (Eqs. Eoffk, epsofk)
 *   4 energy reduction                          5 inverse y FFTs
 *   6 inverse plane FFTs                        7 potential assembly (Eq. Vi)
 *   8 plane FFTs of w                           9 divergence pencils
 *  10 final planes (or the stencil divergence of the finite-difference form)
 * vdw_profile_read synchronises on the last recorded event and writes the
 * durations (ms) of the stages the last call ran into ms[0..10] (-1 for
 * stages it skipped).  Disabled by default; enabling costs up to 12 event
 * records a call. */
#define VDW_NSTAGES 11
int vdw_profile_enable(vdw_handle h, int enable);
int vdw_profile_read(vdw_handle h, float* ms);

/* ---- Delta E without device allocation ---------------------------------
 * The paper has no counterpart to this entry point.  It exists for callers
 * that must not allocate device memory when they evaluate the energy: a
 * program whose device memory all belongs to its own pool allocator, a
 * plugin host that forbids allocations inside a step, or code that cannot
 * afford the synchronisation an allocation may cause.  Create the context
 * once beforehand (vdw_create allocates its tables; vdw_plan is not needed);
 * this call then allocates nothing.
 *
 * Computes Delta E = dOmega sum_i C_s n_i^2 / (2 q_i^3), the local
 * softening correction (the value vdw_energy_potential returns in E[2]),
 * for n[npoints] and grad[3][npoints] (device, FP32) and writes it to *dE
 * (device, FP64).  Its per-block partial sums live in a fixed 32 KiB array
 * of the library (4096 FP64 slots, one per 4096 points), which every GPU that
 * loads the library keeps reserved until the process exits.
 *   - npoints > VDW_NOALLOC_MAX_POINTS (16,777,216) returns VDW_ERR_SIZE.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.
 *   - All calls share the array: two calls that may overlap on the GPU (on
 *     different streams, or from different threads) race and can return
 *     wrong values.  Calls on one stream are ordered and safe.
 * Asynchronous on stream. */
#define VDW_NOALLOC_MAX_POINTS 16777216LL
int vdw_delta_energy_noalloc(vdw_handle h, const float* n, const float* grad, long long npoints,
                             double dOmega, double* dE, void* stream);

/* ---- spectral gradient --------------------------------------------------
 * grad[3][N] = D f for a real field f[N] (device, FP32): grad_c f =
 * IFFT(i G_c f(G)) with the Nyquist component of every even axis removed, the
 * derivative whose transpose is -D (the operator in Eq. (Vi)'s gradient
 * term, spectral form of the finite differences the paper uses).  Uses the
 * context's transform workspace; needs vdw_plan.  Asynchronous on stream. */
int vdw_spectral_gradient(vdw_handle h, const float* f, float* grad, void* stream);

/* ---- learned reduced basis ------------------------------------------------
 * The paper has no learned part.  These entry points replace the Nq
 * cardinal-spline channels theta_a = n p_a(q) (Eq. fofx) and the radial table
 * phi_ab(k) (Eq. Eoffk) by VDW_LEARNED_M = 8 channels theta_m = n w_m whose
 * weights w come from a 2-64-64-8 SiLU network of two features, and by a
 * learned symmetric pair kernel K_mn(k), Catmull-Rom cubic on J uniform knots
 * k_j = j k_max/(J-1) (K even in k: the knot before k = 0 mirrors knot 1; the
 * knot past the last is the linear extrapolation).  The local correction Delta E of Eqs. (DEnl, Depsnl)
 * is kept unchanged.  The contraction, transforms and assembly are those of
 * the plain method (Eqs. Eoffk, epsilon, epsofk, Vi) with M channels.
 *
 * Features (s2 = |grad n|^2 n^(-8/3), a smooth form of |grad n| / n^(4/3)):
 *   x1 = (ln n - feat[0]) / feat[1],  x2 = (1/2 ln(s2 + feat[4]^2) - feat[2]) / feat[3]
 * Network: h1 = bf16(silu(W1 x + b1)), h2 = bf16(silu(W2 h1 + b2)),
 *   w = W3 h2 + b3; the weights are rounded to bf16, layers 2 and 3 run on
 *   the tensor cores with FP32 accumulation, together with the forward-mode
 *   tangents d/dx1, d/dx2 that give the potential the network's Jacobian
 *   (tangents rounded to bf16 where they enter a product).  Points with
 *   n <= n_min carry theta = 0.
 * Parameters: one flat FP32 vector of vdw_learned_param_count(J) values, in
 *   the order W1[64][2], b1[64], W2[64][64], b2[64], W3[8][64], b3[8],
 *   K[36][J] (pairs m <= n, row-major), W[out][in].
 * Errors: VDW_ERR_STATE before vdw_plan or vdw_learned_load; VDW_ERR_SIZE if
 *   the grid's largest |G| exceeds k_max or shared memory does not suffice. */
#define VDW_LEARNED_M 8
#define VDW_LEARNED_H 64
long long vdw_learned_param_count(int J);

/* Load (or reload, e.g. after a training step) a model for the planned grid.
 *   J       knots, 4 <= J <= 256;  k_max  last knot (bohr^-1)
 *   feat    host [5]: mu1, sig1, mu2, sig2, eps of the features
 *   base_q1, base_lambda
 *           0, 0: channel weights w = network output.  base_q1 > 0: w_m =
 *           p_m(q) + network output m, with p_m the cardinal cubic splines
 *           (Eq. fofx) on the 8-point mesh q_a = q_1 + (q_c - q_1)
 *           (lambda^a - 1)/(lambda^7 - 1) and q of Eq. (Sat) clamped to it:
 *           the network then learns a correction to the plain method's basis
 *   params  device [vdw_learned_param_count(J)] FP32; read by a kernel on
 *           stream, so it may be updated right after on the same stream.
 * The context derives its own copies (bf16 operands, knot intervals); the
 * first call allocates them (synchronous), later calls only enqueue. */
int vdw_learned_load(vdw_handle h, int J, double k_max, const double feat[5], double base_q1,
                     double base_lambda, const float* params, void* stream);

/* Tabulate the loaded network for inference.  The network's outputs depend
 * on a point only through its two features (x1, x2); this evaluates the
 * network (tensor cores, bf16 as above) once on the (T+2)^2 nodes
 * x = -D + (i - 1) h, i = 0 .. T + 1, h = 2 D / (T - 1), and from then on
 * vdw_learned_energy_potential takes each point's outputs and their Jacobian
 * from the tensor product of Catmull-Rom cubics through the 4 x 4 nodes
 * around its features (clamped to [-D, D], with zero derivative along a
 * clamped axis), so that v stays the exact derivative of that energy.  The
 * interpolation error is third order in h.  The table follows the parameters
 * of the last vdw_learned_load, which drops it: call this again after a load
 * (training steps run the network itself).  T = 0 drops the table; otherwise
 * 4 <= T <= 4096, D > 0.  Allocates (T+2)^2 x 32 bytes on the first call with
 * a given T.  Asynchronous on stream. */
int vdw_learned_tabulate(vdw_handle h, int T, double D, void* stream);

/* E and v of the learned model; arguments and outputs exactly as
 * vdw_energy_potential (E[1] holds the learned soft part, E[2] Delta E).
 * grad must be given.  Asynchronous on stream. */
int vdw_learned_energy_potential(vdw_handle h, const float* n, const float* grad, double* E, float* v,
                                 float* w, void* stream);

/* Adds coef * dE/dparams of the learned energy at (n, grad) to g_params
 * (device FP64 [vdw_learned_param_count(J)]); E (device FP64 [3]) receives
 * the energy, or NULL.  The gradient treats every bf16 rounding as the
 * identity.  Allocates an [8][N] FP32 buffer on first use.  Asynchronous. */
int vdw_learned_param_grad(vdw_handle h, const float* n, const float* grad, double coef, double* g_params,
                           double* E, void* stream);

/* Adds coef * d/dparams sum_i weight_i sum_m (w_m(x_i) - target[m][i])^2 to
 * g_params (network part only): fitting the channel weights to targets such
 * as vdw_basis_weights.  target [8][N], weight [N] device FP32.  Asynchronous. */
int vdw_learned_fit_grad(vdw_handle h, const float* n, const float* grad, const float* target,
                         const float* weight, double coef, double* g_params, void* stream);

/* Network outputs w_m at every point (0 where n <= n_min): w_out [8][N].
 * Asynchronous. */
int vdw_learned_channels(vdw_handle h, const float* n, const float* grad, float* w_out, void* stream);

/* *tc_error = 1 if a tensor-core wait in a learned kernel gave up (the
 * kernel then skipped its remaining tiles), else 0.  Synchronous. */
int vdw_learned_status(vdw_handle h, int* tc_error);

/* The plain method's cardinal weights p_a(q(n, |grad n|)) (Eq. fofx, with
 * Eq. (Sat)) for the context's Nq mesh: p_out [Nq][N], 0 where n <= n_min.
 * Needs vdw_plan.  Asynchronous. */
int vdw_basis_weights(vdw_handle h, const float* n, const float* grad, float* p_out, void* stream);

/* One Adam step (Kingma and Ba) on count FP32 parameters p with FP64
 * gradients g and FP32 moment buffers m, v (all device); step >= 1 is the
 * 1-based step number for the bias corrections.  Asynchronous. */
int vdw_adam_step(float* p, const double* g, float* m, float* v, long long count, double lr, double beta1,
                  double beta2, double eps, int step, void* stream);

/* *gave_up = 1 if, since vdw_plan, a bounded wait inside a kernel (an
 * asynchronous copy or a tensor-core completion) ran out, else 0.  Every such
 * wait polls a bounded number of times instead of spinning forever; a kernel
 * whose wait gives up waits once more (bounded) for the operation in flight,
 * then stops without using its data (a plane transform leaves its plane
 * as it was, a network warpgroup skips its remaining tiles), so that call's
 * results are wrong.  The flag lives in page-locked host memory: the next call
 * of vdw_energy_potential, vdw_energy_potential_fd, vdw_xc_energy_potential,
 * vdw_energy_potential_host, vdw_learned_energy_potential or
 * vdw_learned_param_grad on the context returns VDW_ERR_TIMEOUT without
 * running (and clears the flag), and this call keeps reporting 1 until the
 * next vdw_plan.  Synchronous. */
int vdw_wait_status(vdw_handle h, int* gave_up);

/* Bytes of device memory the context holds. */
int vdw_workspace_bytes(vdw_handle h, size_t* bytes);

int vdw_destroy(vdw_handle h);

/* Static description of an error code. */
const char* vdw_error_string(int code);

/* Text of the last error raised on this thread (empty if none). */
const char* vdw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VDWNL_H */
