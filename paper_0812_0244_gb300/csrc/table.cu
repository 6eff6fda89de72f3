// Kernel-table generation in FP64 on the GPU (initialisation, not timed).
//
// phi(d1, d2) is the Dion et al. kernel, which the paper takes as given
// (text after Eq. Enl):
//   phi = (2/pi^2) Int a^2 da Int b^2 db W(a,b) T(nu1(a), nu1(b), nu2(a), nu2(b)),
//   W(a,b) = 2 [j0(a) k(b) + j0(b) k(a) - 3 k(a) k(b)],  k(x) = (sin x - x cos x)/x^3,
//   T(w,x,y,z) = 1/2 [1/(w+x) + 1/(y+z)] [1/((w+y)(x+z)) + 1/((w+z)(y+x))],
//   nu_i(y) = y^2 / (2 h(y/d_i)),  h(t) = 1 - exp(-(4 pi/9) t^2),
// by Gauss-Legendre quadrature in t = atan(a); for min(d1, d2) >= d_asym its
// closed-form limit -12 (4 pi/9)^3 / (d1^2 d2^2 (d1^2 + d2^2)).
// Eq. (PhiSoft) softens it below d = d_s, matching value and slope along each
// ray d2/d1 = q_b/q_a; phi0 makes phi4 vanish on the diagonal.  The table is
//   phi_ab(k) = 4 pi Int_0^{r_c} r^2 phi_s(q_a r, q_b r) j0(k r) dr
// (text after Eq. Eoffk) by Simpson's rule, and C_s of Eq. (Depsnl) is
//   C_s = Int_0^{d_s/sqrt2} 4 pi x^2 [phi(x,x) - phi_s(x,x)] dx.
// The hot path then interpolates phi_ab(|G|) with a natural cubic spline in k,
// whose per-interval polynomials are built here too.
#include "common.cuh"

#include <cmath>
#include <vector>

namespace vdw {

namespace {

constexpr double PI_D = 3.14159265358979323846;

__device__ double k_series(double x) {
    // (sin x - x cos x)/x^3 = sum_{n>=1} (-1)^(n+1) 2n x^(2n-2)/(2n+1)!
    if (fabs(x) < 0.5) {
        double x2 = x * x, sum = 0.0, fact = 6.0, xp = 1.0;
        for (int n = 1; n <= 10; ++n) {
            const double term = (double)(2 * n) * xp / fact;
            sum += (n & 1) ? term : -term;
            xp *= x2;
            fact *= (double)(2 * n + 2) * (double)(2 * n + 3);
        }
        return sum;
    }
    return (sin(x) - x * cos(x)) / (x * x * x);
}

__device__ double j0_d(double x) {
    if (fabs(x) < 1e-4) return 1.0 - x * x / 6.0;
    return sin(x) / x;
}

// Per-node factors: c_i = w_i a_i^2, j0(a_i), k(a_i).
__global__ void k_dion_nodes(const double* a, const double* wa, int na, double* c, double* j0v, double* kv) {
    for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < na; i += blockDim.x * gridDim.x) {
        c[i] = wa[i] * a[i] * a[i];
        j0v[i] = j0_d(a[i]);
        kv[i] = k_series(a[i]);
    }
}

__device__ __forceinline__ void nu_dnu(double y, double d, double& nu, double& dnu) {
    if (d <= 0.0) { nu = 0.5 * y * y; dnu = 0.0; return; }
    const double gam = 4.0 * PI_D / 9.0;
    const double s = y / d;
    const double e = exp(-gam * s * s);
    const double h = 1.0 - e;
    if (h <= 0.0) { nu = d * d / (2.0 * gam); dnu = d / gam; return; }
    nu = y * y / (2.0 * h);
    dnu = y * y * gam * s * s * e / (h * h * d);
}

struct Nodes {
    const double* a;
    const double* c;
    const double* j0;
    const double* k;
    int na;
};

__device__ double block_sum_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// Quadrature of phi at (d1, d2) by one block; optional derivative along the
// ray.  Shared memory: 7 na doubles.
__device__ void dion_block(double d1, double d2, const Nodes& nd, double* sm, double* red, double* phi,
                           double* dphi) {
    const int na = nd.na;
    double* n1 = sm;
    double* n2 = n1 + na;
    double* dn1 = n2 + na;
    double* dn2 = dn1 + na;
    double* cc = dn2 + na;
    double* jj = cc + na;
    double* kk = jj + na;
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
        nu_dnu(nd.a[i], d1, n1[i], dn1[i]);
        nu_dnu(nd.a[i], d2, n2[i], dn2[i]);
        cc[i] = nd.c[i];
        jj[i] = nd.j0[i];
        kk[i] = nd.k[i];
    }
    __syncthreads();
    const double pref = 4.0 / (PI_D * PI_D);  // (2/pi^2) times the 2 of W
    double sum = 0.0, s1 = 0.0, s2 = 0.0;
    if (dphi == nullptr) {
        // T and K are symmetric under i <-> j: upper triangle, rows paired for balance
        const int half = (na + 1) / 2;
        for (int t = threadIdx.x; t < half; t += blockDim.x) {
            for (int rr = 0; rr < 2; ++rr) {
                const int i = rr == 0 ? t : na - 1 - t;
                if (rr == 1 && i == t) break;
                const double w = n1[i], y = n2[i];
                const double ci = cc[i], ji = jj[i], ki = kk[i];
                double row = pref * ci * ci * (2.0 * ji * ki - 3.0 * ki * ki) / (2.0 * w * y * (w + y));
                for (int j = i + 1; j < na; ++j) {
                    const double x = n1[j], z = n2[j];
                    const double K = pref * ci * cc[j] * (ji * kk[j] + jj[j] * ki - 3.0 * ki * kk[j]);
                    const double wx = w + x, yz = y + z, wy = w + y, xz = x + z, wz = w + z, yx = y + x;
                    const double T = 0.5 * (wx + yz) * (wz * yx + wy * xz) / (wx * yz * wy * xz * wz * yx);
                    row += 2.0 * K * T;
                }
                sum += row;
            }
        }
    } else {
        for (int i = threadIdx.x; i < na; i += blockDim.x) {
            const double w = n1[i], y = n2[i];
            const double ci = cc[i], ji = jj[i], ki = kk[i];
            for (int j = 0; j < na; ++j) {
                const double x = n1[j], z = n2[j];
                const double K = pref * ci * cc[j] * (ji * kk[j] + jj[j] * ki - 3.0 * ki * kk[j]);
                const double iwx = 1.0 / (w + x), iyz = 1.0 / (y + z);
                const double iwy = 1.0 / (w + y), ixz = 1.0 / (x + z);
                const double iwz = 1.0 / (w + z), iyx = 1.0 / (y + x);
                const double S = iwx + iyz, P = iwy * ixz + iwz * iyx;
                sum += K * 0.5 * S * P;
                const double Pw = -iwy * iwy * ixz - iwz * iwz * iyx;
                const double Px = -iwy * ixz * ixz - iwz * iyx * iyx;
                const double Py = -iwy * iwy * ixz - iwz * iyx * iyx;
                const double Pz = -iwy * ixz * ixz - iwz * iwz * iyx;
                const double Sw = -iwx * iwx, Sy = -iyz * iyz;
                s1 += K * (0.5 * (Sw * P + S * Pw) * dn1[i] + 0.5 * (Sw * P + S * Px) * dn1[j]);
                s2 += K * (0.5 * (Sy * P + S * Py) * dn2[i] + 0.5 * (Sy * P + S * Pz) * dn2[j]);
            }
        }
    }
    const double tot = block_sum_d(sum, red);
    if (dphi) {
        __syncthreads();
        const double t1 = block_sum_d(s1, red);
        __syncthreads();
        const double t2 = block_sum_d(s2, red);
        if (threadIdx.x == 0) {
            const double d = sqrt(d1 * d1 + d2 * d2);
            *dphi = d > 0.0 ? (d1 * t1 + d2 * t2) / d : 0.0;
        }
    }
    if (threadIdx.x == 0) *phi = tot;
}

// phi (and optionally d phi/dd) at a list of points, quadrature only.
__global__ void __launch_bounds__(128) k_dion_points(const double* d1, const double* d2, int npts, Nodes nd,
                                                     double* phi, double* dphi) {
    extern __shared__ double sm[];
    __shared__ double red[32];
    const int p = blockIdx.x;
    if (p >= npts) return;
    dion_block(d1[p], d2[p], nd, sm, red, phi + p, dphi ? dphi + p : nullptr);
}

// Soft-kernel coefficients: F, dF at index 0 belong to the diagonal ray, the
// following npairs to the pair rays.
__global__ void k_soft_coeffs(const double* F, const double* dF, int npairs, double ds, double* phi0,
                              double* phi2, double* phi4) {
    const double p0 = F[0] - dF[0] * ds / 2.0;
    for (int p = threadIdx.x; p <= npairs; p += blockDim.x) {
        const double f4 = (p0 - F[p] + dF[p] * ds / 2.0) / (ds * ds * ds * ds);
        phi4[p] = f4;
        phi2[p] = dF[p] / (2.0 * ds) - 2.0 * ds * ds * f4;
    }
    if (threadIdx.x == 0) *phi0 = p0;
}

// phi_s,ab(r_j) for every pair and radial point.
__global__ void __launch_bounds__(128) k_phi_r(const double* qm, int Nq, int Nr, double dr, double ds, double d_asym,
                                               const double* phi0, const double* phi2, const double* phi4, Nodes nd,
                                               double* phir) {
    extern __shared__ double sm[];
    __shared__ double red[32];
    const int j = blockIdx.x, p = blockIdx.y;
    // pair index -> (a, b), a <= b, row-major
    int a = 0, rem = p;
    while (rem >= Nq - a) { rem -= Nq - a; ++a; }
    const int b = a + rem;
    const double qa = qm[a], qb = qm[b];
    const double r = (double)j * dr;
    const double qq = hypot(qa, qb);
    const double d = qq * r;
    double* out = phir + (size_t)p * (Nr + 1) + j;
    const double d1 = qa * r, d2 = qb * r;
    if (d < ds) {
        if (threadIdx.x == 0) {
            const double d2s = d * d;
            *out = phi0[0] + phi2[p + 1] * d2s + phi4[p + 1] * d2s * d2s;
        }
        return;
    }
    if (fmin(d1, d2) >= d_asym) {
        if (threadIdx.x == 0) {
            const double C = 12.0 * pow(4.0 * PI_D / 9.0, 3.0);
            *out = -C / (d1 * d1 * d2 * d2 * (d1 * d1 + d2 * d2));
        }
        return;
    }
    dion_block(d1, d2, nd, sm, red, out, nullptr);
}

// phi_ab(k_m) = sum_j 4 pi w_j r_j^2 phi_ab(r_j) j0(k_m r_j), Simpson weights w_j.
__global__ void __launch_bounds__(256) k_radial_ft(const double* phir, int npairs, int Nr, double dr, double dk,
                                                   double* phik) {
    extern __shared__ double J[];
    const int m = blockIdx.x;
    const double k = (double)m * dk;
    for (int j = threadIdx.x; j <= Nr; j += blockDim.x) {
        const double r = (double)j * dr;
        double w = (j == 0 || j == Nr) ? 1.0 : ((j & 1) ? 4.0 : 2.0);
        w *= dr / 3.0;
        const double kr = k * r;
        const double j0 = (kr == 0.0) ? 1.0 : sin(kr) / kr;
        J[j] = 4.0 * PI_D * w * r * r * j0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int Nk = gridDim.x;
    for (int p = warp; p < npairs; p += nw) {
        const double* f = phir + (size_t)p * (Nr + 1);
        double s = 0.0;
        for (int j = lane; j <= Nr; j += 32) s += J[j] * f[j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) phik[(size_t)p * Nk + m] = s;
    }
}

// C_s from the diagonal quadrature values phid at Gauss nodes x with weights wx.
__global__ void k_softening(const double* x, const double* wx, const double* phid, int n, const double* phi0,
                            const double* phi2, const double* phi4, double* Cs) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double d2 = 2.0 * x[i] * x[i];
        const double fs = phi0[0] + phi2[0] * d2 + phi4[0] * d2 * d2;
        s += wx[i] * 4.0 * PI_D * x[i] * x[i] * (phid[i] - fs);
    }
    const double t = block_sum_d(s, red);
    if (threadIdx.x == 0) *Cs = t;
}

// Natural cubic spline in k of each pair (Thomas algorithm on the uniform
// mesh), written as per-interval polynomials c0 + c1 t + c2 t^2 + c3 t^3 in
// t = (k - k_j)/dk: kcoef[j * npairs + p].
__global__ void k_kspline(const double* phik, int npairs, int Nk, double dk, double* scratch, float4* kcoef) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const double* y = phik + (size_t)p * Nk;
    double* M = scratch + (size_t)p * 2 * Nk;
    double* cp = M + Nk;
    // rows i = 1..Nk-2: M_{i-1} + 4 M_i + M_{i+1} = 6 (y_{i+1} - 2 y_i + y_{i-1}) / dk^2
    M[0] = 0.0;
    M[Nk - 1] = 0.0;
    const double inv = 6.0 / (dk * dk);
    // forward sweep: cp holds the modified super-diagonal, M the modified rhs
    double prev_c = 0.0, prev_d = 0.0;
    for (int i = 1; i <= Nk - 2; ++i) {
        const double rhs = inv * (y[i + 1] - 2.0 * y[i] + y[i - 1]);
        const double den = 4.0 - (i > 1 ? prev_c : 0.0);
        const double c = 1.0 / den;
        const double d = (rhs - (i > 1 ? prev_d : 0.0)) / den;
        cp[i] = c;
        M[i] = d;
        prev_c = c;
        prev_d = d;
    }
    for (int i = Nk - 3; i >= 1; --i) M[i] -= cp[i] * M[i + 1];
    const double h6 = dk * dk / 6.0;
    for (int j = 0; j < Nk - 1; ++j) {
        const double c0 = y[j];
        const double c1 = (y[j + 1] - y[j]) + h6 * (-2.0 * M[j] - M[j + 1]);
        const double c2 = h6 * 3.0 * M[j];
        const double c3 = h6 * (M[j + 1] - M[j]);
        kcoef[(size_t)j * npairs + p] = make_float4((float)c0, (float)c1, (float)c2, (float)c3);
    }
}

// Cardinal natural cubic splines on the q mesh: M[a][k] for the data delta_ak.
__global__ void k_cardinal(const double* qm, int Nq, double* Mout) {
    const int a = threadIdx.x;
    if (a >= Nq) return;
    double cp[MAX_NQ], dd[MAX_NQ], M[MAX_NQ];
    for (int i = 0; i < Nq; ++i) M[i] = 0.0;
    for (int i = 1; i <= Nq - 2; ++i) {
        const double h0 = qm[i] - qm[i - 1], h1 = qm[i + 1] - qm[i];
        const double y0 = (i - 1 == a), y1 = (i == a), y2 = (i + 1 == a);
        const double rhs = 6.0 * ((y2 - y1) / h1 - (y1 - y0) / h0);
        const double lo = (i > 1) ? h0 : 0.0;
        const double den = 2.0 * (h0 + h1) - (i > 1 ? lo * cp[i - 1] : 0.0);
        cp[i] = h1 / den;
        dd[i] = (rhs - (i > 1 ? lo * dd[i - 1] : 0.0)) / den;
    }
    for (int i = Nq - 2; i >= 1; --i) M[i] = dd[i] - (i < Nq - 2 ? cp[i] * M[i + 1] : 0.0);
    for (int k = 0; k < Nq; ++k) Mout[a * Nq + k] = M[k];
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(PI_D * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

std::vector<double> q_mesh_host(const vdw_params* p) {
    std::vector<double> q(p->Nq);
    const double den = std::pow(p->lambda, p->Nq - 1) - 1.0;
    for (int a = 0; a < p->Nq; ++a) q[a] = p->q_1 + (p->q_c - p->q_1) * (std::pow(p->lambda, a) - 1.0) / den;
    return q;
}

struct DevBuf {
    std::vector<void*> ptrs;
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T** p, size_t n) {
        cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

int check_params(const vdw_params* p) {
    if (!p) return VDW_ERR_ARG;
    if (p->Nq < 4 || p->Nq > MAX_NQ || p->q_1 <= 0 || p->q_c <= p->q_1 || p->lambda <= 1.0 || p->m_c < 1 || p->m_c > MAX_MC ||
        p->d_s <= 0 || p->na < 8 || p->na > 4096 || p->a_max <= 0 || p->d_asym <= p->d_s || p->r_c <= 0 ||
        p->Nr < 2 || (p->Nr & 1) || p->k_max <= 0 || p->Nk < 4 || p->n_cs < 2 || !(p->n_min >= 0))
        return VDW_ERR_ARG;
    return VDW_OK;
}

}  // namespace

int table_build(const vdw_params* p, double* h_qmesh, double* h_phik, double* h_phi0, double* h_Cs) {
    int rc = check_params(p);
    if (rc) { set_error("invalid vdw_params"); return rc; }
    const int Nq = p->Nq, npairs = Nq * (Nq + 1) / 2, na = p->na, Nr = p->Nr, Nk = p->Nk;
    std::vector<double> qm = q_mesh_host(p);
    std::vector<double> gx, gw;
    gauss_legendre(na, gx, gw);
    const double T = std::atan(p->a_max);
    std::vector<double> a(na), wa(na);
    for (int i = 0; i < na; ++i) {
        const double t = 0.5 * T * (gx[i] + 1.0);
        a[i] = std::tan(t);
        wa[i] = 0.5 * T * gw[i] * (1.0 + a[i] * a[i]);
    }
    // points for the soft coefficients: diagonal, then the pair rays at d_s
    std::vector<double> pd1(npairs + 1), pd2(npairs + 1);
    pd1[0] = pd2[0] = p->d_s / std::sqrt(2.0);
    for (int aa = 0, ip = 1; aa < Nq; ++aa)
        for (int bb = aa; bb < Nq; ++bb, ++ip) {
            const double qq = std::hypot(qm[aa], qm[bb]);
            pd1[ip] = p->d_s * (qm[aa] / qq);
            pd2[ip] = p->d_s * (qm[bb] / qq);
        }
    // Gauss nodes of the softening integral
    std::vector<double> cx, cw;
    gauss_legendre(p->n_cs, cx, cw);
    const double X = p->d_s / std::sqrt(2.0);
    for (int i = 0; i < p->n_cs; ++i) {
        cx[i] = 0.5 * X * (cx[i] + 1.0);
        cw[i] = 0.5 * X * cw[i];
    }

    DevBuf B;
    double *d_a, *d_wa, *d_c, *d_j0, *d_k, *d_qm, *d_pd1, *d_pd2, *d_F, *d_dF, *d_phi0, *d_phi2, *d_phi4;
    double *d_phir, *d_phik, *d_cx, *d_cw, *d_cphi, *d_Cs;
    VDW_CUDA(B.alloc(&d_a, na));
    VDW_CUDA(B.alloc(&d_wa, na));
    VDW_CUDA(B.alloc(&d_c, na));
    VDW_CUDA(B.alloc(&d_j0, na));
    VDW_CUDA(B.alloc(&d_k, na));
    VDW_CUDA(B.alloc(&d_qm, Nq));
    VDW_CUDA(B.alloc(&d_pd1, npairs + 1));
    VDW_CUDA(B.alloc(&d_pd2, npairs + 1));
    VDW_CUDA(B.alloc(&d_F, npairs + 1));
    VDW_CUDA(B.alloc(&d_dF, npairs + 1));
    VDW_CUDA(B.alloc(&d_phi0, 1));
    VDW_CUDA(B.alloc(&d_phi2, npairs + 1));
    VDW_CUDA(B.alloc(&d_phi4, npairs + 1));
    VDW_CUDA(B.alloc(&d_phir, (size_t)npairs * (Nr + 1)));
    VDW_CUDA(B.alloc(&d_phik, (size_t)npairs * Nk));
    VDW_CUDA(B.alloc(&d_cx, p->n_cs));
    VDW_CUDA(B.alloc(&d_cw, p->n_cs));
    VDW_CUDA(B.alloc(&d_cphi, p->n_cs));
    VDW_CUDA(B.alloc(&d_Cs, 1));
    VDW_CUDA(cudaMemcpy(d_a, a.data(), sizeof(double) * na, cudaMemcpyHostToDevice));
    VDW_CUDA(cudaMemcpy(d_wa, wa.data(), sizeof(double) * na, cudaMemcpyHostToDevice));
    VDW_CUDA(cudaMemcpy(d_qm, qm.data(), sizeof(double) * Nq, cudaMemcpyHostToDevice));
    VDW_CUDA(cudaMemcpy(d_pd1, pd1.data(), sizeof(double) * (npairs + 1), cudaMemcpyHostToDevice));
    VDW_CUDA(cudaMemcpy(d_pd2, pd2.data(), sizeof(double) * (npairs + 1), cudaMemcpyHostToDevice));
    VDW_CUDA(cudaMemcpy(d_cx, cx.data(), sizeof(double) * p->n_cs, cudaMemcpyHostToDevice));
    VDW_CUDA(cudaMemcpy(d_cw, cw.data(), sizeof(double) * p->n_cs, cudaMemcpyHostToDevice));

    k_dion_nodes<<<(na + 255) / 256, 256>>>(d_a, d_wa, na, d_c, d_j0, d_k);
    Nodes nd{d_a, d_c, d_j0, d_k, na};
    const size_t smq = sizeof(double) * 7 * na;
    raise_smem_limit(k_dion_points, smq);
    raise_smem_limit(k_phi_r, smq);
    k_dion_points<<<npairs + 1, 128, smq>>>(d_pd1, d_pd2, npairs + 1, nd, d_F, d_dF);
    k_soft_coeffs<<<1, 256>>>(d_F, d_dF, npairs, p->d_s, d_phi0, d_phi2, d_phi4);
    const double dr = p->r_c / Nr;
    k_phi_r<<<dim3(Nr + 1, npairs), 128, smq>>>(d_qm, Nq, Nr, dr, p->d_s, p->d_asym, d_phi0, d_phi2, d_phi4, nd,
                                                d_phir);
    const double dk = p->k_max / (Nk - 1);
    const size_t smj = sizeof(double) * (Nr + 1);
    raise_smem_limit(k_radial_ft, smj);
    k_radial_ft<<<Nk, 256, smj>>>(d_phir, npairs, Nr, dr, dk, d_phik);
    k_dion_points<<<p->n_cs, 128, smq>>>(d_cx, d_cx, p->n_cs, nd, d_cphi, nullptr);
    k_softening<<<1, 256>>>(d_cx, d_cw, d_cphi, p->n_cs, d_phi0, d_phi2, d_phi4, d_Cs);
    VDW_CUDA(cudaGetLastError());
    VDW_CUDA(cudaDeviceSynchronize());

    if (h_qmesh)
        for (int i = 0; i < Nq; ++i) h_qmesh[i] = qm[i];
    if (h_phi0) VDW_CUDA(cudaMemcpy(h_phi0, d_phi0, sizeof(double), cudaMemcpyDeviceToHost));
    if (h_Cs) VDW_CUDA(cudaMemcpy(h_Cs, d_Cs, sizeof(double), cudaMemcpyDeviceToHost));
    if (h_phik) {
        std::vector<double> pk((size_t)npairs * Nk);
        VDW_CUDA(cudaMemcpy(pk.data(), d_phik, sizeof(double) * pk.size(), cudaMemcpyDeviceToHost));
        for (int aa = 0, ip = 0; aa < Nq; ++aa)
            for (int bb = aa; bb < Nq; ++bb, ++ip)
                for (int m = 0; m < Nk; ++m) {
                    h_phik[((size_t)aa * Nq + bb) * Nk + m] = pk[(size_t)ip * Nk + m];
                    h_phik[((size_t)bb * Nq + aa) * Nk + m] = pk[(size_t)ip * Nk + m];
                }
    }
    return VDW_OK;
}

int table_upload(vdw_ctx* c, const double* h_phik, double C_s) {
    const vdw_params* p = &c->p;
    const int Nq = p->Nq, npairs = Nq * (Nq + 1) / 2, Nk = p->Nk;
    std::vector<double> qm = q_mesh_host(p);
    std::vector<double> pk((size_t)npairs * Nk);
    for (int aa = 0, ip = 0; aa < Nq; ++aa)
        for (int bb = aa; bb < Nq; ++bb, ++ip)
            for (int m = 0; m < Nk; ++m) pk[(size_t)ip * Nk + m] = h_phik[((size_t)aa * Nq + bb) * Nk + m];
    DevBuf B;
    double *d_phik, *d_scr, *d_qm, *d_M;
    VDW_CUDA(B.alloc(&d_phik, pk.size()));
    VDW_CUDA(B.alloc(&d_scr, (size_t)npairs * 2 * Nk));
    VDW_CUDA(B.alloc(&d_qm, Nq));
    VDW_CUDA(B.alloc(&d_M, (size_t)Nq * Nq));
    VDW_CUDA(cudaMemcpy(d_phik, pk.data(), sizeof(double) * pk.size(), cudaMemcpyHostToDevice));
    VDW_CUDA(cudaMemcpy(d_qm, qm.data(), sizeof(double) * Nq, cudaMemcpyHostToDevice));
    if (c->d_kcoef) { cudaFree(c->d_kcoef); c->d_kcoef = nullptr; }
    VDW_CUDA(cudaMalloc(&c->d_kcoef, sizeof(float4) * (size_t)(Nk - 1) * npairs));
    const double dk = p->k_max / (Nk - 1);
    k_kspline<<<(npairs + 63) / 64, 64>>>(d_phik, npairs, Nk, dk, d_scr, c->d_kcoef);
    k_cardinal<<<1, 32>>>(d_qm, Nq, d_M);
    VDW_CUDA(cudaGetLastError());
    std::vector<double> M((size_t)Nq * Nq);
    VDW_CUDA(cudaMemcpy(M.data(), d_M, sizeof(double) * M.size(), cudaMemcpyDeviceToHost));
    PointParams& P = c->pp;
    if (p->m_c < 1 || p->m_c > MAX_MC) {
        set_error("m_c must be in [1, 32]");
        return VDW_ERR_ARG;
    }
    P.Nq = Nq;
    P.m_c = p->m_c;
    for (int m = 0; m <= MAX_MC; ++m) P.inv_m[m] = m > 0 ? 1.0f / (float)m : 0.f;  // correctly rounded
    P.q_c = (float)p->q_c;
    P.n_min = (float)p->n_min;
    P.C_s = (float)C_s;
    for (int i = 0; i < MAX_NQ; ++i) {
        P.qm[i] = i < Nq ? (float)qm[i] : 0.f;
        for (int k = 0; k < MAX_NQ; ++k) P.Mq[i][k] = (i < Nq && k < Nq) ? (float)M[(size_t)i * Nq + k] : 0.f;
    }
    c->C_s = C_s;
    return VDW_OK;
}

}  // namespace vdw
