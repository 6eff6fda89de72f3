// The hot path of the Roman-Perez--Soler evaluation on one GB300.
//
//   P0 k_pointwise      n, grad n -> q, mesh interval k, position t (Eq. Sat,
//                       Eq. fofx); Delta E partial sums (Eqs. DEnl, Depsnl)
//   P1 k_theta_plane    theta_a = n p_a(q) (text after Eq. Eoffk) on one xz
//                       plane, R2C along x and C2C along z in shared memory
//   P2 k_pencil_contract  C2C along y of all Nq fields of a few columns, then
//                       per G: u_a(G) = sum_b phi_ab(|G|) theta_b(G) with phi_ab
//                       from the radial table, energy of Eq. (Eoffk) in FP64,
//                       inverse C2C along y (Eqs. epsilon, epsofk)
//   P3 k_assemble       inverse plane transform of u_a, Eq. (Vi): v_loc and
//                       w = dE/d grad n, forward plane transform of w
//   P4 k_pencil_div     y transform of w, i G' . w(G), inverse y transform
//   P5 k_div_final      inverse plane transform, v = v_loc - D . w
//
// Layouts: real fields [N3][N2][N1] flat (x fastest); spectra
// [field][N2][N3][Nh] with Nh = N1/2+1 (a y plane of the half spectrum is one
// contiguous block, a pencil along y strides by N3 Nh).
#include "fft.cuh"
#include "pointwise.cuh"

#include <algorithm>
#include <vector>

namespace vdw {

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed order); result valid in thread 0.
__device__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__device__ __forceinline__ void load_twiddles(float2* dst, const float2* src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// P0: pointwise
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_pointwise(const float* __restrict__ n, const float* __restrict__ grad,
                                                   long long N, PointParams P, float* __restrict__ t_out,
                                                   uint8_t* __restrict__ k_out, double* __restrict__ epart,
                                                   unsigned long long* __restrict__ invalid) {
    __shared__ double red[32];
    double acc = 0.0;
    unsigned int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float ni = n[i];
        bad += (!(ni >= 0.f) || !isfinite(ni)) ? 1u : 0u;
        const QPoint qp = q_point(ni, grad[i], grad[N + i], grad[2 * N + i], P);
        t_out[i] = qp.t;
        k_out[i] = (uint8_t)qp.k;
        if (qp.k != K_INVALID) {
            const float q3 = qp.q * qp.q * qp.q;
            acc += (double)(0.5f * P.C_s * ni * ni / q3);
        }
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) epart[blockIdx.x] = s;
    __syncthreads();
    const double b = block_sum((double)bad, red);
    if (threadIdx.x == 0 && b > 0.0) atomicAdd(invalid, (unsigned long long)b);
}

// ---------------------------------------------------------------------------
// plane helpers (one y plane, N3 rows of N1 reals <-> N3 x Nh half spectrum)
// ---------------------------------------------------------------------------
// Real value of point (x, z) in the packed layout: rows 2j and 2j+1 share the
// complex row at offset j (2 Nh), as real and imaginary parts.
__device__ __forceinline__ int packed_index(int x, int z, int Nh) { return 2 * ((z >> 1) * 2 * Nh + x) + (z & 1); }

// Forward: packed real rows -> half spectrum (x R2C, then z C2C).
__device__ void plane_forward(float2* plane, const GridArgs& g, const float2* tw1, const float2* tw3) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int row = warp; row < g.N3 / 2; row += nw) {
        float2* p = plane + row * 2 * g.Nh;
        line_fft<false>(p, 1, g.p1, tw1, lane);
        r2c_untangle(p, g.N1, lane);
    }
    __syncthreads();
    for (int col = warp; col < g.Nh; col += nw) line_fft<false>(plane + col, g.Nh, g.p3, tw3, lane);
    __syncthreads();
}

// Inverse: half spectrum -> packed real rows (z C2C inverse, then x C2R), unscaled.
__device__ void plane_inverse(float2* plane, const GridArgs& g, const float2* tw1, const float2* tw3) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int col = warp; col < g.Nh; col += nw) line_fft<true>(plane + col, g.Nh, g.p3, tw3, lane);
    __syncthreads();
    for (int row = warp; row < g.N3 / 2; row += nw) {
        float2* p = plane + row * 2 * g.Nh;
        c2r_tangle(p, g.N1, lane);
        line_fft<true>(p, 1, g.p1, tw1, lane);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// P1: theta_a planes, forward plane transform
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_theta_plane(const float* __restrict__ n, const float* __restrict__ tk,
                                                     const uint8_t* __restrict__ kk, GridArgs g, PointParams P,
                                                     const float2* __restrict__ tw, float2* __restrict__ spec) {
    extern __shared__ float2 sm[];
    float2* plane = sm;
    float2* tw1 = plane + g.N3 * g.Nh;
    float2* tw3 = tw1 + g.N1;
    const int y = blockIdx.x, a = blockIdx.y;
    load_twiddles(tw1, tw, g.N1);
    load_twiddles(tw3, tw + g.N1 + g.N2, g.N3);
    float* pf = reinterpret_cast<float*>(plane);
    const int np = g.N1 * g.N3;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int x = i % g.N1, z = i / g.N1;
        const long long gi = x + (long long)g.N1 * (y + (long long)g.N2 * z);
        const int k = kk[gi];
        float th = 0.f;
        if (k != K_INVALID) th = n[gi] * cardinal_value(P, a, k, tk[gi]);
        pf[packed_index(x, z, g.Nh)] = th;
    }
    __syncthreads();
    plane_forward(plane, g, tw1, tw3);
    float2* dst = spec + ((long long)a * g.N2 + y) * g.ncols;
    for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) dst[i] = plane[i];
}

// ---------------------------------------------------------------------------
// P2: pencils along y, contraction with the radial kernel table, energy
// ---------------------------------------------------------------------------
template <int NQ>
__global__ void __launch_bounds__(256, 2) k_pencil_contract(float2* __restrict__ spec, GridArgs g,
                                                         const float4* __restrict__ kcoef,
                                                         const float2* __restrict__ tw, double* __restrict__ epart,
                                                         int C, int write_back) {
    extern __shared__ float2 sm[];
    __shared__ double red[32];
    const int N2 = g.N2;
    float2* lines = sm;                  // [NQ][C][N2]
    float2* tw2 = lines + NQ * C * N2;
    load_twiddles(tw2, tw + g.N1, N2);
    const int c0 = blockIdx.x * C;
    const int tot = NQ * N2 * C;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        const int cc = i % C, r = i / C, yy = r % N2, a = r / N2;
        const int col = c0 + cc;
        float2 val = make_float2(0.f, 0.f);
        if (col < g.ncols) val = spec[((long long)a * N2 + yy) * g.ncols + col];
        lines[(a * C + cc) * N2 + yy] = val;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int l = warp; l < NQ * C; l += nw) line_fft<false>(lines + l * N2, 1, g.p2, tw2, lane);
    __syncthreads();

    constexpr int NP = NQ * (NQ + 1) / 2;
    double eacc = 0.0;
    for (int pt = threadIdx.x; pt < C * N2; pt += blockDim.x) {
        const int cc = pt / N2, yy = pt % N2;
        const int col = c0 + cc;
        if (col >= g.ncols) continue;
        const int kx = col % g.Nh, kz = col / g.Nh;
        const int my = (2 * yy <= N2) ? yy : yy - N2;
        const int mz = (2 * kz <= g.N3) ? kz : kz - g.N3;
        const float G2 = g.gx2 * (float)(kx * kx) + g.gy2 * (float)(my * my) + g.gz2 * (float)(mz * mz);
        const float s = sqrtf(G2) * g.inv_dk;
        const int j = min((int)s, g.Nk - 2);
        const float t = s - (float)j;
        const float4* cf = kcoef + (long long)j * NP;
        float2 th[NQ], u[NQ];
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
            th[a] = lines[(a * C + cc) * N2 + yy];
            u[a] = make_float2(0.f, 0.f);
        }
        int p = 0;
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
#pragma unroll
            for (int b = a; b < NQ; ++b, ++p) {
                const float4 c = __ldg(cf + p);
                const float phi = fmaf(t, fmaf(t, fmaf(t, c.w, c.z), c.y), c.x);
                u[a].x = fmaf(phi, th[b].x, u[a].x);
                u[a].y = fmaf(phi, th[b].y, u[a].y);
                if (b != a) {
                    u[b].x = fmaf(phi, th[a].x, u[b].x);
                    u[b].y = fmaf(phi, th[a].y, u[b].y);
                }
            }
        }
        float e = 0.f;
#pragma unroll
        for (int a = 0; a < NQ; ++a) e = fmaf(th[a].x, u[a].x, fmaf(th[a].y, u[a].y, e));
        const bool single = (kx == 0) || (2 * kx == g.N1);
        eacc += (double)e * (single ? 1.0 : 2.0);
        if (write_back) {
#pragma unroll
            for (int a = 0; a < NQ; ++a) lines[(a * C + cc) * N2 + yy] = cscale(u[a], g.invN);
        }
    }
    const double es = block_sum(eacc, red);
    if (threadIdx.x == 0) epart[blockIdx.x] = es;
    if (!write_back) return;
    __syncthreads();
    for (int l = warp; l < NQ * C; l += nw) line_fft<true>(lines + l * N2, 1, g.p2, tw2, lane);
    __syncthreads();
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        const int cc = i % C, r = i / C, yy = r % N2, a = r / N2;
        const int col = c0 + cc;
        if (col < g.ncols) spec[((long long)a * N2 + yy) * g.ncols + col] = lines[(a * C + cc) * N2 + yy];
    }
}

// ---------------------------------------------------------------------------
// P3: inverse plane transforms of u_a and the assembly of Eq. (Vi)
// ---------------------------------------------------------------------------
// mode 0: v = v_loc (if v), w written to w_out; mode 1: v_loc to v, w(G) to wspec
__global__ void __launch_bounds__(512) k_assemble(const float2* __restrict__ spec, const float* __restrict__ n,
                                                  const float* __restrict__ grad, const float* __restrict__ tk,
                                                  const uint8_t* __restrict__ kk, GridArgs g, PointParams P,
                                                  const float2* __restrict__ tw, float* __restrict__ v,
                                                  float* __restrict__ w_out, float2* __restrict__ wspec, int mode,
                                                  float* __restrict__ acc_global) {
    extern __shared__ float2 sm[];
    const int np = g.N1 * g.N3;
    const int y = blockIdx.x;
    float2* plane = sm;
    float2* tw1 = plane + g.N3 * g.Nh;
    float2* tw3 = tw1 + g.N1;
    // per-point accumulators: shared memory when the plane leaves room for
    // them, otherwise this block's slice of a global scratch buffer
    float* S0 = acc_global ? acc_global + (long long)y * 2 * np : reinterpret_cast<float*>(tw3 + g.N3);
    float* S1 = S0 + np;
    load_twiddles(tw1, tw, g.N1);
    load_twiddles(tw3, tw + g.N1 + g.N2, g.N3);
    for (int i = threadIdx.x; i < np; i += blockDim.x) { S0[i] = 0.f; S1[i] = 0.f; }
    const float* pf = reinterpret_cast<const float*>(plane);
    for (int a = 0; a < P.Nq; ++a) {
        const float2* src = spec + ((long long)a * g.N2 + y) * g.ncols;
        __syncthreads();
        for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) plane[i] = src[i];
        __syncthreads();
        plane_inverse(plane, g, tw1, tw3);
        for (int i = threadIdx.x; i < np; i += blockDim.x) {
            const int x = i % g.N1, z = i / g.N1;
            const long long gi = x + (long long)g.N1 * (y + (long long)g.N2 * z);
            const int k = kk[gi];
            if (k == K_INVALID) continue;
            float pa, dpa;
            cardinal(P, a, k, tk[gi], pa, dpa);
            const float u = pf[packed_index(x, z, g.Nh)];
            S0[i] = fmaf(u, pa, S0[i]);
            S1[i] = fmaf(u, dpa, S1[i]);
        }
    }
    __syncthreads();
    const long long N = g.N;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int x = i % g.N1, z = i / g.N1;
        const long long gi = x + (long long)g.N1 * (y + (long long)g.N2 * z);
        const float ni = n[gi];
        const float gx = grad[gi], gy = grad[N + gi], gz = grad[2 * N + gi];
        const QPoint qp = q_point(ni, gx, gy, gz, P);
        float vl = 0.f, gg = 0.f;
        if (qp.k != K_INVALID) {
            const float q = qp.q, q3 = q * q * q, q4 = q3 * q;
            const float cn = 1.5f * P.C_s * ni * ni / q4;
            vl = S0[i] + ni * qp.dq_dn * S1[i] + P.C_s * ni / q3 - cn * qp.dq_dn;
            gg = ni * S1[i] * qp.dq_dg - cn * qp.dq_dg;
        }
        if (v) v[gi] = vl;
        if (mode == 0) {
            if (w_out) {
                w_out[gi] = gg * gx;
                w_out[N + gi] = gg * gy;
                w_out[2 * N + gi] = gg * gz;
            }
        } else {
            S1[i] = gg;
        }
    }
    if (mode == 0) return;
    float* pw = reinterpret_cast<float*>(plane);
    for (int c = 0; c < 3; ++c) {
        __syncthreads();
        for (int i = threadIdx.x; i < np; i += blockDim.x) {
            const int x = i % g.N1, z = i / g.N1;
            const long long gi = x + (long long)g.N1 * (y + (long long)g.N2 * z);
            pw[packed_index(x, z, g.Nh)] = S1[i] * grad[c * N + gi];
        }
        __syncthreads();
        plane_forward(plane, g, tw1, tw3);
        float2* dst = wspec + ((long long)c * g.N2 + y) * g.ncols;
        for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) dst[i] = plane[i];
    }
}

// ---------------------------------------------------------------------------
// P4: spectral divergence along pencils
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_pencil_div(float2* __restrict__ wspec, GridArgs g,
                                                    const float2* __restrict__ tw, int C) {
    extern __shared__ float2 sm[];
    const int N2 = g.N2;
    float2* lines = sm;  // [3][C][N2]
    float2* tw2 = lines + 3 * C * N2;
    load_twiddles(tw2, tw + g.N1, N2);
    const int c0 = blockIdx.x * C;
    const int tot = 3 * N2 * C;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        const int cc = i % C, r = i / C, yy = r % N2, c = r / N2;
        const int col = c0 + cc;
        float2 val = make_float2(0.f, 0.f);
        if (col < g.ncols) val = wspec[((long long)c * N2 + yy) * g.ncols + col];
        lines[(c * C + cc) * N2 + yy] = val;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int l = warp; l < 3 * C; l += nw) line_fft<false>(lines + l * N2, 1, g.p2, tw2, lane);
    __syncthreads();
    for (int pt = threadIdx.x; pt < C * N2; pt += blockDim.x) {
        const int cc = pt / N2, yy = pt % N2;
        const int col = c0 + cc;
        const int kx = col % g.Nh, kz = col / g.Nh;
        // derivative wave numbers with the Nyquist components removed
        const int mx = (2 * kx == g.N1) ? 0 : kx;
        const int my = (2 * yy == N2) ? 0 : ((2 * yy < N2) ? yy : yy - N2);
        const int mz = (2 * kz == g.N3) ? 0 : ((2 * kz < g.N3) ? kz : kz - g.N3);
        const float2 wx = lines[(0 * C + cc) * N2 + yy];
        const float2 wy = lines[(1 * C + cc) * N2 + yy];
        const float2 wz = lines[(2 * C + cc) * N2 + yy];
        const float Gx = g.gx * mx, Gy = g.gy * my, Gz = g.gz * mz;
        // i G . w / N
        const float re = Gx * wx.x + Gy * wy.x + Gz * wz.x;
        const float im = Gx * wx.y + Gy * wy.y + Gz * wz.y;
        lines[(0 * C + cc) * N2 + yy] = make_float2(-im * g.invN, re * g.invN);
    }
    __syncthreads();
    for (int l = warp; l < C; l += nw) line_fft<true>(lines + l * N2, 1, g.p2, tw2, lane);
    __syncthreads();
    for (int i = threadIdx.x; i < N2 * C; i += blockDim.x) {
        const int cc = i % C, yy = i / C;
        const int col = c0 + cc;
        if (col < g.ncols) wspec[(long long)yy * g.ncols + col] = lines[cc * N2 + yy];
    }
}

// ---------------------------------------------------------------------------
// P5: inverse plane transform of D.w, v = v_loc - D.w
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_div_final(const float2* __restrict__ wspec, GridArgs g,
                                                   const float2* __restrict__ tw, float* __restrict__ v) {
    extern __shared__ float2 sm[];
    float2* plane = sm;
    float2* tw1 = plane + g.N3 * g.Nh;
    float2* tw3 = tw1 + g.N1;
    const int y = blockIdx.x;
    load_twiddles(tw1, tw, g.N1);
    load_twiddles(tw3, tw + g.N1 + g.N2, g.N3);
    const float2* src = wspec + (long long)y * g.ncols;
    for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) plane[i] = src[i];
    __syncthreads();
    plane_inverse(plane, g, tw1, tw3);
    const float* pf = reinterpret_cast<const float*>(plane);
    const int np = g.N1 * g.N3;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int x = i % g.N1, z = i / g.N1;
        const long long gi = x + (long long)g.N1 * (y + (long long)g.N2 * z);
        v[gi] -= pf[packed_index(x, z, g.Nh)];
    }
}

// ---------------------------------------------------------------------------
// energy: fixed-order FP64 reduction of the block partials
// ---------------------------------------------------------------------------
__global__ void k_energy_final(const double* __restrict__ epart, int nb0, int nb2, double s0, double s2,
                               double* __restrict__ E) {
    __shared__ double red[32];
    double a0 = 0.0, a2 = 0.0;
    for (int i = threadIdx.x; i < nb0; i += blockDim.x) a0 += epart[i];
    for (int i = threadIdx.x; i < nb2; i += blockDim.x) a2 += epart[nb0 + i];
    const double t0 = block_sum(a0, red);
    __syncthreads();
    const double t2 = block_sum(a2, red);
    if (threadIdx.x == 0) {
        const double dE = s0 * t0, Es = s2 * t2;
        E[0] = Es + dE;
        E[1] = Es;
        E[2] = dE;
    }
}

__global__ void k_twiddles(float2* tw, int n, int off) {
    for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < n; e += blockDim.x * gridDim.x) {
        double s, c;
        sincospi(-2.0 * (double)e / (double)n, &s, &c);
        tw[off + e] = make_float2((float)c, (float)s);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int make_line_plan(int n, LinePlan* lp) {
    lp->n = n;
    int m = n;
    lp->c4 = lp->c2 = lp->c3 = lp->c5 = 0;
    while (m % 4 == 0) { m /= 4; ++lp->c4; }
    while (m % 2 == 0) { m /= 2; ++lp->c2; }
    while (m % 3 == 0) { m /= 3; ++lp->c3; }
    while (m % 5 == 0) { m /= 5; ++lp->c5; }
    return m == 1 ? VDW_OK : VDW_ERR_SIZE;
}

static size_t smem_plane(const GridArgs& g) { return sizeof(float2) * ((size_t)g.N3 * g.Nh + g.N1 + g.N3); }
static size_t smem_assemble(const GridArgs& g, bool acc_in_smem) {
    return sizeof(float2) * ((size_t)g.N3 * g.Nh + g.N1 + g.N3) +
           (acc_in_smem ? sizeof(float) * 2 * (size_t)g.N1 * g.N3 : 0);
}
static size_t smem_pencil(const GridArgs& g, int nq, int C) { return sizeof(float2) * ((size_t)nq * C * g.N2 + g.N2); }

static const size_t SMEM_MAX = 227 * 1024;

int pipeline_plan_check(vdw_ctx* c, size_t* sp, size_t* spen, size_t* sa, size_t* sd) {
    const GridArgs& g = c->g;
    const int nq = c->p.Nq;
    // columns per pencil block: as many as fit in ~110 KB (2 blocks per SM), at most 8
    int C = 8;
    while (C > 1 && smem_pencil(g, nq, C) > 110 * 1024) --C;
    c->pencil_cols = C;
    *sp = smem_plane(g);
    *spen = smem_pencil(g, nq, C);
    c->acc_global = smem_assemble(g, true) > SMEM_MAX;
    *sa = smem_assemble(g, !c->acc_global);
    *sd = smem_pencil(g, 3, 8);
    if (*sp > SMEM_MAX || *spen > SMEM_MAX || *sa > SMEM_MAX || *sd > SMEM_MAX) return VDW_ERR_SIZE;
    return VDW_OK;
}

int pipeline_make_twiddles(vdw_ctx* c) {
    const GridArgs& g = c->g;
    k_twiddles<<<4, 256>>>(c->d_tw, g.N1, 0);
    k_twiddles<<<4, 256>>>(c->d_tw, g.N2, g.N1);
    k_twiddles<<<4, 256>>>(c->d_tw, g.N3, g.N1 + g.N2);
    VDW_CUDA(cudaGetLastError());
    VDW_CUDA(cudaDeviceSynchronize());
    return VDW_OK;
}

template <int NQ>
static void launch_contract(vdw_ctx* c, cudaStream_t s, int write_back) {
    const GridArgs& g = c->g;
    const int C = c->pencil_cols;
    const size_t sm = smem_pencil(g, NQ, C);
    cudaFuncSetAttribute(k_pencil_contract<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_pencil_contract<NQ><<<c->nb_pencil, 256, sm, s>>>(c->d_spec, g, c->d_kcoef, c->d_tw,
                                                        c->d_epart + c->nb_point, C, write_back);
}

int pipeline_run(vdw_ctx* c, const float* n, const float* grad, double* E, float* v, float* w, cudaStream_t s) {
    const GridArgs& g = c->g;
    const PointParams& P = c->pp;
    const bool want_pot = (v != nullptr) || (w != nullptr);
    // stage marks for vdw_profile_read (event k+1 closes stage k)
    auto mark = [&](int stage) {
        if (c->prof) {
            cudaEventRecord(c->ev[stage + 1], s);
            c->ev_done[stage] = 1;
        }
    };
    if (c->prof) {
        for (int i = 0; i < VDW_NSTAGES; ++i) c->ev_done[i] = 0;
        cudaEventRecord(c->ev[0], s);
    }
    VDW_CUDA(cudaMemsetAsync(c->d_invalid, 0, sizeof(unsigned long long), s));
    k_pointwise<<<c->nb_point, 256, 0, s>>>(n, grad, g.N, P, c->d_t, c->d_k, c->d_epart, c->d_invalid);
    mark(0);

    const size_t sp = smem_plane(g);
    cudaFuncSetAttribute(k_theta_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp);
    k_theta_plane<<<dim3(g.N2, P.Nq), 256, sp, s>>>(n, c->d_t, c->d_k, g, P, c->d_tw, c->d_spec);
    mark(1);

    switch (P.Nq) {
        case 20: launch_contract<20>(c, s, want_pot ? 1 : 0); break;
        case 8: launch_contract<8>(c, s, want_pot ? 1 : 0); break;
        case 12: launch_contract<12>(c, s, want_pot ? 1 : 0); break;
        case 16: launch_contract<16>(c, s, want_pot ? 1 : 0); break;
        default: set_error("Nq not compiled in"); return VDW_ERR_UNSUPPORTED;
    }
    mark(2);
    if (E) {
        const double Omega = c->L[0] * c->L[1] * c->L[2];
        const double Nd = (double)g.N;
        k_energy_final<<<1, 256, 0, s>>>(c->d_epart, c->nb_point, c->nb_pencil, Omega / Nd,
                                         0.5 * Omega / (Nd * Nd), E);
        mark(3);
    }
    if (want_pot) {
        const size_t sa = smem_assemble(g, !c->acc_global);
        cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa);
        const int mode = (w != nullptr) ? 0 : 1;
        k_assemble<<<g.N2, 512, sa, s>>>(c->d_spec, n, grad, c->d_t, c->d_k, g, P, c->d_tw, v, w, c->d_wspec, mode,
                                         c->acc_global ? c->d_acc : nullptr);
        mark(4);
        if (mode == 1) {
            const int Cd = 8;
            const size_t sd = smem_pencil(g, 3, Cd);
            cudaFuncSetAttribute(k_pencil_div, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sd);
            k_pencil_div<<<(g.ncols + Cd - 1) / Cd, 256, sd, s>>>(c->d_wspec, g, c->d_tw, Cd);
            mark(5);
            cudaFuncSetAttribute(k_div_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp);
            k_div_final<<<g.N2, 256, sp, s>>>(c->d_wspec, g, c->d_tw, v);
            mark(6);
        }
    }
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

}  // namespace vdw
