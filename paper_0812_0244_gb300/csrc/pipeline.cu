// The hot path of the Roman-Perez--Soler evaluation on one GB300.
//
//   P0 k_pointwise      n, grad n -> q, mesh interval k, position t (Eq. Sat,
//                       Eq. fofx), theta_a = n p_a(q) (text after Eq. Eoffk)
//                       into packed real planes; Delta E partial sums
//                       (Eqs. DEnl, Depsnl)
//   P1 k_planes_inplace forward plane transforms of theta_a in place: R2C
//                       along x and C2C along z in shared memory
//   P2 (contract.cu)    C2C along y of all Nq fields, points written in |G|
//                       order; per G: u_a(G) = sum_b phi_ab(|G|) theta_b(G)
//                       with phi_ab from the radial table, energy of Eq.
//                       (Eoffk) in FP64; inverse C2C along y (Eqs. epsilon,
//                       epsofk)
//   P3 k_planes_inplace inverse plane transform of u_a (in place)
//      k_u_sum          Eq. (Vi) per point: v_loc and g of w = g grad n
//      k_w_planes       forward plane transform of w
//   P4 k_pencil_div     y transform of w, i G' . w(G), inverse y transform
//   P5 k_div_final      inverse plane transform, v = v_loc - D . w
//
// Layouts: real fields [N3][N2][N1] flat (x fastest); spectra
// [field][N2][N3][Nh] with Nh = N1/2+1 (a y plane of the half spectrum is one
// contiguous block, a pencil along y strides by N3 Nh).
//
// Every kernel is a template over the line lengths (CN1, CN2, CN3): the
// grids 180 x 180 x 72 and 256 x 256 x 96 get compile-time transforms, any
// other size (0) the runtime-length engine.
#include "plane.cuh"
#include "pointwise.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <string>
#include <vector>

namespace vdw {

constexpr int XC_BLOCKS = 1024;  // blocks (and partial-sum slots) of the semilocal kernel

// ---------------------------------------------------------------------------
// P0: pointwise
// ---------------------------------------------------------------------------
// q, its mesh interval k and position t per point (flat order out), theta_a
// = n p_a(q) (text after Eq. Eoffk) into the packed real rows of the
// spectrum buffer, and the Delta E partial sums.  aux (flat order) keeps
// what the assembly of Eq. (Vi) needs besides the field sums:
// {n dq/dn, n (dq/d|grad n|)/|grad n|, d(Delta eps)/dn, its grad n coefficient}.
// The grid is cut into slabs of nj complex rows (z = 2 j0 .. 2 (j0 + nj) - 1
// for slab j0 / nj), each walked in packed order within the slab: q = ((y nj
// + (j - j0)) N1 + x) 2 + s, by nbs blocks of which block b writes its
// Delta E partial sum to epart[slab nbs + b].  A launch with slab >= 0 does
// that slab alone (grid nbs); with slab < 0 the grid holds nbs blocks for
// every slab, block b doing block b mod nbs of slab b / nbs, so that both
// forms give the same partial sums.  mnj = ceil(2^32 / nj) when g.fast.
// 40 registers, six blocks of 256 threads per SM: 0.100 ms at 180 x 180 x 72
// against 0.112 ms at 64 registers and four blocks.
template <int NQ>
__global__ void __launch_bounds__(256, 6) k_pointwise(const float* __restrict__ n, const float* __restrict__ grad,
                                                   GridArgs g, PointParams P, int slab, int nj, unsigned mnj,
                                                   int nbs, float* __restrict__ t_out, uint8_t* __restrict__ k_out,
                                                   float4* __restrict__ aux, float* __restrict__ specf,
                                                   double* __restrict__ epart,
                                                   unsigned long long* __restrict__ invalid) {
    __shared__ double red[32];
    __shared__ SplineSmem sp;
    {
        // density blockIdx.y of a batch
        const long long b = blockIdx.y;
        n += b * g.N;
        grad += 3 * b * g.N;
        t_out += b * g.N;
        k_out += b * g.N;
        aux += b * g.N;
        specf += 2 * b * g.bs_spec;
        epart += b * g.bs_epart;
    }
    load_spline_smem(&sp, P);
    __syncthreads();
    const int sl = slab >= 0 ? slab : (int)blockIdx.x / nbs;
    const int lb = slab >= 0 ? (int)blockIdx.x : (int)blockIdx.x - sl * nbs;
    const int j0 = sl * nj;
    const long long N = g.N;
    const long long Nc = 2LL * g.N2 * nj * g.N1;    // points of the slab
    const long long fstride = 2LL * g.N2 * g.ncols;  // floats between the planes of two fields
    double acc = 0.0;
    unsigned int bad = 0;
    for (long long q = lb * (long long)blockDim.x + threadIdx.x; q < Nc; q += (long long)nbs * blockDim.x) {
        int y, x, jj;
        const int s = (int)(q & 1);
        if (g.fast) {
            const unsigned t = (unsigned)(q >> 1);
            const unsigned rr = __umulhi(t, g.m1);
            x = (int)(t - rr * (unsigned)g.N1);
            y = nj == 1 ? (int)rr : (int)__umulhi(rr, mnj);
            jj = (int)(rr - (unsigned)y * (unsigned)nj);
        } else {
            const long long t = q >> 1;
            const long long rr = t / g.N1;
            x = (int)(t - rr * g.N1);
            y = (int)(rr / nj);
            jj = (int)(rr - (long long)y * nj);
        }
        const int j = j0 + jj, z = 2 * j + s;
        const long long i = ((long long)z * g.N2 + y) * g.N1 + x;
        const float ni = n[i];
        bad += (!(ni >= 0.f) || !isfinite(ni)) ? 1u : 0u;
        const QPoint qp = q_point(ni, grad[i], grad[N + i], grad[2 * N + i], P, sp.qm);
        t_out[i] = qp.t;
        k_out[i] = (uint8_t)qp.k;
        float* dst = specf + 2LL * y * g.ncols + packed_offset(x, j, z & 1, g.Nh);
        if (qp.k != K_INVALID) {
            const float q = qp.q, q3 = q * q * q, q4 = q3 * q;
            acc += (double)(0.5f * P.C_s * ni * ni / q3);
            const float cn = 1.5f * P.C_s * ni * ni / q4;
            aux[i] = make_float4(ni * qp.dq_dn, ni * qp.dq_dg, P.C_s * ni / q3 - cn * qp.dq_dn, -cn * qp.dq_dg);
#pragma unroll
            for (int a = 0; a < NQ; ++a) dst[a * fstride] = ni * cardinal_value(&sp, a, qp.k, qp.t);
        } else {
            aux[i] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int a = 0; a < NQ; ++a) dst[a * fstride] = 0.f;
        }
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) epart[sl * nbs + lb] = s;
    __syncthreads();
    const double b = block_sum((double)bad, red);
    if (threadIdx.x == 0 && b > 0.0) atomicAdd(invalid, (unsigned long long)b);
}

// P1 (the forward plane transforms of theta_a) is k_planes_inplace below; P2
// (y transforms and the contraction) is in contract.cu.

// ---------------------------------------------------------------------------
// P3: inverse plane transforms of u_a, in place
// ---------------------------------------------------------------------------
// One block per (y plane, field): the plane arrives by one bulk asynchronous
// copy (completion counted on an mbarrier) while the twiddles load.
// Inverse: the plane of u_a(G) goes through the inverse z and x transforms,
// and its N3 x N1 real values (unscaled: 1/N is folded into the contraction)
// overwrite the start of the same plane of the spectrum buffer, rows of N1
// floats.  Forward: the plane holds real rows in the packed layout of the
// plane transforms (real rows 2j and 2j+1 as the real and imaginary parts of
// complex row j, rows of 2 Nh complex values) and is replaced by its half
// spectrum.
__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global memory into this block's shared memory, counted on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}
// Bounded wait for the phase of the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait_parity(uint64_t* bar, uint32_t parity) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    for (int i = 0; i < (1 << 20); ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Three blocks per SM at N1 = 180 (80 registers, a few spilled: 0.160 and
// 0.157 ms for the forward and inverse stage against 0.171 and 0.165 ms at
// two blocks); two elsewhere.
template <int CN1, int CN3, bool INV>
__global__ void __launch_bounds__(PLANE_THREADS, CN1 == 180 ? 3 : 2)
    k_planes_inplace(float2* __restrict__ spec, GridArgs g, const Tw* __restrict__ tw, int bulk,
                     int* __restrict__ wait_err) {
    extern __shared__ float2 sm[];
    __shared__ uint64_t bar;
    float2* plane = sm;
    // the forward transforms of theta feed the energy: hi/lo twiddles there
    using W = TwOf<!INV>;
    W* tw1 = twiddles_after<W>(plane, (size_t)(g.N3 * g.Nh));
    W* tw3 = tw1 + g.N1;
    const int y = blockIdx.x, a = blockIdx.y;
    float2* src = spec + blockIdx.z * g.bs_spec + ((long long)a * g.N2 + y) * g.ncols;
    // bulk: one copy of the whole plane (16-byte aligned, a multiple of 16
    // bytes), in flight while the twiddles load
    if (bulk) {
        if (threadIdx.x == 0) mbar_init1(&bar);
        __syncthreads();
        if (threadIdx.x == 0) bulk_load(plane, src, (uint32_t)(sizeof(float2) * (size_t)g.ncols), &bar);
    } else {
        for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) plane[i] = src[i];
    }
    load_line_twiddles<CN1>(tw1, tw, g.N1);
    load_line_twiddles<CN3>(tw3, tw + g.N1 + g.N2, g.N3);
    __syncthreads();
    const bool got = !bulk || mbar_wait_parity(&bar, 0u);
    if (__syncthreads_or(!got)) {
        // a wait gave up: record it for the next entry point, give the copy in
        // flight (it writes this block's shared memory) a second bounded wait,
        // and leave the plane as it is rather than transform a partial one
        if (threadIdx.x == 0) {
            *(volatile int*)wait_err = 1;
            __threadfence_system();
        }
        mbar_wait_parity(&bar, 0u);
        return;
    }
    if constexpr (INV) {
        plane_inverse<CN1, CN3>(plane, g, tw1, tw3);
        float* dst = reinterpret_cast<float*>(src);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        // complex row jr holds real rows 2 jr (real parts) and 2 jr + 1 (imaginary parts)
        for (int jr = warp; jr < (g.N3 >> 1); jr += nw) {
            const float2* crow = plane + jr * 2 * g.Nh;
            float* d0 = dst + 2 * jr * g.N1;
            for (int x = lane; x < g.N1; x += 32) {
                const float2 u = crow[x];
                d0[x] = u.x;
                d0[g.N1 + x] = u.y;
            }
        }
    } else {
        plane_forward<CN1, CN3>(plane, g, tw1, tw3);
        for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) src[i] = plane[i];
    }
}

// ---------------------------------------------------------------------------
// P3': the assembly of Eq. (Vi), one thread per point
// ---------------------------------------------------------------------------
// S0 = sum_a u_a p_a(q), S1 = sum_a u_a p_a'(q) from the real u_a planes left
// in the spectrum buffer by the inverse k_planes_inplace.  On interval k with
// A = 1 - t, B = t, p_a = A d_ak + B d_a,k+1 + [(A^3 - A) M_ak + (B^3 - B)
// M_a,k+1] h^2/6 is linear in the second derivatives M, so both sums need
// only u_k, u_k+1 and the two dot products m0 = sum_a u_a M_ak, m1 = sum_a
// u_a M_a,k+1.  Then, with aux from the pointwise pass,
//   v_loc = S0 + S1 n dq/dn + d(Delta eps)/dn,   g = S1 n dq/d|grad n| / |grad n| + ...
// mode 0: v_loc to v (if v), w = g grad n to w_out; mode 1: v_loc to v, g to
// g_out (the plane transforms of w follow in k_w_planes).
constexpr int USUM_THREADS = 256;

template <int NQ>
__global__ void __launch_bounds__(USUM_THREADS) k_u_sum(const float* __restrict__ uf, const float* __restrict__ grad,
                                                        const float* __restrict__ tk, const uint8_t* __restrict__ kk,
                                                        const float4* __restrict__ aux, GridArgs g, PointParams P,
                                                        float* __restrict__ v, float* __restrict__ w_out,
                                                        float* __restrict__ g_out, int mode) {
    __shared__ SplineSmem sp;
    {
        // density blockIdx.y of a batch
        const long long b = blockIdx.y;
        uf += 2 * b * g.bs_spec;
        grad += 3 * b * g.N;
        tk += b * g.N;
        kk += b * g.N;
        aux += b * g.N;
        if (v) v += b * g.N;
        if (w_out) w_out += 3 * b * g.N;
        if (g_out) g_out += b * g.N;
    }
    load_spline_smem(&sp, P);
    __syncthreads();
    const long long N = g.N;
    const long long fstride = 2LL * g.N2 * g.ncols;  // floats between the planes of two fields
    const int N1 = g.N1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        flat_point(i, g, x, y, z);
        const float* up = uf + 2LL * y * g.ncols + (long long)z * N1 + x;
        const int k = kk[i];
        float vl = 0.f, gg = 0.f;
        if (k != K_INVALID) {
            float u[NQ];
#pragma unroll
            for (int a = 0; a < NQ; ++a) u[a] = up[a * fstride];
            const float t = tk[i];
            const float4 ax = aux[i];
            float uk = 0.f, uk1 = 0.f, m0 = 0.f, m1 = 0.f;
#pragma unroll
            for (int a = 0; a < NQ; ++a) {
                m0 = fmaf(u[a], sp.Mq[a * MAX_NQ + k], m0);
                m1 = fmaf(u[a], sp.Mq[a * MAX_NQ + k + 1], m1);
                uk = (a == k) ? u[a] : uk;
                uk1 = (a == k + 1) ? u[a] : uk1;
            }
            const float A = 1.f - t, B = t;
            const float s0 = A * uk + B * uk1 + ((A * A * A - A) * m0 + (B * B * B - B) * m1) * sp.h26[k];
            const float s1 = (uk1 - uk) * sp.ih[k] + ((3.f * B * B - 1.f) * m1 - (3.f * A * A - 1.f) * m0) * sp.h6[k];
            vl = s0 + ax.x * s1 + ax.z;
            gg = ax.y * s1 + ax.w;
        }
        if (v) v[i] = vl;
        if (mode == 0 && w_out) {
            w_out[i] = gg * grad[i];
            w_out[N + i] = gg * grad[N + i];
            w_out[2 * N + i] = gg * grad[2 * N + i];
        }
        if (mode == 1) g_out[i] = gg;
    }
}

// ---------------------------------------------------------------------------
// P3b: forward plane transforms of the three components of w = g grad n
// ---------------------------------------------------------------------------
template <int CN1, int CN3>
__global__ void __launch_bounds__(PLANE_THREADS, 2) k_w_planes(const float* __restrict__ gfield,
                                                                const float* __restrict__ grad, GridArgs g,
                                                                const Tw* __restrict__ tw,
                                                                float2* __restrict__ wspec) {
    extern __shared__ float2 sm[];
    float2* plane = sm;
    float2* tw1 = twiddles_after<float2>(plane, (size_t)(g.N3 * g.Nh));
    float2* tw3 = tw1 + g.N1;
    const int y = blockIdx.x, c = blockIdx.y;
    gfield += blockIdx.z * g.N;  // density blockIdx.z of a batch
    grad += 3 * blockIdx.z * g.N;
    wspec += blockIdx.z * g.bs_wspec;
    load_line_twiddles<CN1>(tw1, tw, g.N1);
    load_line_twiddles<CN3>(tw3, tw + g.N1 + g.N2, g.N3);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float* gc = grad + c * g.N;
    const long long zs = (long long)g.N1 * g.N2;  // flat distance between rows z and z + 1
    for (int jr = warp; jr < (g.N3 >> 1); jr += nw) {
        const long long row = (long long)g.N1 * (y + (long long)g.N2 * 2 * jr);
        float2* crow = plane + jr * 2 * g.Nh;
        for (int x = lane; x < g.N1; x += 32)
            crow[x] = make_float2(gfield[row + x] * gc[row + x], gfield[row + zs + x] * gc[row + zs + x]);
    }
    __syncthreads();
    plane_forward<CN1, CN3>(plane, g, tw1, tw3);
    float2* dst = wspec + ((long long)c * g.N2 + y) * g.ncols;
    for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) dst[i] = plane[i];
}

// ---------------------------------------------------------------------------
// P4: spectral divergence along pencils
// ---------------------------------------------------------------------------
constexpr int DIV_COLS_CT = 8;  // columns per divergence block

template <int CN2>
__global__ void __launch_bounds__(256, 2) k_pencil_div(float2* __restrict__ wspec, GridArgs g,
                                                       const Tw* __restrict__ tw, int C) {
    extern __shared__ float2 sm[];
    const int N2 = CN2 > 0 ? CN2 : g.N2;
    const int S = pencil_stride(N2);
    float2* lines = sm;  // [3][C][S]
    float2* tw2 = twiddles_after<float2>(lines, (size_t)(3 * C * S));
    wspec += blockIdx.y * g.bs_wspec;  // density blockIdx.y of a batch
    load_line_twiddles<CN2>(tw2, tw + g.N1, N2);
    const int c0 = blockIdx.x * C;
    const SmallDiv sC = small_div(C);  // i / C in the staging loops
    const int tot = 3 * N2 * C;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        const int r = sdiv(i, sC), cc = i - r * C, yy = r % N2, c = r / N2;
        const int col = c0 + cc;
        const bool ok = col < g.ncols;
        cp_async8(lines + (c * C + cc) * S + yy, ok ? wspec + ((long long)c * N2 + yy) * g.ncols + col : wspec, ok);
    }
    cp_async_wait_all();
    __syncthreads();
    pencils_fft<CN2, false>(lines, 3 * C, N2, g.p2, tw2, S);
    __syncthreads();
    for (int pt = threadIdx.x; pt < C * N2; pt += blockDim.x) {
        const int cc = pt / N2, yy = pt % N2;
        const int col = c0 + cc;
        if (col >= g.ncols) continue;
        const int kx = col % g.Nh, kz = col / g.Nh;
        // derivative wave numbers with the Nyquist components removed
        const int mx = (2 * kx == g.N1) ? 0 : kx;
        const int my = (2 * yy == N2) ? 0 : ((2 * yy < N2) ? yy : yy - N2);
        const int mz = (2 * kz == g.N3) ? 0 : ((2 * kz < g.N3) ? kz : kz - g.N3);
        const float2 wx = lines[(0 * C + cc) * S + yy];
        const float2 wy = lines[(1 * C + cc) * S + yy];
        const float2 wz = lines[(2 * C + cc) * S + yy];
        const float Gx = g.gx * mx, Gy = g.gy * my, Gz = g.gz * mz;
        // i G . w / N
        const float re = Gx * wx.x + Gy * wy.x + Gz * wz.x;
        const float im = Gx * wx.y + Gy * wy.y + Gz * wz.y;
        lines[(0 * C + cc) * S + yy] = make_float2(-im * g.invN, re * g.invN);
    }
    __syncthreads();
    pencils_fft<CN2, true>(lines, C, N2, g.p2, tw2, S);
    __syncthreads();
    for (int i = threadIdx.x; i < N2 * C; i += blockDim.x) {
        const int yy = sdiv(i, sC), cc = i - yy * C;
        const int col = c0 + cc;
        if (col < g.ncols) wspec[(long long)yy * g.ncols + col] = lines[cc * S + yy];
    }
}

// ---------------------------------------------------------------------------
// P5: inverse plane transform of D.w, v = v_loc - D.w
// ---------------------------------------------------------------------------
template <int CN1, int CN3>
__global__ void __launch_bounds__(PLANE_THREADS, 2) k_div_final(const float2* __restrict__ wspec, GridArgs g,
                                                      const Tw* __restrict__ tw, float* __restrict__ v) {
    extern __shared__ float2 sm[];
    float2* plane = sm;
    float2* tw1 = twiddles_after<float2>(plane, (size_t)(g.N3 * g.Nh));
    float2* tw3 = tw1 + g.N1;
    const int y = blockIdx.x;
    wspec += blockIdx.y * g.bs_wspec;  // density blockIdx.y of a batch
    v += blockIdx.y * g.N;
    load_line_twiddles<CN1>(tw1, tw, g.N1);
    load_line_twiddles<CN3>(tw3, tw + g.N1 + g.N2, g.N3);
    const float2* src = wspec + (long long)y * g.ncols;
    for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) plane[i] = src[i];
    __syncthreads();
    plane_inverse<CN1, CN3>(plane, g, tw1, tw3);
    const float* pf = reinterpret_cast<const float*>(plane);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // real row z: component z & 1 of complex row z / 2 (one row per warp: the
    // read-modify-write of v keeps more rows in flight this way than by pairs)
    for (int z = warp; z < g.N3; z += nw) {
        const long long row = (long long)g.N1 * (y + (long long)g.N2 * z);
        const float* srow = pf + 2 * ((z >> 1) * 2 * g.Nh) + (z & 1);
        for (int x = lane; x < g.N1; x += 32) v[row + x] -= srow[2 * x];
    }
}

// ---------------------------------------------------------------------------
// finite-difference gradient (the paper's own): central differences on the
// periodic grid, and the chain term of Eq. (Vi) as the transposed stencil
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_stencil_gradient(const float* __restrict__ f, GridArgs g, float3 ih2,
                                                          float* __restrict__ grad) {
    const long long N = g.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        flat_point(i, g, x, y, z);
        const long long rowz = (long long)z * g.N2;
        const long long xm = i - x + (x == 0 ? g.N1 - 1 : x - 1), xp = i - x + (x == g.N1 - 1 ? 0 : x + 1);
        const long long ym = ((rowz + (y == 0 ? g.N2 - 1 : y - 1)) * g.N1) + x;
        const long long yp = ((rowz + (y == g.N2 - 1 ? 0 : y + 1)) * g.N1) + x;
        const long long zm = (((long long)(z == 0 ? g.N3 - 1 : z - 1) * g.N2 + y) * g.N1) + x;
        const long long zp = (((long long)(z == g.N3 - 1 ? 0 : z + 1) * g.N2 + y) * g.N1) + x;
        grad[i] = (f[xp] - f[xm]) * ih2.x;
        grad[N + i] = (f[yp] - f[ym]) * ih2.y;
        grad[2 * N + i] = (f[zp] - f[zm]) * ih2.z;
    }
}

// v -= sum_c D_c (g grad_c n): with the antisymmetric central-difference D,
// D^T w = -D w (w = g grad n, g from the assembly)
__global__ void __launch_bounds__(256) k_stencil_div_sub(const float* __restrict__ gg, const float* __restrict__ grad,
                                                         GridArgs g, float3 ih2, float* __restrict__ v) {
    const long long N = g.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        flat_point(i, g, x, y, z);
        const long long rowz = (long long)z * g.N2;
        const long long xm = i - x + (x == 0 ? g.N1 - 1 : x - 1), xp = i - x + (x == g.N1 - 1 ? 0 : x + 1);
        const long long ym = ((rowz + (y == 0 ? g.N2 - 1 : y - 1)) * g.N1) + x;
        const long long yp = ((rowz + (y == g.N2 - 1 ? 0 : y + 1)) * g.N1) + x;
        const long long zm = (((long long)(z == 0 ? g.N3 - 1 : z - 1) * g.N2 + y) * g.N1) + x;
        const long long zp = (((long long)(z == g.N3 - 1 ? 0 : z + 1) * g.N2 + y) * g.N1) + x;
        const float d = (gg[xp] * grad[xp] - gg[xm] * grad[xm]) * ih2.x +
                        (gg[yp] * grad[N + yp] - gg[ym] * grad[N + ym]) * ih2.y +
                        (gg[zp] * grad[2 * N + zp] - gg[zm] * grad[2 * N + zm]) * ih2.z;
        v[i] -= d;
    }
}

// ---------------------------------------------------------------------------
// semilocal partner terms of Eq. (Exc): revPBE exchange (kappa = 1.245,
// mu = 0.066725 pi^2/3) and LDA correlation (the PW92 eps_c of q0)
// ---------------------------------------------------------------------------
// Adds de/dn to v and the coefficient of grad n in de/d(grad n) to g (so that
// the divergence stage takes it with the nonlocal w); FP64 block sums of
// e_x and e_c into epart[block] and epart[nb + block].
__global__ void __launch_bounds__(256) k_semilocal(const float* __restrict__ n, const float* __restrict__ grad,
                                                   long long N, float n_min, float* __restrict__ v,
                                                   float* __restrict__ gg, double* __restrict__ epart) {
    __shared__ double red[32];
    const float PI_F = 3.14159265358979f;
    const float KAPPA = 1.245f, MU = 0.066725f * PI_F * PI_F / 3.f;
    const float AX = -0.75f * 0.98474502184269641f;  // -(3/4) (3/pi)^(1/3)
    const float A = 0.031091f, a1 = 0.21370f;
    const float b1 = 7.5957f, b2 = 3.5876f, b3 = 1.6382f, b4 = 0.49294f;
    double sx = 0.0, sc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float ni = n[i];
        if (!(ni > n_min) || !isfinite(ni)) continue;
        const float gx = grad[i], gy = grad[N + i], gz = grad[2 * N + i];
        const float cb = cbrtf(ni);
        const float kF = cbrtf(3.f * PI_F * PI_F) * cb;
        const float inv_n = 1.f / ni;
        const float s2 = (gx * gx + gy * gy + gz * gz) * (0.25f * inv_n * inv_n) / (kF * kF);
        const float den = 1.f + MU * s2 / KAPPA;
        const float Fx = 1.f + KAPPA - KAPPA / den;
        const float dF = MU / (den * den);
        const float e0 = AX * ni * cb;
        const float ex = e0 * Fx;
        const float dex = (4.f / 3.f) * AX * cb * Fx + e0 * dF * (-(8.f / 3.f) * s2 * inv_n);
        const float gex = e0 * dF * 2.f * (0.25f * inv_n * inv_n) / (kF * kF);
        const float rs = cbrtf(3.f / (4.f * PI_F * ni));
        const float srs = sqrtf(rs);
        const float Q = 2.f * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
        const float dQ = 2.f * A * (0.5f * b1 / srs + b2 + 1.5f * b3 * srs + 2.f * b4 * rs);
        const float Lg = log1pf(1.f / Q);
        const float ec = -2.f * A * (1.f + a1 * rs) * Lg;
        const float dec = -2.f * A * a1 * Lg + 2.f * A * (1.f + a1 * rs) * dQ / (Q * Q + Q);
        if (v) v[i] += dex + ec + ni * dec * (-rs * inv_n * (1.f / 3.f));
        if (gg) gg[i] += gex;
        sx += (double)ex;
        sc += (double)(ni * ec);
    }
    const double tx = block_sum(sx, red);
    __syncthreads();
    const double tcs = block_sum(sc, red);
    if (threadIdx.x == 0) {
        epart[blockIdx.x] = tx;
        epart[gridDim.x + blockIdx.x] = tcs;
    }
}

// E[4] = {E_xc, E_c^nl, E_x, E_c^LDA} from the nonlocal E[0] and the partials
__global__ void k_xc_final(const double* __restrict__ Enl, const double* __restrict__ epart, int nb, double dOmega,
                           double* __restrict__ E) {
    __shared__ double red[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += epart[i];
        b += epart[nb + i];
    }
    const double ta = block_sum(a, red);
    __syncthreads();
    const double tb = block_sum(b, red);
    if (threadIdx.x == 0) {
        const double Ex = dOmega * ta, Ec = dOmega * tb;
        E[0] = Enl[0] + Ex + Ec;
        E[1] = Enl[0];
        E[2] = Ex;
        E[3] = Ec;
    }
}

// ---------------------------------------------------------------------------
// energy: fixed-order FP64 reduction of the block partials, in two passes
// (the GPU's FP64 rate is low: one block summing all partials took 17 us)
// ---------------------------------------------------------------------------
constexpr int ESPLIT_THREADS = 256;

// First pass: block b of density blockIdx.y sums the share
// [b n / EPART_SPLIT, (b + 1) n / EPART_SPLIT) of each partial-sum array.
__global__ void __launch_bounds__(ESPLIT_THREADS) k_energy_split(const double* __restrict__ epart, int nb0, int nb2,
                                                                 double* __restrict__ escr, int bs_epart) {
    __shared__ double red[32];
    epart += (long long)blockIdx.y * bs_epart;  // density blockIdx.y of a batch
    escr += (long long)blockIdx.y * bs_epart;
    const long long b = blockIdx.x;
    const int lo0 = (int)(b * nb0 / EPART_SPLIT), hi0 = (int)((b + 1) * nb0 / EPART_SPLIT);
    const int lo2 = (int)(b * nb2 / EPART_SPLIT), hi2 = (int)((b + 1) * nb2 / EPART_SPLIT);
    double a0 = 0.0, a2 = 0.0;
    for (int i = lo0 + threadIdx.x; i < hi0; i += blockDim.x) a0 += epart[i];
    for (int i = lo2 + threadIdx.x; i < hi2; i += blockDim.x) a2 += epart[nb0 + i];
    const double t0 = block_sum(a0, red);
    __syncthreads();
    const double t2 = block_sum(a2, red);
    if (threadIdx.x == 0) {
        escr[b] = t0;
        escr[EPART_SPLIT + b] = t2;
    }
}

// Second pass (EPART_SPLIT threads per density): the shares in index order,
// scaled into {E, E_soft, Delta E}.
__global__ void __launch_bounds__(EPART_SPLIT) k_energy_final(const double* __restrict__ escr, double s0, double s2,
                                                              double* __restrict__ E, int bs_epart) {
    __shared__ double red[32];
    escr += (long long)blockIdx.x * bs_epart;  // density blockIdx.x of a batch
    E += 3 * blockIdx.x;
    const double t0 = block_sum(escr[threadIdx.x], red);
    __syncthreads();
    const double t2 = block_sum(escr[EPART_SPLIT + threadIdx.x], red);
    if (threadIdx.x == 0) {
        const double dE = s0 * t0, Es = s2 * t2;
        E[0] = Es + dE;
        E[1] = Es;
        E[2] = dE;
    }
}

// W_n^e = exp(-2 pi i e / n) in FP64, stored as the hi/lo FP32 pair of each part
__global__ void k_twiddles(Tw* tw, int n, int off) {
    for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < n; e += blockDim.x * gridDim.x) {
        double s, c;
        sincospi(-2.0 * (double)e / (double)n, &s, &c);
        const float ch = (float)c, sh = (float)s;
        tw[off + e] = make_float4(ch, sh, (float)(c - (double)ch), (float)(s - (double)sh));
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

static size_t smem_plane(const GridArgs& g) {
    return sizeof(float2) * tw_offset((size_t)g.N3 * g.Nh) + sizeof(Tw) * (g.N1 + g.N3);
}
static size_t smem_pencil(const GridArgs& g, int nq, int C) {
    return sizeof(float2) * tw_offset((size_t)nq * C * pencil_stride(g.N2)) + sizeof(Tw) * g.N2;
}
static size_t smem_pencil_run(const GridArgs& g, int nq, int C) { return smem_pencil(g, nq, C); }

// dynamic shared memory per block, leaving room for the kernels' static arrays
static const size_t SMEM_MAX = 227 * 1024 - 5 * 1024;
static const int DIV_COLS = DIV_COLS_CT;

int pipeline_plan_check(vdw_ctx* c, size_t* sp, size_t* spen, size_t* sa, size_t* sd) {
    const GridArgs& g = c->g;
    *sp = smem_plane(g);
    *spen = sorted_pencil_smem(g);
    // the inverse plane transforms of u take their planes by one bulk copy when
    // a plane is a whole multiple of 16 bytes (every plane then starts 16-byte aligned)
    c->bulk_planes = (sizeof(float2) * (size_t)g.ncols) % 16 == 0;
    *sa = *sp;
    *sd = smem_pencil_run(g, 3, DIV_COLS);
    if (*sp > SMEM_MAX || *spen > SMEM_MAX || *sd > SMEM_MAX)
        return VDW_ERR_SIZE;
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

static float3 stencil_ih2(const vdw_ctx* c) {
    return make_float3((float)(c->g.N1 / (2.0 * c->L[0])), (float)(c->g.N2 / (2.0 * c->L[1])),
                       (float)(c->g.N3 / (2.0 * c->L[2])));
}
static int stencil_blocks(const GridArgs& g) { return (int)std::min<long long>((g.N + 255) / 256, 8192); }

int pipeline_stencil_gradient(vdw_ctx* c, const float* f, float* grad, cudaStream_t s) {
    k_stencil_gradient<<<stencil_blocks(c->g), 256, 0, s>>>(f, c->g, stencil_ih2(c), grad);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

// one wave of resident blocks, each thread striding over several points: the
// spline table is staged once per block
static int u_sum_blocks(const vdw_ctx* c) {
    const GridArgs& g = c->g;
    return (int)std::min<long long>((g.N + USUM_THREADS - 1) / USUM_THREADS,
                                    (long long)std::max(c->usum_per_sm, 1) * std::max(c->nsm, 1));
}

static int launch_u_sum(vdw_ctx* c, const float* n, const float* grad, float* v, float* w, int mode, cudaStream_t s,
                        int B) {
    const GridArgs& g = c->g;
    const float* uf = reinterpret_cast<const float*>(c->d_spec);
    const int nb = u_sum_blocks(c);
#define VDW_U_SUM(NQ) \
    k_u_sum<NQ><<<dim3(nb, B), USUM_THREADS, 0, s>>>(uf, grad, c->d_t, c->d_k, c->d_aux, g, c->pp, v, w, c->d_gg, mode)
    switch (c->pp.Nq) {
        case 20: VDW_U_SUM(20); break;
        case 8: VDW_U_SUM(8); break;
        case 12: VDW_U_SUM(12); break;
        case 16: VDW_U_SUM(16); break;
        default: set_error("Nq not compiled in"); return VDW_ERR_UNSUPPORTED;
    }
#undef VDW_U_SUM
    return VDW_OK;
}

template <int CN1, int CN2, int CN3>
static int run_sized(vdw_ctx* c, const float* n, const float* grad, double* E, float* v, float* w, cudaStream_t s,
                     int fd, int xc, const cudaEvent_t* slab_ready, int B) {
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
    float* specf = reinterpret_cast<float*>(c->d_spec);
    // one launch over all slabs, or (host entry point) one per slab as its inputs arrive
    const int nlaunch = slab_ready ? c->p0_chunks : 1;
    for (int sl = 0; sl < nlaunch; ++sl) {
        if (slab_ready) VDW_CUDA(cudaStreamWaitEvent(s, slab_ready[sl], 0));
        const int slab = slab_ready ? sl : -1;
        const int nblk = slab_ready ? c->nb_p0 : c->nb_point;
#define VDW_POINTWISE(NQ)                                                                                  \
    k_pointwise<NQ><<<dim3(nblk, B), 256, 0, s>>>(n, grad, g, P, slab, c->p0_nj, c->p0_mnj, c->nb_p0, c->d_t, c->d_k, \
                                         c->d_aux, specf, c->d_epart, c->d_invalid)
        switch (P.Nq) {
            case 20: VDW_POINTWISE(20); break;
            case 8: VDW_POINTWISE(8); break;
            case 12: VDW_POINTWISE(12); break;
            case 16: VDW_POINTWISE(16); break;
            default: set_error("Nq not compiled in"); return VDW_ERR_UNSUPPORTED;
        }
#undef VDW_POINTWISE
    }
    mark(ST_POINTWISE);

    const size_t sp = smem_plane(g);
    k_planes_inplace<CN1, CN3, false><<<dim3(g.N2, P.Nq, B), PLANE_THREADS, sp, s>>>(c->d_spec, g, c->d_tw,
                                                                                     c->bulk_planes, c->d_flags);
    mark(ST_PLANES_FWD);

    // y transforms, contraction in |G| order, inverse y transforms (contract.cu)
    int rc = sorted_forward(c, P.Nq, s, B);
    if (rc) return rc;
    mark(ST_PENCILS_FWD);
    rc = sorted_contract(c, c->d_epart + c->nb_point, want_pot ? 1 : 0, s, B);
    if (rc) return rc;
    mark(ST_CONTRACT);
    // With a potential to follow (and no stage timing), the energy reduction
    // runs on the context's side stream beside the inverse transforms, which
    // do not touch the partial sums; the caller's stream waits for it before
    // the call returns (so the next call's partial sums come after it).
    bool forked = false;
    auto join = [&]() {
        if (forked) cudaStreamWaitEvent(s, c->ev_join, 0);
        forked = false;
    };
    if (E) {
        const double Omega = c->L[0] * c->L[1] * c->L[2];
        const double Nd = (double)g.N;
        double* escr = c->d_epart + c->nb_point + c->nb_sorted;
        cudaStream_t se = s;
        if (want_pot && !c->prof) {
            VDW_CUDA(cudaEventRecord(c->ev_fork, s));
            VDW_CUDA(cudaStreamWaitEvent(c->s_side, c->ev_fork, 0));
            se = c->s_side;
        }
        k_energy_split<<<dim3(EPART_SPLIT, B), ESPLIT_THREADS, 0, se>>>(c->d_epart, c->nb_point, c->nb_sorted, escr,
                                                                        g.bs_epart);
        k_energy_final<<<B, EPART_SPLIT, 0, se>>>(escr, Omega / Nd, 0.5 * Omega / (Nd * Nd), E, g.bs_epart);
        if (se != s) {
            VDW_CUDA(cudaEventRecord(c->ev_join, se));
            forked = true;
        }
        mark(ST_ENERGY);
    }
    if (xc && !want_pot)
        k_semilocal<<<XC_BLOCKS, 256, 0, s>>>(n, grad, g.N, P.n_min, nullptr, nullptr, c->d_xc + 4);
    if (want_pot) {
        rc = sorted_inverse(c, P.Nq, s, B);
        if (rc) {
            join();
            return rc;
        }
        mark(ST_PENCILS_INV);
        const int mode = (w != nullptr) ? 0 : 1;
        k_planes_inplace<CN1, CN3, true><<<dim3(g.N2, P.Nq, B), PLANE_THREADS, sp, s>>>(c->d_spec, g, c->d_tw,
                                                                                        c->bulk_planes, c->d_flags);
        mark(ST_PLANES_INV);
        const int rcs = launch_u_sum(c, n, grad, v, w, mode, s, B);
        if (rcs) {
            join();
            return rcs;
        }
        if (xc)
            k_semilocal<<<XC_BLOCKS, 256, 0, s>>>(n, grad, g.N, P.n_min, v, mode == 1 ? c->d_gg : nullptr,
                                                  c->d_xc + 4);
        mark(ST_USUM);
        if (mode == 1 && fd) {
            // finite-difference gradient: the chain term is a stencil, no transforms
            k_stencil_div_sub<<<stencil_blocks(g), 256, 0, s>>>(c->d_gg, grad, g, stencil_ih2(c), v);
            mark(ST_DIV_FINAL);
        } else if (mode == 1) {
            k_w_planes<CN1, CN3><<<dim3(g.N2, 3, B), PLANE_THREADS, sp, s>>>(c->d_gg, grad, g, c->d_tw, c->d_wspec);
            mark(ST_W_PLANES);
            const size_t sd = smem_pencil_run(g, 3, DIV_COLS);
            k_pencil_div<CN2><<<dim3((g.ncols + DIV_COLS - 1) / DIV_COLS, B), 256, sd, s>>>(c->d_wspec, g, c->d_tw,
                                                                                          DIV_COLS);
            mark(ST_PENCIL_DIV);
            k_div_final<CN1, CN3><<<dim3(g.N2, B), PLANE_THREADS, sp, s>>>(c->d_wspec, g, c->d_tw, v);
            mark(ST_DIV_FINAL);
        }
    }
    join();
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

// Dynamic shared-memory limits of the kernels a plan uses (set once per plan).
// Sets a kernel's dynamic shared-memory limit and checks that the block size
// it will be launched with fits its register use.
template <class K>
static int set_and_check(K kernel, const char* name, int smem, int threads) {
    if (const int rs = raise_smem_limit(kernel, (size_t)smem)) return rs;
    cudaFuncAttributes fa;
    VDW_CUDA(cudaFuncGetAttributes(&fa, kernel));
    if (fa.maxThreadsPerBlock < threads) {
        set_error(std::string(name) + ": " + std::to_string(threads) + " threads requested, " +
                  std::to_string(fa.maxThreadsPerBlock) + " possible with " + std::to_string(fa.numRegs) +
                  " registers");
        return VDW_ERR_UNSUPPORTED;
    }
    return VDW_OK;
}

template <int CN1, int CN2, int CN3>
static int configure_sized(vdw_ctx* c) {
    const GridArgs& g = c->g;
    const int sp = (int)smem_plane(g);
    const int sd = (int)smem_pencil_run(g, 3, DIV_COLS);
    int rc = set_and_check(k_planes_inplace<CN1, CN3, true>, "k_planes_inplace", sp, PLANE_THREADS);
    if (!rc) rc = set_and_check(k_planes_inplace<CN1, CN3, false>, "k_planes_inplace", sp, PLANE_THREADS);
    if (!rc) rc = set_and_check(k_pencil_div<CN2>, "k_pencil_div", sd, 256);
    if (!rc) rc = set_and_check(k_div_final<CN1, CN3>, "k_div_final", sp, PLANE_THREADS);
    if (!rc) rc = set_and_check(k_w_planes<CN1, CN3>, "k_w_planes", sp, PLANE_THREADS);
    if (rc) return rc;
    rc = sorted_configure(c);
    if (rc) return rc;
    // resident blocks per SM of the field sum (its grid is one wave of them)
    int per_sm = 0;
    switch (c->p.Nq) {
        case 20: VDW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_u_sum<20>, USUM_THREADS, 0)); break;
        case 16: VDW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_u_sum<16>, USUM_THREADS, 0)); break;
        case 12: VDW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_u_sum<12>, USUM_THREADS, 0)); break;
        default: VDW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_u_sum<8>, USUM_THREADS, 0));
    }
    c->usum_per_sm = per_sm;
    return VDW_OK;
}

int pipeline_configure(vdw_ctx* c) {
    const GridArgs& g = c->g;
    if (g.N1 == 180 && g.N2 == 180 && g.N3 == 72) return configure_sized<180, 180, 72>(c);
    if (g.N1 == 256 && g.N2 == 256 && g.N3 == 96) return configure_sized<256, 256, 96>(c);
    return configure_sized<0, 0, 0>(c);
}

template <int CN1, int CN2, int CN3>
static void launch_divergence(vdw_ctx* c, float* v, cudaStream_t s) {
    const GridArgs& g = c->g;
    const size_t sd = smem_pencil_run(g, 3, DIV_COLS);
    k_pencil_div<CN2><<<(g.ncols + DIV_COLS - 1) / DIV_COLS, 256, sd, s>>>(c->d_wspec, g, c->d_tw, DIV_COLS);
    k_div_final<CN1, CN3><<<g.N2, PLANE_THREADS, smem_plane(g), s>>>(c->d_wspec, g, c->d_tw, v);
}

template <int CN1, int CN3>
static void launch_w_planes(vdw_ctx* c, const float* grad, cudaStream_t s) {
    const GridArgs& g = c->g;
    k_w_planes<CN1, CN3><<<dim3(g.N2, 3), PLANE_THREADS, smem_plane(g), s>>>(c->d_gg, grad, g, c->d_tw, c->d_wspec);
}

int pipeline_w_planes(vdw_ctx* c, const float* grad, cudaStream_t s) {
    const GridArgs& g = c->g;
    if (g.N1 == 180 && g.N2 == 180 && g.N3 == 72) launch_w_planes<180, 72>(c, grad, s);
    else if (g.N1 == 256 && g.N2 == 256 && g.N3 == 96) launch_w_planes<256, 96>(c, grad, s);
    else launch_w_planes<0, 0>(c, grad, s);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

template <int CN1, int CN3>
static void launch_planes_inplace(vdw_ctx* c, int nfields, bool inverse, cudaStream_t s) {
    const GridArgs& g = c->g;
    if (inverse)
        k_planes_inplace<CN1, CN3, true><<<dim3(g.N2, nfields), PLANE_THREADS, smem_plane(g), s>>>(
            c->d_spec, g, c->d_tw, c->bulk_planes, c->d_flags);
    else
        k_planes_inplace<CN1, CN3, false><<<dim3(g.N2, nfields), PLANE_THREADS, smem_plane(g), s>>>(
            c->d_spec, g, c->d_tw, c->bulk_planes, c->d_flags);
}

int pipeline_planes_inplace(vdw_ctx* c, int nfields, bool inverse, cudaStream_t s) {
    const GridArgs& g = c->g;
    if (g.N1 == 180 && g.N2 == 180 && g.N3 == 72) launch_planes_inplace<180, 72>(c, nfields, inverse, s);
    else if (g.N1 == 256 && g.N2 == 256 && g.N3 == 96) launch_planes_inplace<256, 96>(c, nfields, inverse, s);
    else launch_planes_inplace<0, 0>(c, nfields, inverse, s);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int pipeline_divergence(vdw_ctx* c, float* v, cudaStream_t s) {
    const GridArgs& g = c->g;
    if (g.N1 == 180 && g.N2 == 180 && g.N3 == 72) launch_divergence<180, 180, 72>(c, v, s);
    else if (g.N1 == 256 && g.N2 == 256 && g.N3 == 96) launch_divergence<256, 256, 96>(c, v, s);
    else launch_divergence<0, 0, 0>(c, v, s);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int pipeline_energy_final(vdw_ctx* c, const double* epart, int nb0, int nb2, double* E, cudaStream_t s) {
    const double Omega = c->L[0] * c->L[1] * c->L[2];
    const double Nd = (double)c->g.N;
    // the shares go to the context's own scratch (after density 0's partial sums)
    double* escr = c->d_epart + c->nb_point + c->nb_sorted;
    k_energy_split<<<dim3(EPART_SPLIT, 1), ESPLIT_THREADS, 0, s>>>(epart, nb0, nb2, escr, 0);
    k_energy_final<<<1, EPART_SPLIT, 0, s>>>(escr, Omega / Nd, 0.5 * Omega / (Nd * Nd), E, 0);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int pipeline_run(vdw_ctx* c, const float* n, const float* grad, double* E, float* v, float* w, cudaStream_t s,
                 int fd, int xc, const cudaEvent_t* slab_ready, int B) {
    const GridArgs& g = c->g;
    if (g.N1 == 180 && g.N2 == 180 && g.N3 == 72)
        return run_sized<180, 180, 72>(c, n, grad, E, v, w, s, fd, xc, slab_ready, B);
    if (g.N1 == 256 && g.N2 == 256 && g.N3 == 96)
        return run_sized<256, 256, 96>(c, n, grad, E, v, w, s, fd, xc, slab_ready, B);
    return run_sized<0, 0, 0>(c, n, grad, E, v, w, s, fd, xc, slab_ready, B);
}

int pipeline_xc_final(vdw_ctx* c, double* E, cudaStream_t s) {
    const double dOmega = c->L[0] * c->L[1] * c->L[2] / (double)c->g.N;
    k_xc_final<<<1, 256, 0, s>>>(c->d_xc, c->d_xc + 4, XC_BLOCKS, dOmega, E);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

}  // namespace vdw
