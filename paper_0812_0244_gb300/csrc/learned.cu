// Learned reduced basis: M = 8 channels theta_m = n w_m(x(n, |grad n|)) whose
// weights come from a 2-64-64-8 SiLU network (bf16 operands on the tensor
// cores, FP32 accumulation in tensor memory), contracted with a learned
// pair kernel K_mn(|G|) (Catmull-Rom pieces between uniform knots), plus the paper's
// local correction Delta E (Eqs. DEnl, Depsnl).  The transform structure is
// the plain method's (Eqs. Eoffk, epsilon, epsofk, Vi) with M channels:
//
//   L1 k_learned_net       persistent, one block per SM: the network and its
//                          Jacobian (forward mode) on tiles of 128 points;
//                          theta_m to the packed real rows of the spectrum
//                          buffer, Delta E partial sums; then the forward plane
//                          transforms in place (k_planes_inplace)
//   L2 y transforms into |G| order, u_m(G) = sum_n K_mn(|G|) theta_n(G) and
//                          the FP64 energy over the sorted points (the plain
//                          method's kernels of contract.cu with the knot
//                          table), inverse y transforms; in training
//                          k_learned_contract_gradk, which also gives dE/dK
//   L3 inverse plane transforms in place (k_planes_inplace), then
//      k_learned_usum      per point: v_loc and g of w = g grad n (Eq. Vi)
//                          from u, the stored weights and Jacobian;
//                          forward plane transforms of w (k_w_planes)
//   then the plain method's divergence kernels (P4, P5).
//
// Training kernels: the parameter gradient of E through the network
// (k_learned_param_grad, CUDA cores, FP32 sums into FP64), a regression
// gradient for fitting the channel weights to targets, and an Adam step.
// Utilities: the plain cardinal weights p_a(q) and the spectral gradient.
#include "plane.cuh"
#include "pointwise.cuh"
#include "tc.cuh"

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>

namespace vdw {
namespace {

namespace cg = cooperative_groups;

constexpr int L_SLOTS = 8;        // network partial-sum slots per y plane (epart scratch)
constexpr int L_THREADS = 256;    // two warpgroups (channel kernel)
constexpr int L_NET_WG = 3;       // warpgroups of the network kernel
constexpr int L_NET_THREADS = 128 * L_NET_WG;
constexpr int L_TILE = 128;       // points per warpgroup tile
constexpr int L_MAXJ = 256;       // knots held in shared memory by the knot-gradient bins

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// SiLU and its derivative with the fast exponential and division: their
// error (a few FP32 ulp) is far below the bf16 rounding the activations get.
// The exponent is capped so that 1 + e stays inside __fdividef's range.
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(fminf(-z, 80.f))); }
__device__ __forceinline__ float silu_prime(float z) {
    const float s = __fdividef(1.f, 1.f + __expf(fminf(-z, 80.f)));
    return s * (1.f + z * (1.f - s));
}
// both from one exponential
__device__ __forceinline__ void silu_both(float z, float& f, float& fp) {
    const float s = __fdividef(1.f, 1.f + __expf(fminf(-z, 80.f)));
    f = z * s;
    fp = s * (1.f + z * (1.f - s));
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
// two values -> bf16x2 (a in the low half), one conversion instruction
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}
// 8 values -> one 16-byte core-matrix row
__device__ __forceinline__ void store8_bf16(uint16_t* dst, const float* v) {
    uint4 q;
    q.x = pack_bf16(v[0], v[1]);
    q.y = pack_bf16(v[2], v[3]);
    q.z = pack_bf16(v[4], v[5]);
    q.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(dst) = q;
}

__device__ __forceinline__ void wg_bar(int wg) { asm volatile("bar.sync %0, %1;" ::"r"(1 + wg), "r"(128) : "memory"); }

// Network features of Eq.-free form (no counterpart in the paper):
// x1 = (ln n - mu1)/sig1, x2 = (1/2 ln(s2 + eps^2) - mu2)/sig2,
// s2 = |grad n|^2 n^(-8/3), and the derivatives the potential needs.
struct Feat {
    float x1, x2;
    float dx1_dn, dx2_dn;  // d x / d n
    float gx2;             // (d x2 / d grad_c) / grad_c
    bool ok;
};
__device__ __forceinline__ Feat features(float n, float gx, float gy, float gz, const LearnedArgs& la, float n_min) {
    Feat f;
    f.ok = (n > n_min) && isfinite(n);
    const float ns = f.ok ? n : 1.f;
    const float cb = cbrtf(ns);
    const float n83 = 1.f / (ns * ns * cb * cb);
    const float s2 = (gx * gx + gy * gy + gz * gz) * n83;
    const float den = s2 + la.eps2;
    f.x1 = (logf(ns) - la.mu1) * la.inv_sig1;
    f.x2 = (0.5f * logf(den) - la.mu2) * la.inv_sig2;
    f.dx1_dn = la.inv_sig1 / ns;
    f.dx2_dn = -(4.f / 3.f) * s2 / (ns * den) * la.inv_sig2;
    f.gx2 = n83 / den * la.inv_sig2;
    return f;
}

// Cardinal cubic splines of the base mesh (Eq. fofx on an M-point mesh): p_m
// and dp_m/dq at q clamped to the mesh; returns false where the clamp acts
// (the derivative of the clamped basis is then zero).
// bMq: the base splines' second derivatives (la.bMq, or a shared-memory copy
// of it: indexed by the lane's interval, a parameter-space read serialises)
// The coefficients shared by the channels at one q: interval k, A = (x1 - q)/h,
// B = 1 - A and the cubic terms of the value and of d/dq.
struct BaseCoef {
    int k;
    float A, B, cA, cB, dA, dB, ih;
    bool inside;
};
__device__ __forceinline__ BaseCoef base_coef(float q, const LearnedArgs& la) {
    BaseCoef c;
    const float lo = la.bqm[0], hi = la.bqm[LRN_M - 1];
    c.inside = (q >= lo) && (q <= hi);
    const float qc = fminf(fmaxf(q, lo), hi);
    int k = 0;  // knots <= q among the interior ones: interval in [0, M - 2]
#pragma unroll
    for (int i = 1; i < LRN_M - 1; ++i) k += (qc >= la.bqm[i]) ? 1 : 0;
    const float x0 = la.bqm[k], x1 = la.bqm[k + 1], h = x1 - x0;
    c.k = k;
    c.ih = 1.f / h;
    c.A = (x1 - qc) * c.ih;
    c.B = 1.f - c.A;
    const float h6 = h * h * (1.f / 6.f);
    c.cA = (c.A * c.A * c.A - c.A) * h6;
    c.cB = (c.B * c.B * c.B - c.B) * h6;
    c.dA = -(3.f * c.A * c.A - 1.f) * (1.f / 6.f) * h;
    c.dB = (3.f * c.B * c.B - 1.f) * (1.f / 6.f) * h;
    return c;
}
// p_m and dp_m/dq of channel m
__device__ __forceinline__ void base_channel(const BaseCoef& c, int m, const float* bMq, float& p, float& dp) {
    const float Ma = bMq[m * LRN_M + c.k], Mb = bMq[m * LRN_M + c.k + 1];
    const float ya = (m == c.k) ? 1.f : 0.f, yb = (m == c.k + 1) ? 1.f : 0.f;
    p = c.A * ya + c.B * yb + c.cA * Ma + c.cB * Mb;
    dp = (yb - ya) * c.ih + c.dA * Ma + c.dB * Mb;
}
__device__ __forceinline__ bool base_weights(float q, const LearnedArgs& la, float* p, float* dp,
                                             const float* bMq) {
    const BaseCoef c = base_coef(q, la);
#pragma unroll
    for (int m = 0; m < LRN_M; ++m) base_channel(c, m, bMq, p[m], dp[m]);
    return c.inside;
}

// ---------------------------------------------------------------------------
// shared memory of the tensor-core network
// ---------------------------------------------------------------------------
// forward operands and the small layers
struct __align__(128) MlpShared {
    uint16_t w2f[LRN_H * LRN_H];
    uint16_t w3f[LRN_N3 * LRN_H];
    float w1[2 * LRN_H], b1[LRN_H], b2[LRN_H], b3[LRN_M];
};
// One warpgroup's activation operand.
struct __align__(128) MlpWG {
    uint16_t A[L_TILE * LRN_H];
};
// One warpgroup's operands of the forward pass with its two tangents.
struct __align__(128) MlpWG3 {
    uint16_t A[3][L_TILE * LRN_H];
};
constexpr int L_MAXWG = 4;  // warpgroups per block at most
struct MlpCtl {
    uint64_t bar[L_MAXWG];
    uint32_t tmem;
    uint32_t wgcols;  // tensor-memory columns per warpgroup
    uint32_t cols;    // columns allocated (a power of two >= warpgroups x wgcols)
    int abort[L_MAXWG];  // per warpgroup: a wait gave up
};

__device__ void mlp_load_weights(MlpShared* S, const LearnedArgs& la) {
    const uint4* s1 = reinterpret_cast<const uint4*>(la.w2f);
    uint4* d1 = reinterpret_cast<uint4*>(S->w2f);
    for (int i = threadIdx.x; i < LRN_H * LRN_H / 8; i += blockDim.x) d1[i] = s1[i];
    const uint4* s2 = reinterpret_cast<const uint4*>(la.w3f);
    uint4* d2 = reinterpret_cast<uint4*>(S->w3f);
    for (int i = threadIdx.x; i < LRN_N3 * LRN_H / 8; i += blockDim.x) d2[i] = s2[i];
    for (int i = threadIdx.x; i < 2 * LRN_H; i += blockDim.x) S->w1[i] = la.w1[i];
    for (int i = threadIdx.x; i < LRN_H; i += blockDim.x) {
        S->b1[i] = la.b1[i];
        S->b2[i] = la.b2[i];
    }
    for (int i = threadIdx.x; i < LRN_M; i += blockDim.x) S->b3[i] = la.b3[i];
}

// Block setup: barriers, tensor memory (wgcols columns per warpgroup, a
// power of two of at least 32; the allocation is rounded up to a power of two).
__device__ void mlp_setup(MlpCtl* ctl, uint32_t wgcols) {
    const int nwg = blockDim.x >> 7;
    uint32_t cols = 32;
    while (cols < (uint32_t)nwg * wgcols) cols <<= 1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < nwg; ++i) {
            tc::mbar_init(&ctl->bar[i], 1);
            ctl->abort[i] = 0;
        }
        ctl->wgcols = wgcols;
        ctl->cols = cols;
    }
    if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&ctl->tmem, cols);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

__device__ void mlp_teardown(MlpCtl* ctl) {
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_free(ctl->tmem, ctl->cols);
}

// Issue, for each of nA operands A[i] (K-wide), the K/16 MMAs of A[i] x B^T
// into column col[i] of this warpgroup's tensor memory (one elected thread,
// one commit to the warpgroup's mbarrier).
__device__ __forceinline__ void wg_mma_issue(MlpCtl* ctl, int wg, int r, const uint16_t* const* A, const uint32_t* col,
                                             int nA, const uint16_t* B, int K, int N) {
    tc::fence_async_smem();
    tc::fence_before_sync();
    wg_bar(wg);
    if (r == 0) {
        tc::fence_after_sync();
        const uint32_t b = tc::smem_u32(B);
        for (int i = 0; i < nA; ++i) {
            const uint32_t a = tc::smem_u32(A[i]);
            const uint32_t d = ctl->tmem + (uint32_t)wg * ctl->wgcols + col[i];
            for (int k = 0; k < K / 16; ++k)
                tc::mma_bf16(d, tc::operand_desc(a, K, k), tc::operand_desc(b, K, k), tc::idesc_bf16(128, N), k > 0);
        }
        tc::mma_commit(&ctl->bar[wg]);
    }
}
// Wait for the warpgroup's last commit and agree across the warpgroup on success.
__device__ __forceinline__ bool wg_mma_wait(MlpCtl* ctl, int wg, uint32_t& phase, int* err) {
    const bool ok = tc::mbar_wait(&ctl->bar[wg], phase);
    if (!ok) {
        atomicExch(&ctl->abort[wg], 1);
        *(volatile int*)err = 1;  // page-locked host word, read by the next entry point
        __threadfence_system();
        // the committed MMAs may still be writing this warpgroup's tensor
        // memory: give them a second bounded wait before the warpgroup stops
        // and the block frees that memory
        tc::mbar_wait(&ctl->bar[wg], phase);
    }
    phase ^= 1u;
    wg_bar(wg);
    tc::fence_after_sync();
    return ctl->abort[wg] == 0;
}
__device__ __forceinline__ bool wg_mma_n(MlpCtl* ctl, int wg, int r, uint32_t& phase, const uint16_t* const* A,
                                         const uint32_t* col, int nA, const uint16_t* B, int K, int N, int* err) {
    wg_mma_issue(ctl, wg, r, A, col, nA, B, K, N);
    return wg_mma_wait(ctl, wg, phase, err);
}

__device__ __forceinline__ bool wg_mma(MlpCtl* ctl, int wg, int r, uint32_t& phase, const uint16_t* A,
                                       const uint16_t* B, int K, int N, uint32_t col, int* err) {
    return wg_mma_n(ctl, wg, r, phase, &A, &col, 1, B, K, N, err);
}

// tensor-memory address of this thread's lane, column col of its warpgroup
__device__ __forceinline__ uint32_t lane_addr(const MlpCtl* ctl, int wg, uint32_t col) {
    const int warp = threadIdx.x >> 5;
    return ctl->tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)wg * ctl->wgcols + col;
}

// Forward network on the warpgroup's tile (row r = this thread's point):
// layer 1 on the CUDA cores, layers 2 and 3 on the tensor cores.  Leaves the
// layer-2 accumulator in columns [0, 64) and returns the 8 outputs in o.
__device__ bool mlp_forward(MlpShared* S, MlpWG* W, MlpCtl* ctl, int wg, int r, uint32_t& phase, float x1,
                            float x2, float* o, int* err) {
#pragma unroll
    for (int c = 0; c < LRN_H / 8; ++c) {
        float h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = 8 * c + q;
            h[q] = silu(fmaf(S->w1[2 * j], x1, fmaf(S->w1[2 * j + 1], x2, S->b1[j])));
        }
        store8_bf16(W->A + tc::kmaj(r, 8 * c, LRN_H), h);
    }
    if (!wg_mma(ctl, wg, r, phase, W->A, S->w2f, LRN_H, LRN_H, 0, err)) return false;
#pragma unroll
    for (int c = 0; c < LRN_H / 16; ++c) {
        float v[16];
        tc::tmem_ld16(lane_addr(ctl, wg, 16 * c), v);
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = silu(v[q] + S->b2[16 * c + q]);
        store8_bf16(W->A + tc::kmaj(r, 16 * c, LRN_H), v);
        store8_bf16(W->A + tc::kmaj(r, 16 * c + 8, LRN_H), v + 8);
    }
    if (!wg_mma(ctl, wg, r, phase, W->A, S->w3f, LRN_H, LRN_N3, 64, err)) return false;
    float v[16];
    tc::tmem_ld16(lane_addr(ctl, wg, 64), v);
#pragma unroll
    for (int m = 0; m < LRN_M; ++m) o[m] = v[m] + S->b3[m];
    return true;
}

// Forward network with its Jacobian by forward mode (two tangents, one per
// feature), on the warpgroup's tile: layer 1 and its tangents on the CUDA
// cores, then layers 2 and 3 on the tensor cores.  Tangents enter the
// products as bf16 like the activations.  Tensor memory: 128 columns per
// warpgroup.  Layer 2 runs in two batches: the activation into [0, 64) and
// the first tangent into [64, 128); after their epilogue the second tangent
// reuses [64, 128) while the layer-2 pre-activation stays in [0, 64) for its
// SiLU derivative.  Layer 3 then writes [0, 16), [16, 32), [32, 48).
// Returns o (8 outputs) and J1, J2 (d o / d x1, d o / d x2).
// overlap() runs on every thread of the warpgroup while the first layer-2
// batch is in flight (work that does not depend on the network).
template <class Overlap>
__device__ bool mlp_forward_jac(MlpShared* S, MlpWG3* W, MlpCtl* ctl, int wg, int r, uint32_t& phase, float x1,
                                float x2, float* o, float* J1, float* J2, int* err, Overlap overlap) {
#pragma unroll
    for (int c = 0; c < LRN_H / 8; ++c) {
        float h[8], t1[8], t2[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = 8 * c + q;
            const float z = fmaf(S->w1[2 * j], x1, fmaf(S->w1[2 * j + 1], x2, S->b1[j]));
            float sp;
            silu_both(z, h[q], sp);
            t1[q] = sp * S->w1[2 * j];
            t2[q] = sp * S->w1[2 * j + 1];
        }
        store8_bf16(W->A[0] + tc::kmaj(r, 8 * c, LRN_H), h);
        store8_bf16(W->A[1] + tc::kmaj(r, 8 * c, LRN_H), t1);
        store8_bf16(W->A[2] + tc::kmaj(r, 8 * c, LRN_H), t2);
    }
    {
        const uint16_t* As[2] = {W->A[0], W->A[1]};
        const uint32_t cols[2] = {0, 64};
        wg_mma_issue(ctl, wg, r, As, cols, 2, S->w2f, LRN_H, LRN_H);
        overlap();
        if (!wg_mma_wait(ctl, wg, phase, err)) return false;
    }
#pragma unroll
    for (int c = 0; c < LRN_H / 16; ++c) {
        float z[16], d1[16];
        tc::tmem_ld16(lane_addr(ctl, wg, 16 * c), z);
        tc::tmem_ld16(lane_addr(ctl, wg, 64 + 16 * c), d1);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float sp;
            silu_both(z[q] + S->b2[16 * c + q], z[q], sp);
            d1[q] *= sp;
        }
        store8_bf16(W->A[0] + tc::kmaj(r, 16 * c, LRN_H), z);
        store8_bf16(W->A[0] + tc::kmaj(r, 16 * c + 8, LRN_H), z + 8);
        store8_bf16(W->A[1] + tc::kmaj(r, 16 * c, LRN_H), d1);
        store8_bf16(W->A[1] + tc::kmaj(r, 16 * c + 8, LRN_H), d1 + 8);
    }
    {
        // the first tangent's columns are read (tcgen05.wait::ld in tmem_ld16)
        const uint16_t* As[1] = {W->A[2]};
        const uint32_t cols[1] = {64};
        wg_mma_issue(ctl, wg, r, As, cols, 1, S->w2f, LRN_H, LRN_H);
        if (!wg_mma_wait(ctl, wg, phase, err)) return false;
    }
#pragma unroll
    for (int c = 0; c < LRN_H / 16; ++c) {
        float z[16], d2[16];
        tc::tmem_ld16(lane_addr(ctl, wg, 16 * c), z);
        tc::tmem_ld16(lane_addr(ctl, wg, 64 + 16 * c), d2);
#pragma unroll
        for (int q = 0; q < 16; ++q) d2[q] *= silu_prime(z[q] + S->b2[16 * c + q]);
        store8_bf16(W->A[2] + tc::kmaj(r, 16 * c, LRN_H), d2);
        store8_bf16(W->A[2] + tc::kmaj(r, 16 * c + 8, LRN_H), d2 + 8);
    }
    {
        const uint16_t* As[3] = {W->A[0], W->A[1], W->A[2]};
        const uint32_t cols[3] = {0, 16, 32};
        if (!wg_mma_n(ctl, wg, r, phase, As, cols, 3, S->w3f, LRN_H, LRN_N3, err)) return false;
    }
    float v[16];
    tc::tmem_ld16(lane_addr(ctl, wg, 0), v);
#pragma unroll
    for (int m = 0; m < LRN_M; ++m) o[m] = v[m] + S->b3[m];
    tc::tmem_ld16(lane_addr(ctl, wg, 16), v);
#pragma unroll
    for (int m = 0; m < LRN_M; ++m) J1[m] = v[m];
    tc::tmem_ld16(lane_addr(ctl, wg, 32), v);
#pragma unroll
    for (int m = 0; m < LRN_M; ++m) J2[m] = v[m];
    return true;
}

// ---------------------------------------------------------------------------
// L0: model preparation (flat FP32 parameters -> device operands)
// ---------------------------------------------------------------------------
__global__ void k_learned_prepare(const float* __restrict__ flat, LearnedArgs la) {
    float* w1 = const_cast<float*>(la.w1);
    float* b1 = const_cast<float*>(la.b1);
    float* b2 = const_cast<float*>(la.b2);
    float* b3 = const_cast<float*>(la.b3);
    float* w2r = const_cast<float*>(la.w2r);
    float* w3r = const_cast<float*>(la.w3r);
    uint16_t* w2f = const_cast<uint16_t*>(la.w2f);
    uint16_t* w3f = const_cast<uint16_t*>(la.w3f);
    float4* kn = const_cast<float4*>(la.knots);
    const int t = threadIdx.x + blockIdx.x * blockDim.x, nt = blockDim.x * gridDim.x;
    auto bfu = [](float x) { return (uint16_t)__bfloat16_as_ushort(__float2bfloat16_rn(x)); };
    for (int i = t; i < 2 * LRN_H; i += nt) w1[i] = bf16r(flat[LRN_OFF_W1 + i]);
    for (int i = t; i < LRN_H; i += nt) {
        b1[i] = flat[LRN_OFF_B1 + i];
        b2[i] = flat[LRN_OFF_B2 + i];
    }
    for (int i = t; i < LRN_M; i += nt) b3[i] = flat[LRN_OFF_B3 + i];
    for (int i = t; i < LRN_H * LRN_H; i += nt) {
        const int o = i / LRN_H, j = i % LRN_H;  // W2[o][j]: output o, input j
        const float x = flat[LRN_OFF_W2 + i];
        w2r[i] = bf16r(x);
        w2f[tc::kmaj(o, j, LRN_H)] = bfu(x);
    }
    for (int i = t; i < LRN_N3 * LRN_H; i += nt) {
        const int m = i / LRN_H, j = i % LRN_H;  // W3[m][j], rows m >= M are zero
        const float x = m < LRN_M ? flat[LRN_OFF_W3 + m * LRN_H + j] : 0.f;
        if (m < LRN_M) w3r[m * LRN_H + j] = bf16r(x);
        w3f[tc::kmaj(m, j, LRN_H)] = bfu(x);
    }
    // Catmull-Rom piece on [k_j, k_j+1] from knots j-1 .. j+2: K is even in k
    // (K_-1 = K_1) and continues linearly past the last knot
    const float* K = flat + LRN_OFF_K;
    const int J = la.J;
    for (int i = t; i < (J - 1) * LRN_P; i += nt) {
        const int j = i / LRN_P, p = i % LRN_P;
        const float* Kp = K + p * J;
        const float P0 = Kp[j == 0 ? 1 : j - 1], P1 = Kp[j], P2 = Kp[j + 1];
        const float P3 = j + 2 <= J - 1 ? Kp[j + 2] : 2.f * Kp[J - 1] - Kp[J - 2];
        kn[i] = make_float4(P1, 0.5f * (P2 - P0), P0 - 2.5f * P1 + 2.f * P2 - 0.5f * P3,
                            -0.5f * P0 + 1.5f * P1 - 1.5f * P2 + 0.5f * P3);
    }
}

// ---------------------------------------------------------------------------
// L1: network and channels
// ---------------------------------------------------------------------------
// One persistent block per SM, three warpgroups, each running the network and
// its two tangents on tiles of 128 points (packed order): layer 1 on CUDA
// cores gives three bf16 operands in the tcgen05 core-matrix layout; layer 2
// is 2 x 4 and then 1 x 4 MMAs into the warpgroup's 128 tensor-memory
// columns, layer 3 is 3 x 4 MMAs (mlp_forward_jac).  theta_m = n w_m goes to the packed real rows of plane (m, y) of the
// spectrum buffer (the forward plane transforms follow in place).  With lw
// the per-point coefficients of the assembly of Eq. (Vi) are stored,
// lw[c][q] in packed order (LW_ROWS rows): v_loc = sum_m u_m lw[m] + lw[2M]
// and g = sum_m u_m lw[M + m] + lw[2M + 1], i.e.
//   lw[m]     = w_m + n dw_m/dn          (network Jacobian through x1, x2; base through q)
//   lw[M + m] = n (dw_m/d|grad n|)/|grad n|
//   lw[2M], lw[2M + 1] = the Delta E derivatives.
// Delta E partial sums per block.
__global__ void __launch_bounds__(L_NET_THREADS, 1)
    k_learned_net(const float* __restrict__ n, const float* __restrict__ grad, GridArgs g, PointParams P,
                  LearnedArgs la, float* __restrict__ specf, double* __restrict__ epart,
                  unsigned long long* __restrict__ invalid, float* __restrict__ lw) {
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ MlpCtl ctl;
    __shared__ double red[32];
    __shared__ float qm[MAX_NQ];
    __shared__ float bMq_s[LRN_M * LRN_M];
    MlpShared* S = reinterpret_cast<MlpShared*>(smraw);
    MlpWG3* Wb = reinterpret_cast<MlpWG3*>(smraw + sizeof(MlpShared));
    const int wg = threadIdx.x >> 7, r = threadIdx.x & 127;
    MlpWG3* W = Wb + wg;
    mlp_load_weights(S, la);
    for (int i = threadIdx.x; i < MAX_NQ; i += blockDim.x) qm[i] = P.qm[i];
    for (int i = threadIdx.x; i < LRN_M * LRN_M; i += blockDim.x) bMq_s[i] = la.bMq[i];
    mlp_setup(&ctl, 128);
    const long long N = g.N;
    const long long ntiles = (N + L_TILE - 1) / L_TILE;
    const long long fstride = 2LL * g.N2 * g.ncols;  // floats between the planes of two channels
    uint32_t phase = 0;
    double eacc = 0.0;
    unsigned int bad = 0;
    for (long long T = L_NET_WG * (long long)blockIdx.x + wg; T < ntiles; T += L_NET_WG * (long long)gridDim.x) {
        const long long q = T * L_TILE + r;
        const bool in = q < N;
        int y = 0, z = 0, x = 0, j = 0;
        long long gi = 0;
        float ni = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        if (in) {
            gi = packed_point(q, g, y, z, x, j);
            ni = n[gi];
            gx = grad[gi];
            gy = grad[N + gi];
            gz = grad[2 * N + gi];
        }
        const Feat f = features(ni, gx, gy, gz, la, P.n_min);
        const bool ok = in && f.ok;
        float pb[LRN_M], dpb[LRN_M];
#pragma unroll
        for (int m = 0; m < LRN_M; ++m) pb[m] = dpb[m] = 0.f;
        float bn = 0.f, bg = 0.f, dEn = 0.f, dEg = 0.f;
        // q chain, Delta E and the spline base while the layer-2 MMAs run
        auto qwork = [&]() {
            if (in) {
                bad += (!(ni >= 0.f) || !isfinite(ni)) ? 1u : 0u;
                const QPoint qp = q_point(ni, gx, gy, gz, P, qm);
                if (qp.k != K_INVALID) {
                    const float qq = qp.q, q3 = qq * qq * qq, q4 = q3 * qq;
                    eacc += (double)(0.5f * P.C_s * ni * ni / q3);
                    const float cn = 1.5f * P.C_s * ni * ni / q4;
                    dEn = P.C_s * ni / q3 - cn * qp.dq_dn;
                    dEg = -cn * qp.dq_dg;
                    // the clamped base has no q derivative
                    if (la.base && base_weights(qq, la, pb, dpb, bMq_s)) {
                        bn = qp.dq_dn;
                        bg = qp.dq_dg;
                    }
                }
            }
        };
        float o[LRN_M], J1[LRN_M], J2[LRN_M];
        if (!mlp_forward_jac(S, W, &ctl, wg, r, phase, ok ? f.x1 : 0.f, ok ? f.x2 : 0.f, o, J1, J2, la.err, qwork))
            break;
        if (in) {
            float* dst = specf + 2LL * y * g.ncols + packed_offset(x, j, z & 1, g.Nh);
#pragma unroll
            for (int m = 0; m < LRN_M; ++m) dst[m * fstride] = ok ? ni * (o[m] + pb[m]) : 0.f;
            if (lw) {
#pragma unroll
                for (int m = 0; m < LRN_M; ++m) {
                    const float dwn = J1[m] * f.dx1_dn + J2[m] * f.dx2_dn + dpb[m] * bn;
                    const float dwg = J2[m] * f.gx2 + dpb[m] * bg;
                    lw[m * N + q] = ok ? o[m] + pb[m] + ni * dwn : 0.f;
                    lw[(LRN_M + m) * N + q] = ok ? ni * dwg : 0.f;
                }
                lw[2 * LRN_M * N + q] = ok ? dEn : 0.f;
                lw[(2 * LRN_M + 1) * N + q] = ok ? dEg : 0.f;
            }
        }
    }
    mlp_teardown(&ctl);
    const double es = block_sum(eacc, red);
    if (threadIdx.x == 0) epart[blockIdx.x] = es;
    __syncthreads();
    const double b = block_sum((double)bad, red);
    if (threadIdx.x == 0 && b > 0.0) atomicAdd(invalid, (unsigned long long)b);
}

// ---------------------------------------------------------------------------
// L1' the network tabulated on the features' node grid, and its lookup
// ---------------------------------------------------------------------------
// The network's outputs o(x1, x2) depend on a point only through its two
// features.  k_learned_tabulate runs the network (tensor cores, as
// k_learned_channels) once on the (T+2)^2 nodes x = -D + (i - 1) h; the
// inference kernel k_learned_lookup then takes each point's o and its
// Jacobian from the tensor product of Catmull-Rom cubics through the 4 x 4
// nodes around (x1, x2) (features clamped to [-D, D], zero derivative along a
// clamped axis): the interpolant is C1 and its derivative is what the
// potential uses, so v is the exact derivative of the tabulated energy.
__global__ void __launch_bounds__(L_THREADS, 1) k_learned_tabulate(LearnedArgs la, float4* __restrict__ tab) {
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ MlpCtl ctl;
    MlpShared* S = reinterpret_cast<MlpShared*>(smraw);
    MlpWG* Wb = reinterpret_cast<MlpWG*>(smraw + sizeof(MlpShared));
    const int wg = threadIdx.x >> 7, r = threadIdx.x & 127;
    mlp_load_weights(S, la);
    mlp_setup(&ctl, 128);
    uint32_t phase = 0;
    const int T2 = la.tabT + 2;
    const long long nodes = (long long)T2 * T2;
    const long long ntiles = (nodes + L_TILE - 1) / L_TILE;
    for (long long T = 2 * (long long)blockIdx.x + wg; T < ntiles; T += 2 * (long long)gridDim.x) {
        const long long i = T * L_TILE + r;
        const bool in = i < nodes;
        const int i1 = in ? (int)(i / T2) : 0, i2 = in ? (int)(i - (long long)i1 * T2) : 0;
        const float x1 = -la.tabD + (float)(i1 - 1) * la.tab_h, x2 = -la.tabD + (float)(i2 - 1) * la.tab_h;
        float o[LRN_M];
        if (!mlp_forward(S, Wb + wg, &ctl, wg, r, phase, x1, x2, o, la.err)) break;
        if (in) {
            tab[i] = make_float4(o[0], o[1], o[2], o[3]);
            tab[nodes + i] = make_float4(o[4], o[5], o[6], o[7]);
        }
    }
    mlp_teardown(&ctl);
}

// Catmull-Rom weights of nodes i-1 .. i+2 at local position s, and d/ds.
__device__ __forceinline__ void catmull_rom(float s, float* w, float* dw) {
    const float s2 = s * s, s3 = s2 * s;
    w[0] = 0.5f * (-s3 + 2.f * s2 - s);
    w[1] = 0.5f * (3.f * s3 - 5.f * s2) + 1.f;
    w[2] = 0.5f * (-3.f * s3 + 4.f * s2 + s);
    w[3] = 0.5f * (s3 - s2);
    dw[0] = 0.5f * (-3.f * s2 + 4.f * s - 1.f);
    dw[1] = 0.5f * (9.f * s2 - 10.f * s);
    dw[2] = 0.5f * (-9.f * s2 + 8.f * s + 1.f);
    dw[3] = 0.5f * (3.f * s2 - 2.f * s);
}

// node index of the interval start, local position and the axis's d/dx factor
__device__ __forceinline__ int table_axis(float x, const LearnedArgs& la, float& s, float& dscale) {
    const float xc = fminf(fmaxf(x, -la.tabD), la.tabD);
    const float u = (xc + la.tabD) * la.tab_inv_h;
    const int i = min((int)u, la.tabT - 2);
    s = u - (float)i;
    dscale = (x >= -la.tabD && x <= la.tabD) ? la.tab_inv_h : 0.f;
    return i;
}

// One thread per point (packed order, grid-stride); writes what k_learned_net
// writes (theta channels, the assembly coefficients, Delta E partials).  The
// channels go in two halves of four (one float4 of each node per half), so
// that a thread holds one half's sums at a time.
constexpr int LOOKUP_THREADS = 256;
__global__ void __launch_bounds__(LOOKUP_THREADS, 3) k_learned_lookup(const float* __restrict__ n,
                                                                     const float* __restrict__ grad, GridArgs g,
                                                                     PointParams P, LearnedArgs la,
                                                                     float* __restrict__ specf,
                                                                     double* __restrict__ epart,
                                                                     unsigned long long* __restrict__ invalid,
                                                                     float* __restrict__ lw) {
    __shared__ double red[32];
    __shared__ float qm[MAX_NQ];
    __shared__ float bMq_s[LRN_M * LRN_M];
    for (int i = threadIdx.x; i < MAX_NQ; i += blockDim.x) qm[i] = P.qm[i];
    for (int i = threadIdx.x; i < LRN_M * LRN_M; i += blockDim.x) bMq_s[i] = la.bMq[i];
    __syncthreads();
    const long long N = g.N;
    const long long fstride = 2LL * g.N2 * g.ncols;  // floats between the planes of two channels
    const int T2 = la.tabT + 2;
    const long long hstride = (long long)T2 * T2;    // float4s between the two halves of the table
    double eacc = 0.0;
    unsigned int bad = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int y, z, x, j;
        const long long gi = packed_point(q, g, y, z, x, j);
        const float ni = n[gi], gx = grad[gi], gy = grad[N + gi], gz = grad[2 * N + gi];
        bad += (!(ni >= 0.f) || !isfinite(ni)) ? 1u : 0u;
        const Feat f = features(ni, gx, gy, gz, la, P.n_min);
        const bool ok = f.ok;
        // q chain: Delta E and the spline base's coefficients
        float bn = 0.f, bg = 0.f, dEn = 0.f, dEg = 0.f;
        BaseCoef bc = {};
        bool base_on = false;
        const QPoint qp = q_point(ni, gx, gy, gz, P, qm);
        if (qp.k != K_INVALID) {
            const float qq = qp.q, q3 = qq * qq * qq, q4 = q3 * qq;
            eacc += (double)(0.5f * P.C_s * ni * ni / q3);
            const float cn = 1.5f * P.C_s * ni * ni / q4;
            dEn = P.C_s * ni / q3 - cn * qp.dq_dn;
            dEg = -cn * qp.dq_dg;
            if (la.base) {
                // the clamped base has no q derivative
                bc = base_coef(qq, la);
                base_on = true;
                if (bc.inside) {
                    bn = qp.dq_dn;
                    bg = qp.dq_dg;
                }
            }
        }
        // the network from the table: Catmull-Rom weights along both axes
        float s1, s2, ds1, ds2;
        const int i1 = table_axis(ok ? f.x1 : 0.f, la, s1, ds1);
        const int i2 = table_axis(ok ? f.x2 : 0.f, la, s2, ds2);
        float a[4], da[4], b[4], db[4];
        catmull_rom(s1, a, da);
        catmull_rom(s2, b, db);
        float* dst = specf + 2LL * y * g.ncols + packed_offset(x, j, z & 1, g.Nh);
        const float4* node = la.tab + (long long)i1 * T2 + i2;
#pragma unroll 1
        for (int h = 0; h < 2; ++h, node += hstride) {
            // per row k of nodes: R = sum_l b_l v, S = sum_l b'_l v; then
            // o = sum_k a_k R_k, d/dx1 = sum_k a'_k R_k, d/dx2 = sum_k a_k S_k
            float o[4], J1[4], J2[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) o[m] = J1[m] = J2[m] = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float R[4], Sd[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) R[m] = Sd[m] = 0.f;
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const float4 v4 = __ldg(node + k * T2 + l);
                    const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        R[m] = fmaf(b[l], v[m], R[m]);
                        Sd[m] = fmaf(db[l], v[m], Sd[m]);
                    }
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    o[m] = fmaf(a[k], R[m], o[m]);
                    J1[m] = fmaf(da[k], R[m], J1[m]);
                    J2[m] = fmaf(a[k], Sd[m], J2[m]);
                }
            }
#pragma unroll
            for (int mm = 0; mm < 4; ++mm) {
                const int m = 4 * h + mm;
                float pb = 0.f, dpb = 0.f;
                if (base_on) base_channel(bc, m, bMq_s, pb, dpb);
                const float j1 = J1[mm] * ds1, j2 = J2[mm] * ds2;
                dst[m * fstride] = ok ? ni * (o[mm] + pb) : 0.f;
                if (lw) {
                    const float dwn = j1 * f.dx1_dn + j2 * f.dx2_dn + dpb * bn;
                    const float dwg = j2 * f.gx2 + dpb * bg;
                    lw[m * N + q] = ok ? o[mm] + pb + ni * dwn : 0.f;
                    lw[(LRN_M + m) * N + q] = ok ? ni * dwg : 0.f;
                }
            }
        }
        if (lw) {
            lw[2 * LRN_M * N + q] = ok ? dEn : 0.f;
            lw[(2 * LRN_M + 1) * N + q] = ok ? dEg : 0.f;
        }
    }
    const double es = block_sum(eacc, red);
    if (threadIdx.x == 0) epart[blockIdx.x] = es;
    __syncthreads();
    const double bsum = block_sum((double)bad, red);
    if (threadIdx.x == 0 && bsum > 0.0) atomicAdd(invalid, (unsigned long long)bsum);
}

// ---------------------------------------------------------------------------
// L2 (training form): contraction over the points in |G| order with dE/dK
// ---------------------------------------------------------------------------
// The energy and potential forms use the plain method's sorted contraction
// (contract.cu) with the knot table.  This form also accumulates
//   dE/dK_p(k_i) = sum_G 1/2 Omega w_G (2 - delta_ab) Re(conj th_a th_b) c_i(|G|)
// for the four Catmull-Rom weights c_i of the knots around |G| (Eq. Eoffk
// differentiated through the interpolation), in shared-memory bins [P][J].
// In |G| order the 32 points of a warp nearly always share their interval:
// the warp then sums its contributions first and one lane adds them.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(SORTED_BLOCK) k_learned_contract_gradk(float4* __restrict__ Q, long long qstride,
                                                                       const float* __restrict__ gs, LearnedArgs la,
                                                                       float invN, double* __restrict__ epart,
                                                                       double* __restrict__ gK, float halfOmega) {
    constexpr int NQ = LRN_M;
    extern __shared__ float bins[];  // [P][J]
    __shared__ double red[32];
    const int J = la.J;
    for (int i = threadIdx.x; i < LRN_P * J; i += blockDim.x) bins[i] = 0.f;
    __syncthreads();
    const long long r = (long long)blockIdx.x * SORTED_BLOCK + threadIdx.x;
    const int lane = threadIdx.x & 31;
    float2 th[NQ];
#pragma unroll
    for (int q = 0; q < NQ / 4; ++q) {
        const float4 a = Q[q * qstride + 2 * r], b = Q[q * qstride + 2 * r + 1];
        th[4 * q] = make_float2(a.x, a.y);
        th[4 * q + 1] = make_float2(a.z, a.w);
        th[4 * q + 2] = make_float2(b.x, b.y);
        th[4 * q + 3] = make_float2(b.z, b.w);
    }
    const float gm = gs[r];
    const float wgt = signbit(gm) ? 1.f : 2.f;
    const float sk = fabsf(gm) * la.inv_dk;
    const int j = min((int)sk, J - 2);
    const float t = sk - (float)j;
    const float4* cf = la.knots + (long long)j * LRN_P;
    // Catmull-Rom weights of the knots j-1 .. j+2
    const float wm1 = 0.5f * t * (t * (2.f - t) - 1.f), w0 = 1.f + t * t * (1.5f * t - 2.5f);
    const float w1 = 0.5f * t * (1.f + t * (4.f - 3.f * t)), w2 = 0.5f * t * t * (t - 1.f);
    // knots of the four weights: the knot before k = 0 mirrors knot 1; past the
    // last knot the linear extrapolation 2 K_{J-1} - K_{J-2}
    const int km1 = j == 0 ? 1 : j - 1;
    const bool tail = j + 2 > J - 1;
    const bool uni = __all_sync(0xffffffffu, j == __shfl_sync(0xffffffffu, j, 0));
    float2 u[NQ];
#pragma unroll
    for (int a = 0; a < NQ; ++a) u[a] = make_float2(0.f, 0.f);
    int p = 0;
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
#pragma unroll
        for (int b = a; b < NQ; ++b, ++p) {
            const float4 c = cf[p];
            const float phi = fmaf(t, fmaf(t, fmaf(t, c.w, c.z), c.y), c.x);
            u[a].x = fmaf(phi, th[b].x, u[a].x);
            u[a].y = fmaf(phi, th[b].y, u[a].y);
            if (b != a) {
                u[b].x = fmaf(phi, th[a].x, u[b].x);
                u[b].y = fmaf(phi, th[a].y, u[b].y);
            }
            const float rv = halfOmega * wgt * (b != a ? 2.f : 1.f) * (th[a].x * th[b].x + th[a].y * th[b].y);
            float* bp = bins + p * J;
            if (uni) {
                const float s0 = warp_sum_f(wm1 * rv), s1 = warp_sum_f(w0 * rv);
                const float s2 = warp_sum_f(w1 * rv), s3 = warp_sum_f(w2 * rv);
                if (lane == 0) {
                    atomicAdd(&bp[km1], s0);
                    atomicAdd(&bp[j], s1);
                    atomicAdd(&bp[j + 1], s2);
                    if (!tail) {
                        atomicAdd(&bp[j + 2], s3);
                    } else {
                        atomicAdd(&bp[J - 1], 2.f * s3);
                        atomicAdd(&bp[J - 2], -s3);
                    }
                }
            } else {
                atomicAdd(&bp[km1], wm1 * rv);
                atomicAdd(&bp[j], w0 * rv);
                atomicAdd(&bp[j + 1], w1 * rv);
                if (!tail) {
                    atomicAdd(&bp[j + 2], w2 * rv);
                } else {
                    atomicAdd(&bp[J - 1], 2.f * w2 * rv);
                    atomicAdd(&bp[J - 2], -w2 * rv);
                }
            }
        }
    }
    float e = 0.f;
#pragma unroll
    for (int a = 0; a < NQ; ++a) e = fmaf(th[a].x, u[a].x, fmaf(th[a].y, u[a].y, e));
    const double es = block_sum((double)(wgt * e), red);
    if (threadIdx.x == 0) epart[blockIdx.x] = es;
#pragma unroll
    for (int q = 0; q < NQ / 4; ++q) {
        Q[q * qstride + 2 * r] =
            make_float4(u[4 * q].x * invN, u[4 * q].y * invN, u[4 * q + 1].x * invN, u[4 * q + 1].y * invN);
        Q[q * qstride + 2 * r + 1] =
            make_float4(u[4 * q + 2].x * invN, u[4 * q + 2].y * invN, u[4 * q + 3].x * invN, u[4 * q + 3].y * invN);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < LRN_P * J; i += blockDim.x)
        if (bins[i] != 0.f) atomicAdd(&gK[i], (double)bins[i]);
}

// ---------------------------------------------------------------------------
// L3: assembly of Eq. (Vi), one thread per point (packed order)
// ---------------------------------------------------------------------------
// The inverse plane transforms of u_m have left N3 x N1 real rows at the start
// of each plane of the spectrum buffer.  Per point: v_loc and g from the 8 u
// values and the coefficients the network pass stored in lw.
// mode 0: v_loc to v, w = g grad n to w_out; mode 1: v_loc to v, g to g_out
// (the plane transforms of w follow in k_w_planes).
// 40 registers, six blocks per SM: 0.053 ms at 180 x 180 x 72 against
// 0.076 ms at 80 registers and three blocks (a stream of 26 loads per point)
__global__ void __launch_bounds__(256, 6) k_learned_usum(const float* __restrict__ uf, const float* __restrict__ grad,
                                                      GridArgs g, const float* __restrict__ lw, float* __restrict__ v,
                                                      float* __restrict__ w_out, float* __restrict__ g_out, int mode) {
    const long long N = g.N;
    const long long fstride = 2LL * g.N2 * g.ncols;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        int y, z, x, j;
        const long long gi = packed_point(q, g, y, z, x, j);
        const float* up = uf + 2LL * y * g.ncols + (long long)z * g.N1 + x;
        float vl = lw[2 * LRN_M * N + q], gg = lw[(2 * LRN_M + 1) * N + q];
#pragma unroll
        for (int m = 0; m < LRN_M; ++m) {
            const float u = up[m * fstride];
            vl = fmaf(u, lw[m * N + q], vl);
            gg = fmaf(u, lw[(LRN_M + m) * N + q], gg);
        }
        if (v) v[gi] = vl;
        if (mode == 0 && w_out) {
            w_out[gi] = gg * grad[gi];
            w_out[N + gi] = gg * grad[N + gi];
            w_out[2 * N + gi] = gg * grad[2 * N + gi];
        }
        if (mode == 1) g_out[gi] = gg;
    }
}

// real-space u_m of the in-place planes -> U[m][N] (flat order), for the
// parameter gradient
__global__ void __launch_bounds__(256) k_u_fields(const float* __restrict__ uf, GridArgs g, float* __restrict__ U) {
    const long long N = g.N;
    const long long fstride = 2LL * g.N2 * g.ncols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        flat_point(i, g, x, y, z);
        const float* up = uf + 2LL * y * g.ncols + (long long)z * g.N1 + x;
#pragma unroll
        for (int m = 0; m < LRN_M; ++m) U[m * N + i] = up[m * fstride];
    }
}

// ---------------------------------------------------------------------------
// network outputs alone (tests, fitting): w_m at every point
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(L_THREADS, 1) k_learned_channels(const float* __restrict__ n,
                                                                   const float* __restrict__ grad, long long N,
                                                                   PointParams P, LearnedArgs la,
                                                                   float* __restrict__ wout) {
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ MlpCtl ctl;
    __shared__ float qm[MAX_NQ];
    for (int i = threadIdx.x; i < MAX_NQ; i += blockDim.x) qm[i] = P.qm[i];
    const float n_min = P.n_min;
    MlpShared* S = reinterpret_cast<MlpShared*>(smraw);
    MlpWG* Wb = reinterpret_cast<MlpWG*>(smraw + sizeof(MlpShared));
    const int wg = threadIdx.x >> 7, r = threadIdx.x & 127;
    mlp_load_weights(S, la);
    mlp_setup(&ctl, 128);
    uint32_t phase = 0;
    const long long ntiles = (N + L_TILE - 1) / L_TILE;
    for (long long T = 2 * (long long)blockIdx.x + wg; T < ntiles; T += 2 * (long long)gridDim.x) {
        const long long i = T * L_TILE + r;
        const bool in = i < N;
        float ni = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        if (in) {
            ni = n[i];
            gx = grad[i];
            gy = grad[N + i];
            gz = grad[2 * N + i];
        }
        const Feat f = features(ni, gx, gy, gz, la, n_min);
        const bool ok = in && f.ok;
        float pb[LRN_M], dpb[LRN_M];
#pragma unroll
        for (int m = 0; m < LRN_M; ++m) pb[m] = 0.f;
        if (ok && la.base) {
            const QPoint qp = q_point(ni, gx, gy, gz, P, qm);
            if (qp.k != K_INVALID) base_weights(qp.q, la, pb, dpb, la.bMq);
        }
        float o[LRN_M];
        if (!mlp_forward(S, Wb + wg, &ctl, wg, r, phase, ok ? f.x1 : 0.f, ok ? f.x2 : 0.f, o, la.err)) break;
        if (in)
#pragma unroll
            for (int m = 0; m < LRN_M; ++m) wout[m * N + i] = ok ? o[m] + pb[m] : 0.f;
    }
    mlp_teardown(&ctl);
}

// ---------------------------------------------------------------------------
// parameter gradient through the network (CUDA cores, FP32, FP64 totals)
// ---------------------------------------------------------------------------
// mode 0 (energy): cotangent of w_m at point i is coef dOmega n_i U[m][i];
// mode 1 (fit):    coef 2 wt_i (w_m - T[m][i]) for the loss sum_i wt_i |w - T|^2.
constexpr int PG_TILE = 128;
constexpr int PG_THREADS = 256;
constexpr int PG_LD = LRN_H + 1;  // padded row of the per-point tiles

__global__ void __launch_bounds__(PG_THREADS, 1) k_learned_param_grad(
    const float* __restrict__ n, const float* __restrict__ grad, long long N, float n_min, LearnedArgs la,
    const float* __restrict__ cot, const float* __restrict__ wt, int mode, float coef, double* __restrict__ gout) {
    extern __shared__ float smf[];
    float* W2 = smf;                          // [H][H]
    float* W3 = W2 + LRN_H * LRN_H;           // [M][H]
    float* w1 = W3 + LRN_M * LRN_H;           // [H][2]
    float* b1 = w1 + 2 * LRN_H;
    float* b2 = b1 + LRN_H;
    float* b3 = b2 + LRN_H;                   // [M] (padded to 8)
    float* H1 = b3 + LRN_M;                   // [TILE][LD]
    float* H2 = H1 + PG_TILE * PG_LD;         // [TILE][LD]; later delta z1
    float* DZ2 = H2 + PG_TILE * PG_LD;        // [TILE][LD]
    float* DO = DZ2 + PG_TILE * PG_LD;        // [TILE][M]
    float* X = DO + PG_TILE * LRN_M;          // [TILE][2]
    const int t = threadIdx.x;
    for (int i = t; i < LRN_H * LRN_H; i += PG_THREADS) W2[i] = la.w2r[i];
    for (int i = t; i < LRN_M * LRN_H; i += PG_THREADS) W3[i] = la.w3r[i];
    for (int i = t; i < 2 * LRN_H; i += PG_THREADS) w1[i] = la.w1[i];
    for (int i = t; i < LRN_H; i += PG_THREADS) {
        b1[i] = la.b1[i];
        b2[i] = la.b2[i];
    }
    if (t < LRN_M) b3[t] = la.b3[t];
    // accumulators: dW2[o][i0..i0+15] (o = t / 4, i0 = 16 (t % 4)), dW3[m][j0, j0+1]
    // (m = t / 32, j0 = 2 (t % 32)), db2[o] (t % 4 == 0), db3 (t < M),
    // dW1[j][c] and db1[j] for t < 64 (j = t)
    float aW2[16], aW3[2], ab2 = 0.f, ab3 = 0.f, aW1[2] = {0.f, 0.f}, ab1 = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) aW2[q] = 0.f;
    aW3[0] = aW3[1] = 0.f;
    const float dOmegaCoef = coef;
    const long long ntiles = (N + PG_TILE - 1) / PG_TILE;
    for (long long T = blockIdx.x; T < ntiles; T += gridDim.x) {
        __syncthreads();
        if (t < PG_TILE) {
            const long long i = T * PG_TILE + t;
            const bool in = i < N;
            float ni = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
            if (in) {
                ni = n[i];
                gx = grad[i];
                gy = grad[N + i];
                gz = grad[2 * N + i];
            }
            const Feat f = features(ni, gx, gy, gz, la, n_min);
            const bool ok = in && f.ok;
            const float x1 = ok ? f.x1 : 0.f, x2 = ok ? f.x2 : 0.f;
            X[2 * t] = x1;
            X[2 * t + 1] = x2;
            float* h1 = H1 + t * PG_LD;
            for (int j = 0; j < LRN_H; ++j)
                h1[j] = bf16r(silu(fmaf(w1[2 * j], x1, fmaf(w1[2 * j + 1], x2, b1[j]))));
            float* h2 = H2 + t * PG_LD;
            float* dz2 = DZ2 + t * PG_LD;
            for (int o = 0; o < LRN_H; ++o) {
                float z = b2[o];
                for (int j = 0; j < LRN_H; ++j) z = fmaf(W2[o * LRN_H + j], h1[j], z);
                dz2[o] = z;  // pre-activation, replaced by its delta below
                h2[o] = bf16r(silu(z));
            }
            float dout[LRN_M];
            for (int m = 0; m < LRN_M; ++m) {
                float d = 0.f;
                if (ok) {
                    if (mode == 0) {
                        d = dOmegaCoef * ni * cot[m * N + i];
                    } else {
                        float om = b3[m];
                        for (int j = 0; j < LRN_H; ++j) om = fmaf(W3[m * LRN_H + j], h2[j], om);
                        d = dOmegaCoef * 2.f * wt[i] * (om - cot[m * N + i]);
                    }
                }
                dout[m] = d;
                DO[t * LRN_M + m] = d;
            }
            for (int o = 0; o < LRN_H; ++o) {
                float dh = 0.f;
                for (int m = 0; m < LRN_M; ++m) dh = fmaf(W3[m * LRN_H + o], dout[m], dh);
                dz2[o] = dh * silu_prime(dz2[o]);
            }
        }
        __syncthreads();
        {
            const int o = t >> 2, i0 = 16 * (t & 3);
            for (int p = 0; p < PG_TILE; ++p) {
                const float d = DZ2[p * PG_LD + o];
                const float* h1 = H1 + p * PG_LD + i0;
#pragma unroll
                for (int q = 0; q < 16; ++q) aW2[q] = fmaf(d, h1[q], aW2[q]);
                if ((t & 3) == 0) ab2 += d;
            }
            const int m = t >> 5, j0 = 2 * (t & 31);
            for (int p = 0; p < PG_TILE; ++p) {
                const float d = DO[p * LRN_M + m];
                aW3[0] = fmaf(d, H2[p * PG_LD + j0], aW3[0]);
                aW3[1] = fmaf(d, H2[p * PG_LD + j0 + 1], aW3[1]);
                if (t < LRN_M) ab3 += DO[p * LRN_M + t];
            }
        }
        __syncthreads();
        if (t < PG_TILE) {
            // delta z1 = (W2^T delta z2) * silu'(z1), into this point's H2 row
            const float x1 = X[2 * t], x2 = X[2 * t + 1];
            const float* dz2 = DZ2 + t * PG_LD;
            float* dz1 = H2 + t * PG_LD;
            for (int j = 0; j < LRN_H; ++j) {
                float dh = 0.f;
                for (int o = 0; o < LRN_H; ++o) dh = fmaf(W2[o * LRN_H + j], dz2[o], dh);
                dz1[j] = dh * silu_prime(fmaf(w1[2 * j], x1, fmaf(w1[2 * j + 1], x2, b1[j])));
            }
        }
        __syncthreads();
        if (t < LRN_H) {
            for (int p = 0; p < PG_TILE; ++p) {
                const float d = H2[p * PG_LD + t];
                aW1[0] = fmaf(d, X[2 * p], aW1[0]);
                aW1[1] = fmaf(d, X[2 * p + 1], aW1[1]);
                ab1 += d;
            }
        }
    }
    {
        const int o = t >> 2, i0 = 16 * (t & 3);
#pragma unroll
        for (int q = 0; q < 16; ++q) atomicAdd(&gout[LRN_OFF_W2 + o * LRN_H + i0 + q], (double)aW2[q]);
        if ((t & 3) == 0) atomicAdd(&gout[LRN_OFF_B2 + o], (double)ab2);
        const int m = t >> 5, j0 = 2 * (t & 31);
        atomicAdd(&gout[LRN_OFF_W3 + m * LRN_H + j0], (double)aW3[0]);
        atomicAdd(&gout[LRN_OFF_W3 + m * LRN_H + j0 + 1], (double)aW3[1]);
        if (t < LRN_M) atomicAdd(&gout[LRN_OFF_B3 + t], (double)ab3);
        if (t < LRN_H) {
            atomicAdd(&gout[LRN_OFF_W1 + 2 * t], (double)aW1[0]);
            atomicAdd(&gout[LRN_OFF_W1 + 2 * t + 1], (double)aW1[1]);
            atomicAdd(&gout[LRN_OFF_B1 + t], (double)ab1);
        }
    }
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double a, int n) {
    for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < n; i += blockDim.x * gridDim.x) y[i] += a * x[i];
}

// ---------------------------------------------------------------------------
// plain cardinal weights p_a(q(n, |grad n|)) at every point (fitting targets)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_basis_weights(const float* __restrict__ n, const float* __restrict__ grad,
                                                       long long N, PointParams P, float* __restrict__ out) {
    __shared__ SplineSmem sp;
    load_spline_smem(&sp, P);
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const QPoint qp = q_point(n[i], grad[i], grad[N + i], grad[2 * N + i], P, sp.qm);
        for (int a = 0; a < P.Nq; ++a) out[a * N + i] = qp.k == K_INVALID ? 0.f : cardinal_value(&sp, a, qp.k, qp.t);
    }
}

// ---------------------------------------------------------------------------
// spectral gradient: grad f = IFFT(i G f(G)), Nyquist components removed
// ---------------------------------------------------------------------------
template <int CN1, int CN3>
__global__ void __launch_bounds__(PLANE_THREADS, 2) k_field_plane(const float* __restrict__ f, GridArgs g,
                                                                   const Tw* __restrict__ tw,
                                                                   float2* __restrict__ spec) {
    extern __shared__ float2 sm[];
    float2* plane = sm;
    Tw* tw1 = twiddles_after(plane, (size_t)(g.N3 * g.Nh));
    Tw* tw3 = tw1 + g.N1;
    const int y = blockIdx.x;
    load_line_twiddles<CN1>(tw1, tw, g.N1);
    load_line_twiddles<CN3>(tw3, tw + g.N1 + g.N2, g.N3);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long zs = (long long)g.N1 * g.N2;  // flat distance between rows z and z + 1
    for (int jr = warp; jr < (g.N3 >> 1); jr += nw) {
        const long long row = (long long)g.N1 * (y + (long long)g.N2 * 2 * jr);
        float2* crow = plane + jr * 2 * g.Nh;
        for (int x = lane; x < g.N1; x += 32) crow[x] = make_float2(f[row + x], f[row + zs + x]);
    }
    __syncthreads();
    plane_forward<CN1, CN3>(plane, g, tw1, tw3);
    float2* dst = spec + (long long)y * g.ncols;
    for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) dst[i] = plane[i];
}

template <int CN2>
__global__ void __launch_bounds__(256, 2) k_pencil_grad(const float2* __restrict__ spec, float2* __restrict__ wspec,
                                                        GridArgs g, const Tw* __restrict__ tw, int C) {
    extern __shared__ float2 sm[];
    const int N2 = CN2 > 0 ? CN2 : g.N2;
    float2* lines = sm;  // [4][C][N2]: the field, then its three derivatives
    Tw* tw2 = twiddles_after(lines, (size_t)(4 * C * N2));
    load_line_twiddles<CN2>(tw2, tw + g.N1, N2);
    const int c0 = blockIdx.x * C;
    const SmallDiv sC = small_div(C);  // i / C in the staging loops
    for (int i = threadIdx.x; i < N2 * C; i += blockDim.x) {
        const int yy = sdiv(i, sC), cc = i - yy * C;
        const int col = c0 + cc;
        lines[cc * N2 + yy] = col < g.ncols ? spec[(long long)yy * g.ncols + col] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    pencils_fft<CN2, false>(lines, C, N2, g.p2, tw2);
    __syncthreads();
    for (int pt = threadIdx.x; pt < C * N2; pt += blockDim.x) {
        const int cc = pt / N2, yy = pt % N2;
        const int col = c0 + cc;
        const int kx = col % g.Nh, kz = col / g.Nh;
        const int mx = (2 * kx == g.N1) ? 0 : kx;
        const int my = (2 * yy == N2) ? 0 : ((2 * yy < N2) ? yy : yy - N2);
        const int mz = (2 * kz == g.N3) ? 0 : ((2 * kz < g.N3) ? kz : kz - g.N3);
        const float2 fv = lines[cc * N2 + yy];
        const float G[3] = {g.gx * mx, g.gy * my, g.gz * mz};
#pragma unroll
        for (int c = 0; c < 3; ++c)  // i G f / N
            lines[((1 + c) * C + cc) * N2 + yy] = make_float2(-G[c] * fv.y * g.invN, G[c] * fv.x * g.invN);
    }
    __syncthreads();
    pencils_fft<CN2, true>(lines + C * N2, 3 * C, N2, g.p2, tw2);
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * N2 * C; i += blockDim.x) {
        const int rr = sdiv(i, sC), cc = i - rr * C, yy = rr % N2, c = rr / N2;
        const int col = c0 + cc;
        if (col < g.ncols) wspec[((long long)c * N2 + yy) * g.ncols + col] = lines[((1 + c) * C + cc) * N2 + yy];
    }
}

template <int CN1, int CN3>
__global__ void __launch_bounds__(PLANE_THREADS, 2) k_plane_inv3(const float2* __restrict__ wspec, GridArgs g,
                                                                  const Tw* __restrict__ tw,
                                                                  float* __restrict__ out) {
    extern __shared__ float2 sm[];
    float2* plane = sm;
    Tw* tw1 = twiddles_after(plane, (size_t)(g.N3 * g.Nh));
    Tw* tw3 = tw1 + g.N1;
    const int y = blockIdx.x, c = blockIdx.y;
    load_line_twiddles<CN1>(tw1, tw, g.N1);
    load_line_twiddles<CN3>(tw3, tw + g.N1 + g.N2, g.N3);
    const float2* src = wspec + ((long long)c * g.N2 + y) * g.ncols;
    for (int i = threadIdx.x; i < g.ncols; i += blockDim.x) plane[i] = src[i];
    __syncthreads();
    plane_inverse<CN1, CN3>(plane, g, tw1, tw3);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long zs = (long long)g.N1 * g.N2;
    float* oc = out + c * g.N;
    for (int jr = warp; jr < (g.N3 >> 1); jr += nw) {
        const long long row = (long long)g.N1 * (y + (long long)g.N2 * 2 * jr);
        const float2* crow = plane + jr * 2 * g.Nh;
        for (int x = lane; x < g.N1; x += 32) {
            const float2 d = crow[x];
            oc[row + x] = d.x;
            oc[row + zs + x] = d.y;
        }
    }
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba) on FP32 parameters with FP64 gradients
// ---------------------------------------------------------------------------
__global__ void k_adam(float* __restrict__ p, const double* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2) {
    for (long long i = threadIdx.x + blockIdx.x * (long long)blockDim.x; i < n; i += (long long)blockDim.x * gridDim.x) {
        const float gi = (float)g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// the network kernel: its shared block and the three warpgroups' operands.
// It allocates all 512 tensor-memory columns of its SM, so the request is at
// least 116 KB: a second block never fits beside it.
size_t smem_net() { return std::max(sizeof(MlpShared) + L_NET_WG * sizeof(MlpWG3), (size_t)116 * 1024); }
// network blocks: one per SM, at most the partial-sum slots of the epart scratch
int net_blocks(vdw_ctx* c) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, std::min(nsm, c->g.N2 * L_SLOTS));
}
// blocks of the table lookup: grid-stride over the points, at most the
// partial-sum slots the network kernel has
// one wave of resident blocks (grid-stride loop), within the partial-sum slots
int lookup_blocks(vdw_ctx* c) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_learned_lookup, LOOKUP_THREADS, 0) != cudaSuccess)
            b = 1;
        per_sm = std::max(1, b);
    }
    const long long want = (c->g.N + LOOKUP_THREADS - 1) / LOOKUP_THREADS;
    const long long wave = (long long)std::max(1, c->nsm) * per_sm;
    return (int)std::max(1LL, std::min(std::min(want, wave), (long long)c->g.N2 * L_SLOTS));
}
// knot-gradient bins of k_learned_contract_gradk
size_t smem_gradk(int J) { return sizeof(float) * (size_t)LRN_P * J; }
size_t smem_plane1(const GridArgs& g) {
    return sizeof(float2) * tw_offset((size_t)g.N3 * g.Nh) + sizeof(Tw) * (g.N1 + g.N3);
}
size_t smem_pgrad() {
    return sizeof(float) * ((size_t)LRN_H * LRN_H + LRN_M * LRN_H + 2 * LRN_H + 2 * LRN_H + LRN_M +
                            3 * (size_t)PG_TILE * PG_LD + PG_TILE * LRN_M + 2 * PG_TILE);
}
constexpr int GRAD_COLS = 8;
size_t smem_pgrad_pencil(const GridArgs& g) {
    return sizeof(float2) * tw_offset((size_t)4 * GRAD_COLS * g.N2) + sizeof(Tw) * g.N2;
}
const size_t SMEM_LIMIT = 227 * 1024 - 4 * 1024;

template <class K>
int set_smem(K kernel, size_t bytes, const char* name) {
    if (bytes > SMEM_LIMIT) {
        set_error(std::string(name) + ": shared memory beyond the limit");
        return VDW_ERR_SIZE;
    }
    return raise_smem_limit(kernel, bytes);
}

template <int CN1, int CN2, int CN3>
int configure(vdw_ctx* c) {
    const GridArgs& g = c->g;
    int rc = set_smem(k_learned_net, smem_net(), "k_learned_net");
    if (!rc) rc = set_smem(k_learned_contract_gradk, smem_gradk(c->lrn_J), "k_learned_contract_gradk");
    if (!rc) rc = set_smem(k_field_plane<CN1, CN3>, smem_plane1(g), "k_field_plane");
    if (!rc) rc = set_smem(k_plane_inv3<CN1, CN3>, smem_plane1(g), "k_plane_inv3");
    if (!rc) rc = set_smem(k_pencil_grad<CN2>, smem_pgrad_pencil(g), "k_pencil_grad");
    if (!rc) rc = set_smem(k_learned_param_grad, smem_pgrad(), "k_learned_param_grad");
    return rc;
}

int configure_all(vdw_ctx* c) {
    const GridArgs& g = c->g;
    if (g.N1 == 180 && g.N2 == 180 && g.N3 == 72) return configure<180, 180, 72>(c);
    if (g.N1 == 256 && g.N2 == 256 && g.N3 == 96) return configure<256, 256, 96>(c);
    return configure<0, 0, 0>(c);
}

// learned scratch: partial sums [N2 * 8 + nb_sorted]
double* lrn_epart(vdw_ctx* c) {
    return reinterpret_cast<double*>(static_cast<unsigned char*>(c->d_lrn) + 0);
}

enum RunKind { RUN_ENERGY = 0, RUN_GRAD = 1 };

template <int CN1, int CN2, int CN3>
int run(vdw_ctx* c, const float* n, const float* grad, double* E, float* v, float* w, int kind, double coef,
        double* gout, cudaStream_t s) {
    const GridArgs& g = c->g;
    const PointParams& P = c->pp;
    const LearnedArgs& la = c->la;
    // the inference form takes the network from its table when there is one;
    // the training form (parameter gradients) always runs the network
    const bool lookup = la.tabT > 0 && kind != RUN_GRAD;
    const int nb0 = lookup ? lookup_blocks(c) : net_blocks(c);
    double* ep = lrn_epart(c);
    float* specf = reinterpret_cast<float*>(c->d_spec);
    const double Omega = c->L[0] * c->L[1] * c->L[2];
    // stage marks for vdw_profile_read (the network kernel is stage 0; the
    // divergence pencils and final planes are one mark)
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
    const bool want_pot = (v != nullptr) || (w != nullptr);
    if (lookup)
        k_learned_lookup<<<nb0, LOOKUP_THREADS, 0, s>>>(n, grad, g, P, la, specf, ep, c->d_invalid,
                                                       want_pot ? c->d_lw : nullptr);
    else
        k_learned_net<<<nb0, L_NET_THREADS, smem_net(), s>>>(n, grad, g, P, la, specf, ep, c->d_invalid,
                                                         (want_pot && kind != RUN_GRAD) ? c->d_lw : nullptr);
    mark(ST_POINTWISE);
    int rc = pipeline_planes_inplace(c, LRN_M, false, s);
    if (rc) return rc;
    mark(ST_PLANES_FWD);
    rc = sorted_forward(c, LRN_M, s);
    if (rc) return rc;
    mark(ST_PENCILS_FWD);
    if (kind == RUN_GRAD) {
        VDW_CUDA(cudaMemsetAsync(c->d_gK, 0, sizeof(double) * LRN_P * c->lrn_J, s));
        k_learned_contract_gradk<<<c->nb_sorted, SORTED_BLOCK, smem_gradk(c->lrn_J), s>>>(
            c->d_Q, 2 * c->Npad, c->d_gs, la, g.invN, ep + nb0, c->d_gK,
            (float)(0.5 * Omega / ((double)g.N * (double)g.N)));
        VDW_CUDA(cudaGetLastError());
    } else {
        rc = sorted_contract_table(c, LRN_M, la.knots, la.inv_dk, la.J, ep + nb0, want_pot ? 1 : 0, s);
        if (rc) return rc;
    }
    mark(ST_CONTRACT);
    // as in the plain path: with a potential to follow (and no stage timing)
    // the energy reduction runs on the side stream beside the inverse
    // transforms, joined before the call returns
    bool forked = false;
    auto join = [&]() {
        if (forked) cudaStreamWaitEvent(s, c->ev_join, 0);
        forked = false;
    };
    if (E) {
        cudaStream_t se = s;
        if (want_pot && kind != RUN_GRAD && !c->prof) {
            VDW_CUDA(cudaEventRecord(c->ev_fork, s));
            VDW_CUDA(cudaStreamWaitEvent(c->s_side, c->ev_fork, 0));
            se = c->s_side;
        }
        rc = pipeline_energy_final(c, ep, nb0, c->nb_sorted, E, se);
        if (se != s) {
            VDW_CUDA(cudaEventRecord(c->ev_join, se));
            forked = true;
        }
        if (rc) {
            join();
            return rc;
        }
        mark(ST_ENERGY);
    }
    const int nb_pt = (int)std::min<long long>((g.N + 255) / 256, 1 << 16);
    if (kind == RUN_GRAD || want_pot) {
        rc = sorted_inverse(c, LRN_M, s);
        if (rc) {
            join();
            return rc;
        }
        mark(ST_PENCILS_INV);
    }
    if (kind == RUN_GRAD) {
        rc = pipeline_planes_inplace(c, LRN_M, true, s);
        if (rc) return rc;
        k_u_fields<<<nb_pt, 256, 0, s>>>(specf, g, c->d_U);
        const double dOmega = Omega / (double)g.N;
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        k_learned_param_grad<<<nsm, PG_THREADS, smem_pgrad(), s>>>(n, grad, g.N, P.n_min, la, c->d_U, nullptr, 0,
                                                                   (float)(coef * dOmega), gout);
        k_axpy<<<36, 256, 0, s>>>(gout + LRN_OFF_K, c->d_gK, coef, LRN_P * c->lrn_J);
    } else if (want_pot) {
        const int mode = (w != nullptr) ? 0 : 1;
        rc = pipeline_planes_inplace(c, LRN_M, true, s);
        if (!rc) {
            mark(ST_PLANES_INV);
            k_learned_usum<<<nb_pt, 256, 0, s>>>(specf, grad, g, c->d_lw, v, w, c->d_gg, mode);
            mark(ST_USUM);
        }
        if (!rc && mode == 1) {
            rc = pipeline_w_planes(c, grad, s);
            if (!rc) {
                mark(ST_W_PLANES);
                rc = pipeline_divergence(c, v, s);
            }
            if (!rc) mark(ST_DIV_FINAL);
        }
        join();
        if (rc) return rc;
    }
    join();
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int run_any(vdw_ctx* c, const float* n, const float* grad, double* E, float* v, float* w, int kind, double coef,
            double* gout, cudaStream_t s) {
    const GridArgs& g = c->g;
    if (g.N1 == 180 && g.N2 == 180 && g.N3 == 72) return run<180, 180, 72>(c, n, grad, E, v, w, kind, coef, gout, s);
    if (g.N1 == 256 && g.N2 == 256 && g.N3 == 96) return run<256, 256, 96>(c, n, grad, E, v, w, kind, coef, gout, s);
    return run<0, 0, 0>(c, n, grad, E, v, w, kind, coef, gout, s);
}

template <int CN1, int CN2, int CN3>
void spectral_gradient(vdw_ctx* c, const float* f, float* out, cudaStream_t s) {
    const GridArgs& g = c->g;
    k_field_plane<CN1, CN3><<<g.N2, PLANE_THREADS, smem_plane1(g), s>>>(f, g, c->d_tw, c->d_spec);
    k_pencil_grad<CN2><<<(g.ncols + GRAD_COLS - 1) / GRAD_COLS, 256, smem_pgrad_pencil(g), s>>>(
        c->d_spec, c->d_wspec, g, c->d_tw, GRAD_COLS);
    k_plane_inv3<CN1, CN3><<<dim3(g.N2, 3), PLANE_THREADS, smem_plane1(g), s>>>(c->d_wspec, g, c->d_tw, out);
}

bool lrn_ready(vdw_ctx* c) {
    if (!c->planned) {
        set_error("no plan");
        return false;
    }
    if (!c->lrn_loaded) {
        set_error("no learned model loaded");
        return false;
    }
    return true;
}

}  // namespace

// Size of the learned context's allocation and its layout (256-byte aligned pieces).
struct LrnLayout {
    size_t epart, w1, b1, b2, b3, w2r, w3r, w2f, w3f, knots, err, gK, total;
};
static LrnLayout lrn_layout(const GridArgs& g, int J, int nb_sorted) {
    LrnLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 255) & ~(size_t)255;
        return at;
    };
    // energy partials: the network blocks (at most N2 L_SLOTS), then the
    // contraction's blocks over the sorted points
    L.epart = take(sizeof(double) * ((size_t)g.N2 * L_SLOTS + (size_t)nb_sorted + 1));
    L.w1 = take(sizeof(float) * 2 * LRN_H);
    L.b1 = take(sizeof(float) * LRN_H);
    L.b2 = take(sizeof(float) * LRN_H);
    L.b3 = take(sizeof(float) * LRN_M);
    L.w2r = take(sizeof(float) * LRN_H * LRN_H);
    L.w3r = take(sizeof(float) * LRN_M * LRN_H);
    L.w2f = take(2 * LRN_H * LRN_H);
    L.w3f = take(2 * LRN_N3 * LRN_H);
    L.knots = take(sizeof(float4) * (size_t)(J - 1) * LRN_P);
    L.err = take(sizeof(int));
    L.gK = take(sizeof(double) * (size_t)LRN_P * J);
    L.total = o;
    return L;
}

void learned_free(vdw_ctx* c) {
    cudaFree(c->d_lrn_tab);
    c->d_lrn_tab = nullptr;
    c->lrn_tab_bytes = 0;
    c->la.tabT = 0;
    c->la.tab = nullptr;
    cudaFree(c->d_lrn);
    cudaFree(c->d_U);
    cudaFree(c->d_lw);
    c->d_lrn = nullptr;
    c->d_U = nullptr;
    c->d_lw = nullptr;
    c->d_gK = nullptr;
    c->lrn_loaded = 0;
}

int learned_run(vdw_ctx* c, const float* n, const float* grad, double* E, float* v, float* w, cudaStream_t s) {
    if (!lrn_ready(c)) return VDW_ERR_STATE;
    if ((v || w) && !c->d_lw) VDW_CUDA(cudaMalloc(&c->d_lw, sizeof(float) * (2 * LRN_M + 2) * (size_t)c->g.N));
    return run_any(c, n, grad, E, v, w, RUN_ENERGY, 0.0, nullptr, s);
}

}  // namespace vdw

using namespace vdw;

extern "C" {

long long vdw_learned_param_count(int J) { return (long long)LRN_OFF_K + (long long)LRN_P * J; }

int vdw_learned_load(vdw_handle c, int J, double k_max, const double feat[5], double base_q1, double base_lambda,
                     const float* params, void* stream) {
    if (!c || !feat || !params || J < 4 || J > L_MAXJ || !(k_max > 0.0)) return VDW_ERR_ARG;
    if (base_q1 > 0.0 && !(base_q1 < c->p.q_c && base_lambda > 0.0 && base_lambda != 1.0)) return VDW_ERR_ARG;
    if (!c->planned) {
        set_error("vdw_learned_load: plan the grid first");
        return VDW_ERR_STATE;
    }
    if (!(feat[1] > 0.0) || !(feat[3] > 0.0) || !(feat[4] > 0.0)) return VDW_ERR_ARG;
    const GridArgs& g = c->g;
    const double PI_D = 3.14159265358979323846;
    const double gmax = 2.0 * PI_D * std::sqrt(std::pow((g.N1 / 2) / c->L[0], 2) + std::pow((g.N2 / 2) / c->L[1], 2) +
                                               std::pow((g.N3 / 2) / c->L[2], 2));
    if (gmax > k_max) {
        set_error("vdw_learned_load: largest |G| of the grid exceeds the knots' k_max");
        return VDW_ERR_SIZE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->d_lrn || c->lrn_J != J) {
        cudaFree(c->d_lrn);
        c->d_lrn = nullptr;
        const LrnLayout L = lrn_layout(g, J, c->nb_sorted);
        VDW_CUDA(cudaMalloc(&c->d_lrn, L.total));
        VDW_CUDA(cudaMemset(c->d_lrn, 0, L.total));
        unsigned char* b = static_cast<unsigned char*>(c->d_lrn);
        LearnedArgs& la = c->la;
        la.w1 = reinterpret_cast<float*>(b + L.w1);
        la.b1 = reinterpret_cast<float*>(b + L.b1);
        la.b2 = reinterpret_cast<float*>(b + L.b2);
        la.b3 = reinterpret_cast<float*>(b + L.b3);
        la.w2r = reinterpret_cast<float*>(b + L.w2r);
        la.w3r = reinterpret_cast<float*>(b + L.w3r);
        la.w2f = reinterpret_cast<uint16_t*>(b + L.w2f);
        la.w3f = reinterpret_cast<uint16_t*>(b + L.w3f);
        la.knots = reinterpret_cast<float4*>(b + L.knots);
        la.err = c->d_flags + 1;
        c->d_gK = reinterpret_cast<double*>(b + L.gK);
        c->lrn_J = J;
    }
    LearnedArgs& la = c->la;
    la.J = J;
    la.dk = (float)(k_max / (J - 1));
    la.inv_dk = (float)((J - 1) / k_max);
    la.mu1 = (float)feat[0];
    la.inv_sig1 = (float)(1.0 / feat[1]);
    la.mu2 = (float)feat[2];
    la.inv_sig2 = (float)(1.0 / feat[3]);
    la.eps2 = (float)(feat[4] * feat[4]);
    c->lrn_kmax = k_max;
    la.base = base_q1 > 0.0 ? 1 : 0;
    if (la.base) {
        // base mesh q_a = q_1 + (q_c - q_1)(lambda^a - 1)/(lambda^(M-1) - 1) and its
        // cardinal natural splines (second derivatives by the tridiagonal solve)
        double qb[LRN_M], Mb[LRN_M][LRN_M];
        const double den = std::pow(base_lambda, LRN_M - 1) - 1.0;
        for (int a = 0; a < LRN_M; ++a)
            qb[a] = base_q1 + (c->p.q_c - base_q1) * (std::pow(base_lambda, a) - 1.0) / den;
        for (int a = 0; a < LRN_M; ++a) {
            double cp[LRN_M], dd[LRN_M];
            for (int i = 0; i < LRN_M; ++i) Mb[a][i] = 0.0;
            for (int i = 1; i <= LRN_M - 2; ++i) {
                const double h0 = qb[i] - qb[i - 1], h1 = qb[i + 1] - qb[i];
                const double y0 = (i - 1 == a), y1 = (i == a), y2 = (i + 1 == a);
                const double rhs = 6.0 * ((y2 - y1) / h1 - (y1 - y0) / h0);
                const double lo = (i > 1) ? h0 : 0.0;
                const double dn = 2.0 * (h0 + h1) - (i > 1 ? lo * cp[i - 1] : 0.0);
                cp[i] = h1 / dn;
                dd[i] = (rhs - (i > 1 ? lo * dd[i - 1] : 0.0)) / dn;
            }
            for (int i = LRN_M - 2; i >= 1; --i) Mb[a][i] = dd[i] - (i < LRN_M - 2 ? cp[i] * Mb[a][i + 1] : 0.0);
        }
        for (int a = 0; a < LRN_M; ++a) {
            la.bqm[a] = (float)qb[a];
            for (int k = 0; k < LRN_M; ++k) la.bMq[a * LRN_M + k] = (float)Mb[a][k];
        }
    }
    k_learned_prepare<<<16, 256, 0, s>>>(params, la);
    VDW_CUDA(cudaGetLastError());
    const int rc = configure_all(c);
    if (rc) return rc;
    c->la.tabT = 0;  // a table made for the previous parameters no longer applies
    c->lrn_loaded = 1;
    return VDW_OK;
}

int vdw_learned_energy_potential(vdw_handle c, const float* n, const float* grad, double* E, float* v, float* w,
                                 void* stream) {
    if (!c || !n || !grad) return VDW_ERR_ARG;
    if (c->planned)
        if (const int rw = check_wait(c)) return rw;
    return learned_run(c, n, grad, E, v, w, (cudaStream_t)stream);
}

int vdw_learned_param_grad(vdw_handle c, const float* n, const float* grad, double coef, double* g_params, double* E,
                           void* stream) {
    if (!c || !n || !grad || !g_params) return VDW_ERR_ARG;
    if (!lrn_ready(c)) return VDW_ERR_STATE;
    if (const int rw = check_wait(c)) return rw;
    if (!c->d_U) VDW_CUDA(cudaMalloc(&c->d_U, sizeof(float) * LRN_M * (size_t)c->g.N));
    return run_any(c, n, grad, E, nullptr, nullptr, RUN_GRAD, coef, g_params, (cudaStream_t)stream);
}

int vdw_learned_fit_grad(vdw_handle c, const float* n, const float* grad, const float* target, const float* weight,
                         double coef, double* g_params, void* stream) {
    if (!c || !n || !grad || !target || !weight || !g_params) return VDW_ERR_ARG;
    if (!lrn_ready(c)) return VDW_ERR_STATE;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (const int rs = raise_smem_limit(k_learned_param_grad, smem_pgrad())) return rs;
    k_learned_param_grad<<<nsm, PG_THREADS, smem_pgrad(), (cudaStream_t)stream>>>(
        n, grad, c->g.N, c->pp.n_min, c->la, target, weight, 1, (float)coef, g_params);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int vdw_learned_channels(vdw_handle c, const float* n, const float* grad, float* w_out, void* stream) {
    if (!c || !n || !grad || !w_out) return VDW_ERR_ARG;
    if (!lrn_ready(c)) return VDW_ERR_STATE;
    const size_t sm = sizeof(MlpShared) + 2 * sizeof(MlpWG);
    if (const int rs = raise_smem_limit(k_learned_channels, sm)) return rs;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (c->g.N + 2 * L_TILE - 1) / (2 * L_TILE);
    const int nb = (int)std::min<long long>(tiles, 2LL * nsm);
    k_learned_channels<<<nb, L_THREADS, sm, (cudaStream_t)stream>>>(n, grad, c->g.N, c->pp, c->la, w_out);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int vdw_learned_tabulate(vdw_handle c, int T, double D, void* stream) {
    if (!c || T < 0 || T == 1 || T == 2 || T == 3 || T > 4096 || (T > 0 && !(D > 0.0))) return VDW_ERR_ARG;
    if (!lrn_ready(c)) return VDW_ERR_STATE;
    LearnedArgs& la = c->la;
    if (T == 0) {
        la.tabT = 0;
        return VDW_OK;
    }
    const size_t bytes = sizeof(float4) * 2 * (size_t)(T + 2) * (size_t)(T + 2);
    if (bytes != c->lrn_tab_bytes) {
        cudaFree(c->d_lrn_tab);
        c->d_lrn_tab = nullptr;
        c->lrn_tab_bytes = 0;
        VDW_CUDA(cudaMalloc(&c->d_lrn_tab, bytes));
        c->lrn_tab_bytes = bytes;
    }
    la.tab = c->d_lrn_tab;
    la.tabT = T;
    la.tabD = (float)D;
    la.tab_h = (float)(2.0 * D / (T - 1));
    la.tab_inv_h = (float)((T - 1) / (2.0 * D));
    const size_t sm = sizeof(MlpShared) + 2 * sizeof(MlpWG);
    if (const int rs = raise_smem_limit(k_learned_tabulate, sm)) return rs;
    const long long tiles = ((long long)(T + 2) * (T + 2) + L_TILE - 1) / L_TILE;
    const int nb = (int)std::max(1LL, std::min<long long>((tiles + 1) / 2, 2LL * std::max(c->nsm, 1)));
    k_learned_tabulate<<<nb, L_THREADS, sm, (cudaStream_t)stream>>>(la, c->d_lrn_tab);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int vdw_learned_status(vdw_handle c, int* tc_error) {
    if (!c || !tc_error) return VDW_ERR_ARG;
    if (!c->lrn_loaded) return VDW_ERR_STATE;
    VDW_CUDA(cudaDeviceSynchronize());
    *tc_error = (((volatile int*)c->h_flags)[1] || c->wait_seen) ? 1 : 0;
    return VDW_OK;
}

int vdw_basis_weights(vdw_handle c, const float* n, const float* grad, float* p_out, void* stream) {
    if (!c || !n || !grad || !p_out) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    const int nb = (int)std::min<long long>((c->g.N + 255) / 256, 4096);
    k_basis_weights<<<nb, 256, 0, (cudaStream_t)stream>>>(n, grad, c->g.N, c->pp, p_out);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int vdw_spectral_gradient(vdw_handle c, const float* f, float* grad, void* stream) {
    if (!c || !f || !grad) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    const GridArgs& g = c->g;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = VDW_OK;
    if (g.N1 == 180 && g.N2 == 180 && g.N3 == 72) {
        rc = set_smem(k_field_plane<180, 72>, smem_plane1(g), "k_field_plane");
        if (!rc) rc = set_smem(k_plane_inv3<180, 72>, smem_plane1(g), "k_plane_inv3");
        if (!rc) rc = set_smem(k_pencil_grad<180>, smem_pgrad_pencil(g), "k_pencil_grad");
        if (!rc) spectral_gradient<180, 180, 72>(c, f, grad, s);
    } else if (g.N1 == 256 && g.N2 == 256 && g.N3 == 96) {
        rc = set_smem(k_field_plane<256, 96>, smem_plane1(g), "k_field_plane");
        if (!rc) rc = set_smem(k_plane_inv3<256, 96>, smem_plane1(g), "k_plane_inv3");
        if (!rc) rc = set_smem(k_pencil_grad<256>, smem_pgrad_pencil(g), "k_pencil_grad");
        if (!rc) spectral_gradient<256, 256, 96>(c, f, grad, s);
    } else {
        rc = set_smem(k_field_plane<0, 0>, smem_plane1(g), "k_field_plane");
        if (!rc) rc = set_smem(k_plane_inv3<0, 0>, smem_plane1(g), "k_plane_inv3");
        if (!rc) rc = set_smem(k_pencil_grad<0>, smem_pgrad_pencil(g), "k_pencil_grad");
        if (!rc) spectral_gradient<0, 0, 0>(c, f, grad, s);
    }
    if (rc) return rc;
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int vdw_adam_step(float* p, const double* g, float* m, float* v, long long count, double lr, double beta1,
                  double beta2, double eps, int step, void* stream) {
    if (!p || !g || !m || !v || count <= 0 || step < 1) return VDW_ERR_ARG;
    const float bc1 = (float)(1.0 - std::pow(beta1, step)), bc2 = (float)(1.0 - std::pow(beta2, step));
    const int nb = (int)std::min<long long>((count + 255) / 256, 1024);
    k_adam<<<nb, 256, 0, (cudaStream_t)stream>>>(p, g, m, v, count, (float)lr, (float)beta1, (float)beta2,
                                                 (float)eps, bc1, bc2);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

}  // extern "C"
