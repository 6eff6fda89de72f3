// Pointwise chain of the method, FP32: q0(n, |grad n|) (Dion et al., with the
// Perdew-Wang 1992 LDA correlation), saturation h(q0, q_c) of Eq. (Sat), the
// interval of the logarithmic q mesh and the cardinal cubic splines p_a of
// Eq. (fofx) with their q derivatives.
#pragma once

#include "common.cuh"

namespace vdw {

struct QPoint {
    float q;      // saturated q, clamped to the mesh
    float dq_dn;  // d q / d n
    float dq_dg;  // (d q / d|grad n|) / |grad n|
    float t;      // (q - q_k) / (q_{k+1} - q_k)
    int k;        // mesh interval, or K_INVALID when theta = 0
};

// S = sum_{m=1}^{mc} y^m / m and dS/dy = sum_{m=0}^{mc-1} y^m by Horner's rule
// (inv_m[m] = 1/m).
template <int MC>
__device__ __forceinline__ void saturation_sum(float y, const float* inv_m, float& S, float& dS) {
    float a = inv_m[MC], d = 1.f;
#pragma unroll
    for (int m = MC - 1; m >= 1; --m) {
        a = fmaf(a, y, inv_m[m]);
        d = fmaf(d, y, 1.f);
    }
    S = a * y;
    dS = d;
}
__device__ __forceinline__ void saturation_sum_n(float y, int mc, const float* inv_m, float& S, float& dS) {
    float a = inv_m[mc], d = 1.f;
    for (int m = mc - 1; m >= 1; --m) {
        a = fmaf(a, y, inv_m[m]);
        d = fmaf(d, y, 1.f);
    }
    S = a * y;
    dS = d;
}

// qm: the q mesh (Nq values), normally a shared-memory copy of P.qm so that
// the divergent interval search does not serialise on the constant bank.
__device__ __forceinline__ QPoint q_point(float n, float gx, float gy, float gz, const PointParams& P,
                                          const float* qm) {
    QPoint r;
    if (!(n > P.n_min) || !isfinite(n)) {
        r.q = qm[0]; r.dq_dn = 0.f; r.dq_dg = 0.f; r.t = 0.f; r.k = K_INVALID;
        return r;
    }
    const float PI_F = 3.14159265358979f;
    const float A = 0.031091f, a1 = 0.21370f;
    const float b1 = 7.5957f, b2 = 3.5876f, b3 = 1.6382f, b4 = 0.49294f;
    const float Z = -0.8491f;
    // one cube root: k_F = (3 pi^2 n)^(1/3), r_s = (3 / (4 pi n))^(1/3)
    const float cb = cbrtf(n);
    const float icb = 1.0f / cb;
    const float kF = 3.0936677262801355f * cb;   // (3 pi^2)^(1/3) n^(1/3)
    const float rs = 0.6203504908994001f * icb;  // (3 / (4 pi))^(1/3) n^(-1/3)
    const float ikF = 0.323240919347991f * icb;  // 1 / k_F
    const float g2 = gx * gx + gy * gy + gz * gz;
    const float inv_n = 1.0f / n;
    const float s2 = g2 * (0.25f * inv_n * inv_n) * (ikF * ikF);
    const float rsq = rsqrtf(rs);
    const float srs = rs * rsq;  // sqrt(r_s)
    const float Q = 2.f * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
    const float dQ = 2.f * A * (0.5f * b1 * rsq + b2 + 1.5f * b3 * srs + 2.f * b4 * rs);
    const float Lg = log1pf(1.0f / Q);
    const float ec = -2.f * A * (1.f + a1 * rs) * Lg;
    const float dec = -2.f * A * a1 * Lg + 2.f * A * (1.f + a1 * rs) * dQ / (Q * Q + Q);
    const float q0 = kF * (1.f - Z / 9.f * s2) - 4.f * PI_F / 3.f * ec;
    const float dq0_dn = kF * inv_n * (1.f / 3.f) - Z / 9.f * (kF * s2 * inv_n * (1.f / 3.f) - kF * 8.f * s2 * inv_n * (1.f / 3.f))
                         + 4.f * PI_F / 3.f * dec * rs * inv_n * (1.f / 3.f);
    const float dq0_dg = -Z / 18.f * ikF * inv_n * inv_n;
    // saturation: h = q_c (1 - exp(-S)), S = sum_{m=1}^{m_c} y^m/m, y = q0/q_c.
    // For y > 4 exp(-S) is far below the FP32 (and FP64) range: h = q_c, h' = 0.
    const float y = q0 / P.q_c;
    float h, hp;
    if (y > 4.f) {
        h = P.q_c; hp = 0.f;
    } else {
        float S, dS;
        if (P.m_c == 12) saturation_sum<12>(y, P.inv_m, S, dS);  // Dion et al.'s choice, unrolled
        else saturation_sum_n(y, P.m_c, P.inv_m, S, dS);
        // 1 - exp(-S) through expm1: no cancellation for small q0
        const float em1 = expm1f(-S);
        h = -P.q_c * em1;
        hp = (1.f + em1) * dS;
    }
    // below the mesh q is clamped to q_1 and no longer varies with n, grad n
    if (h < qm[0]) hp = 0.f;
    float q = fminf(fmaxf(h, qm[0]), qm[P.Nq - 1]);
    // interval: number of knots <= q, minus one, in [0, Nq-2]
    int lo = 0, hi = P.Nq - 1;  // invariant: qm[lo] <= q (or lo = 0), answer in [lo, hi)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (qm[mid] <= q) lo = mid; else hi = mid;
    }
    r.k = lo;
    r.t = (q - qm[lo]) / (qm[lo + 1] - qm[lo]);
    r.q = q;
    r.dq_dn = hp * dq0_dn;
    r.dq_dg = hp * dq0_dg;
    return r;
}

// Shared-memory copy of the spline tables: qm[MAX_NQ], Mq[a][k] as
// Mq[a * MAX_NQ + k].  Indexing them by the per-point interval k from the
// constant bank would serialise the warp.
struct SplineSmem {
    float qm[MAX_NQ];
    float Mq[MAX_NQ * MAX_NQ];
    float ih[MAX_NQ];   // 1 / h_k, h_k = q_{k+1} - q_k
    float h26[MAX_NQ];  // h_k^2 / 6
    float h6[MAX_NQ];   // h_k / 6
};

__device__ __forceinline__ void load_spline_smem(SplineSmem* sp, const PointParams& P) {
    for (int i = threadIdx.x; i < MAX_NQ; i += blockDim.x) {
        sp->qm[i] = P.qm[i];
        const float h = (i + 1 < P.Nq) ? P.qm[i + 1] - P.qm[i] : 1.f;
        sp->ih[i] = 1.f / h;
        sp->h26[i] = h * h * (1.f / 6.f);
        sp->h6[i] = h * (1.f / 6.f);
    }
    for (int i = threadIdx.x; i < MAX_NQ * MAX_NQ; i += blockDim.x) sp->Mq[i] = P.Mq[i / MAX_NQ][i % MAX_NQ];
}

// p_a and dp_a/dq on interval k at local position t.
__device__ __forceinline__ void cardinal(const SplineSmem* sp, int a, int k, float t, float& pa, float& dpa) {
    const float A = 1.f - t, B = t;
    const float M0 = sp->Mq[a * MAX_NQ + k], M1 = sp->Mq[a * MAX_NQ + k + 1];
    const float y0 = (a == k) ? 1.f : 0.f, y1 = (a == k + 1) ? 1.f : 0.f;
    pa = A * y0 + B * y1 + ((A * A * A - A) * M0 + (B * B * B - B) * M1) * sp->h26[k];
    dpa = (y1 - y0) * sp->ih[k] + ((3.f * B * B - 1.f) * M1 - (3.f * A * A - 1.f) * M0) * sp->h6[k];
}

__device__ __forceinline__ float cardinal_value(const SplineSmem* sp, int a, int k, float t) {
    const float A = 1.f - t, B = t;
    const float M0 = sp->Mq[a * MAX_NQ + k], M1 = sp->Mq[a * MAX_NQ + k + 1];
    const float y0 = (a == k) ? 1.f : 0.f, y1 = (a == k + 1) ? 1.f : 0.f;
    return A * y0 + B * y1 + ((A * A * A - A) * M0 + (B * B * B - B) * M1) * sp->h26[k];
}

}  // namespace vdw
