// Warp-per-line mixed-radix FFTs on shared memory (sm_103a).
//
// One warp transforms one line of complex FP32 values held in shared memory
// (any element stride), in place, by Stockham autosort passes of radix 4, 2,
// 3 or 5: in each pass every lane loads its butterflies' inputs into
// registers, the warp synchronises, and the lanes write the outputs to their
// autosorted positions.  Lines are independent, so a block spreads its lines
// over its warps with no block-wide barrier between passes.
//
// Pass (radix R, Ns = product of the previous radices, m = n/R butterflies):
//   for j in [0, m):  k = j mod Ns
//     v_r = x[j + r m] * W_n^{r k n/(Ns R)}        (W_n = exp(-2 pi i/n))
//     V   = DFT_R(v)
//     y[(j - k) R + k + r Ns] = V_r
// Forward uses W_n, inverse its conjugate; neither scales.
#pragma once

#include "common.cuh"

namespace vdw {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// -i a (forward) or +i a (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v);

template <>
__device__ __forceinline__ void dft<2, false>(float2* v) {
    float2 a = cadd(v[0], v[1]), b = csub(v[0], v[1]);
    v[0] = a; v[1] = b;
}
template <>
__device__ __forceinline__ void dft<2, true>(float2* v) { dft<2, false>(v); }

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
    const float s3 = 0.86602540378443864676f;  // sin(2 pi/3)
    float2 s = cadd(v[1], v[2]);
    float2 d = csub(v[1], v[2]);
    float2 x0 = cadd(v[0], s);
    float2 t = make_float2(fmaf(-0.5f, s.x, v[0].x), fmaf(-0.5f, s.y, v[0].y));
    float2 u = cscale(mul_mi<INV>(d), s3);
    v[0] = x0;
    v[1] = cadd(t, u);
    v[2] = csub(t, u);
}
template <>
__device__ __forceinline__ void dft<3, false>(float2* v) { dft3<false>(v); }
template <>
__device__ __forceinline__ void dft<3, true>(float2* v) { dft3<true>(v); }

template <bool INV>
__device__ __forceinline__ void dft4(float2* v) {
    float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    float2 c = cadd(v[1], v[3]), d = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
}
template <>
__device__ __forceinline__ void dft<4, false>(float2* v) { dft4<false>(v); }
template <>
__device__ __forceinline__ void dft<4, true>(float2* v) { dft4<true>(v); }

template <bool INV>
__device__ __forceinline__ void dft5(float2* v) {
    const float c1 = 0.30901699437494742410f;   // cos(2 pi/5)
    const float c2 = -0.80901699437494742410f;  // cos(4 pi/5)
    const float s1 = 0.95105651629515357212f;   // sin(2 pi/5)
    const float s2 = 0.58778525229247312917f;   // sin(4 pi/5)
    float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    float2 x0 = cadd(v[0], cadd(a1, a2));
    float2 t1 = make_float2(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    float2 t2 = make_float2(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    float2 u1 = mul_mi<INV>(make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
    float2 u2 = mul_mi<INV>(make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
    v[0] = x0;
    v[1] = cadd(t1, u1);
    v[4] = csub(t1, u1);
    v[2] = cadd(t2, u2);
    v[3] = csub(t2, u2);
}
template <>
__device__ __forceinline__ void dft<5, false>(float2* v) { dft5<false>(v); }
template <>
__device__ __forceinline__ void dft<5, true>(float2* v) { dft5<true>(v); }

// One Stockham pass of radix R over a line of length n (n <= MAX_DIM), by one warp.
// j mod Ns through a multiply-high: with M = floor((2^32-1)/Ns) + 1 the
// quotient umulhi(j, M) is exact for j < 2048, Ns <= 512 (checked
// exhaustively); Ns = 1 is special-cased.
__device__ __forceinline__ unsigned magic_of(int Ns) { return Ns > 1 ? 0xFFFFFFFFu / (unsigned)Ns + 1u : 0u; }
__device__ __forceinline__ int mod_magic(int j, int Ns, unsigned M) {
    return Ns > 1 ? j - (int)__umulhi((unsigned)j, M) * Ns : 0;
}

template <int R, bool INV>
__device__ __forceinline__ void line_pass(float2* p, int es, int n, int Ns, const float2* tw, int lane) {
    constexpr int MAXB = (MAX_DIM / R + 31) / 32;
    const int m = n / R;
    const int tstride = n / (Ns * R);
    const unsigned M = magic_of(Ns);
    float2 v[MAXB][R];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int j0 = lane + 32 * b;
        const int j = j0 < m ? j0 : 0;  // in-range index for tail lanes
        if (j0 < m) {
            const int k = mod_magic(j, Ns, M);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = p[(j + r * m) * es];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 w = tw[r * k * tstride];  // r k n/(Ns R) < n
                v[b][r] = INV ? cmulc(v[b][r], w) : cmul(v[b][r], w);
            }
            dft<R, INV>(v[b]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int j0 = lane + 32 * b;
        const int j = j0 < m ? j0 : 0;
        if (j0 < m) {
            const int k = mod_magic(j, Ns, M);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) p[(base + r * Ns) * es] = v[b][r];
        }
    }
    __syncwarp();
}

// Full line transform: tw holds W_n^e = exp(-2 pi i e/n), e in [0, n).  One
// loop per radix keeps each pass's registers separate.
template <bool INV>
__device__ __forceinline__ void line_fft(float2* p, int es, const LinePlan& pl, const float2* tw, int lane) {
    int Ns = 1;
#pragma unroll 1
    for (int s = 0; s < pl.c4; ++s) { line_pass<4, INV>(p, es, pl.n, Ns, tw, lane); Ns *= 4; }
#pragma unroll 1
    for (int s = 0; s < pl.c2; ++s) { line_pass<2, INV>(p, es, pl.n, Ns, tw, lane); Ns *= 2; }
#pragma unroll 1
    for (int s = 0; s < pl.c3; ++s) { line_pass<3, INV>(p, es, pl.n, Ns, tw, lane); Ns *= 3; }
#pragma unroll 1
    for (int s = 0; s < pl.c5; ++s) { line_pass<5, INV>(p, es, pl.n, Ns, tw, lane); Ns *= 5; }
}

// Two real rows a, b packed as Z = a + i b, after the forward transform of Z:
// split into the half spectra A[k], B[k], k in [0, N/2], written to p[0..Nh)
// and p[Nh..2Nh) (the region holds 2 Nh = N + 2 values).
__device__ __forceinline__ void r2c_untangle(float2* p, int N, int lane) {
    constexpr int MAXK = (MAX_DIM / 2 + 1 + 31) / 32;
    const int Nh = N / 2 + 1;
    float2 A[MAXK], B[MAXK];
#pragma unroll
    for (int b = 0; b < MAXK; ++b) {
        const int k0 = lane + 32 * b;
        const int k = k0 < Nh ? k0 : 0;  // in-range index for tail lanes
        if (k0 < Nh) {
            const float2 zk = p[k == N ? 0 : k];
            const float2 zm = p[k == 0 ? 0 : N - k];
            // A = (Z_k + conj Z_{-k})/2,  B = -i (Z_k - conj Z_{-k})/2
            A[b] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            B[b] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        }
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < MAXK; ++b) {
        const int k0 = lane + 32 * b;
        const int k = k0 < Nh ? k0 : 0;
        if (k0 < Nh) {
            p[k] = A[b];
            p[Nh + k] = B[b];
        }
    }
    __syncwarp();
}

// Inverse of the above: from half spectra A (p[0..Nh)), B (p[Nh..2Nh)) of two
// real rows build Z[0..N) = A + i B on the full circle (Hermitian extension;
// the imaginary parts of the k = 0 and k = N/2 terms are dropped, as a
// complex-to-real transform does).  The inverse transform of Z then gives
// N a in its real part and N b in its imaginary part.
__device__ __forceinline__ void c2r_tangle(float2* p, int N, int lane) {
    constexpr int MAXK = (MAX_DIM / 2 + 1 + 31) / 32;
    const int Nh = N / 2 + 1;
    float2 A[MAXK], B[MAXK];
#pragma unroll
    for (int b = 0; b < MAXK; ++b) {
        const int k0 = lane + 32 * b;
        const int k = k0 < Nh ? k0 : 0;
        if (k0 < Nh) {
            A[b] = p[k];
            B[b] = p[Nh + k];
            if (k == 0 || 2 * k == N) { A[b].y = 0.f; B[b].y = 0.f; }
        }
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < MAXK; ++b) {
        const int k0 = lane + 32 * b;
        const int k = k0 < Nh ? k0 : 0;
        if (k0 < Nh) {
            p[k] = make_float2(A[b].x - B[b].y, A[b].y + B[b].x);
            if (k >= 1 && 2 * k < N) p[N - k] = make_float2(A[b].x + B[b].y, B[b].x - A[b].y);
        }
    }
    __syncwarp();
}

}  // namespace vdw

// ---------------------------------------------------------------------------
// Compile-time line lengths: the same Stockham passes with constant radices,
// strides and twiddle steps, radix 8 first, and several lines per warp so
// that short lines still fill the 32 lanes.
// ---------------------------------------------------------------------------
namespace vdw {

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
    const float r2 = 0.70710678118654752440f;
    // two radix-4 transforms of the even and odd samples
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    // odd twiddles W8^k, k = 1..3 (conjugate for the inverse)
    const float s = INV ? 1.f : -1.f;
    const float2 o1 = make_float2(r2 * (o[1].x - s * o[1].y), r2 * (o[1].y + s * o[1].x));
    const float2 o2 = make_float2(-s * o[2].y, s * o[2].x);
    const float2 o3 = make_float2(r2 * (-o[3].x - s * o[3].y), r2 * (-o[3].y + s * o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}
template <>
__device__ __forceinline__ void dft<8, false>(float2* v) { dft8<false>(v); }
template <>
__device__ __forceinline__ void dft<8, true>(float2* v) { dft8<true>(v); }

constexpr int ct_radix(int n) {
    return n % 8 == 0 ? 8 : n % 4 == 0 ? 4 : n % 2 == 0 ? 2 : n % 3 == 0 ? 3 : n % 5 == 0 ? 5 : 0;
}
constexpr int ct_npasses(int n) { return n <= 1 ? 0 : 1 + ct_npasses(n / ct_radix(n)); }
// radix of pass s (in order) and the product Ns of the radices before it
constexpr int ct_radix_at(int n, int s) { return s == 0 ? ct_radix(n) : ct_radix_at(n / ct_radix(n), s - 1); }
constexpr int ct_ns_at(int n, int s) { return s == 0 ? 1 : ct_radix(n) * ct_ns_at(n / ct_radix(n), s - 1); }

// One pass over L lines (line l at p + l*ls, element stride es) by one warp.
template <int N, int S, int L, bool INV>
__device__ __forceinline__ void ct_pass(float2* p, int es, int ls, const float2* tw, int lane) {
    constexpr int R = ct_radix_at(N, S);
    constexpr int Ns = ct_ns_at(N, S);
    constexpr int M = N / R;
    constexpr int TS = N / (Ns * R);
    constexpr int TOT = L * M;
    constexpr int B = (TOT + 31) / 32;
    float2 v[B][R];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int t0 = lane + 32 * b;
        const int t = (TOT % 32 == 0 || t0 < TOT) ? t0 : 0;  // in-range index for tail lanes
        if (TOT % 32 == 0 || t0 < TOT) {
            const int l = t / M, j = t - l * M;
            const int k = j % Ns;
            const float2* q = p + l * ls;
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = q[(j + r * M) * es];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 w = tw[r * k * TS];
                v[b][r] = INV ? cmulc(v[b][r], w) : cmul(v[b][r], w);
            }
            dft<R, INV>(v[b]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int t0 = lane + 32 * b;
        const int t = (TOT % 32 == 0 || t0 < TOT) ? t0 : 0;  // in-range index for tail lanes
        if (TOT % 32 == 0 || t0 < TOT) {
            const int l = t / M, j = t - l * M;
            const int k = j % Ns;
            float2* q = p + l * ls;
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) q[(base + r * Ns) * es] = v[b][r];
        }
    }
    __syncwarp();
}

template <int N, int L, bool INV, int S = 0>
__device__ __forceinline__ void ct_fft(float2* p, int es, int ls, const float2* tw, int lane) {
    if constexpr (S < ct_npasses(N)) {
        ct_pass<N, S, L, INV>(p, es, ls, tw, lane);
        ct_fft<N, L, INV, S + 1>(p, es, ls, tw, lane);
    }
}

}  // namespace vdw
