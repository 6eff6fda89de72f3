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
//
// Every constant of a transform (table twiddles, the sines and cosines inside
// the radix 3, 5, 8, 9 and 16 butterflies) is held as a pair hi + lo of FP32
// numbers whose sum is the FP64 value, and a product x W is formed as
// x W_hi + x W_lo.  With the constants rounded to FP32 alone, the rounding
// errors of the few twiddles a smooth field's low frequencies go through add
// up coherently: the transform's low-frequency amplitudes come out biased by
// a few 1e-8, which shifts the energy of Eq. (Eoffk) (dominated by those
// frequencies) by ~1e-7 of itself.  With the pair the constants are exact to
// ~1e-15 and only the (unbiased) rounding of the arithmetic remains.
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

// A twiddle W as {W_hi.x, W_hi.y, W_lo.x, W_lo.y}, W = W_hi + W_lo.
using Tw = float4;
// a W (the small product a W_lo first, then the main one accumulated on it)
__device__ __forceinline__ float2 cmul_tw(float2 a, Tw w) {
    const float lr = fmaf(a.x, w.z, -a.y * w.w);
    const float li = fmaf(a.x, w.w, a.y * w.z);
    return make_float2(fmaf(a.x, w.x, fmaf(-a.y, w.y, lr)), fmaf(a.x, w.y, fmaf(a.y, w.x, li)));
}
// a conj(W)
__device__ __forceinline__ float2 cmulc_tw(float2 a, Tw w) {
    const float lr = fmaf(a.x, w.z, a.y * w.w);
    const float li = fmaf(a.y, w.z, -a.x * w.w);
    return make_float2(fmaf(a.x, w.x, fmaf(a.y, w.y, lr)), fmaf(a.y, w.x, fmaf(-a.x, w.y, li)));
}
template <bool INV>
__device__ __forceinline__ float2 tw_mul(float2 a, Tw w) {
    return INV ? cmulc_tw(a, w) : cmul_tw(a, w);
}
// A twiddle held as its FP32 value only (transforms whose results tolerate
// the constant rounding: the inverse transforms and those of w).
template <bool INV>
__device__ __forceinline__ float2 tw_mul(float2 a, float2 w) {
    return INV ? cmulc(a, w) : cmul(a, w);
}
// store a hi/lo twiddle as a table entry of either kind
__device__ __forceinline__ void tw_put(Tw* d, Tw s) { *d = s; }
__device__ __forceinline__ void tw_put(float2* d, Tw s) { *d = make_float2(s.x, s.y); }
// Real constant c = hi + lo from its FP64 value.
struct KPair {
    float h, l;
};
__host__ __device__ constexpr KPair kpair(double c) { return KPair{(float)c, (float)(c - (double)(float)c)}; }
// x c
__device__ __forceinline__ float kmul(float x, KPair c) { return fmaf(x, c.h, x * c.l); }
// x c + y d (one rounding of the main products' sum)
__device__ __forceinline__ float kmul2(float x, KPair c, float y, KPair d) {
    return fmaf(x, c.h, fmaf(y, d.h, fmaf(x, c.l, y * d.l)));
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
    constexpr KPair s3 = kpair(0.86602540378443864676);  // sin(2 pi/3)
    float2 s = cadd(v[1], v[2]);
    float2 d = csub(v[1], v[2]);
    float2 x0 = cadd(v[0], s);
    float2 t = make_float2(fmaf(-0.5f, s.x, v[0].x), fmaf(-0.5f, s.y, v[0].y));
    const float2 dm = mul_mi<INV>(d);
    float2 u = make_float2(kmul(dm.x, s3), kmul(dm.y, s3));
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
    constexpr KPair c1 = kpair(0.30901699437494742410);   // cos(2 pi/5)
    constexpr KPair c2 = kpair(-0.80901699437494742410);  // cos(4 pi/5)
    constexpr KPair s1 = kpair(0.95105651629515357212);   // sin(2 pi/5)
    constexpr KPair s2 = kpair(0.58778525229247312917);   // sin(4 pi/5)
    constexpr KPair ms1 = kpair(-0.95105651629515357212);
    float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    float2 x0 = cadd(v[0], cadd(a1, a2));
    float2 t1 = make_float2(v[0].x + kmul2(a1.x, c1, a2.x, c2), v[0].y + kmul2(a1.y, c1, a2.y, c2));
    float2 t2 = make_float2(v[0].x + kmul2(a1.x, c2, a2.x, c1), v[0].y + kmul2(a1.y, c2, a2.y, c1));
    float2 u1 = mul_mi<INV>(make_float2(kmul2(b1.x, s1, b2.x, s2), kmul2(b1.y, s1, b2.y, s2)));
    float2 u2 = mul_mi<INV>(make_float2(kmul2(b1.x, s2, b2.x, ms1), kmul2(b1.y, s2, b2.y, ms1)));
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

template <int R, bool INV, class W>
__device__ __forceinline__ void line_pass(float2* p, int es, int n, int Ns, const W* tw, int lane) {
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
                const W w = tw[r * k * tstride];  // r k n/(Ns R) < n
                v[b][r] = tw_mul<INV>(v[b][r], w);
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

// Full line transform: tw holds W_n^e = exp(-2 pi i e/n), e in [0, n), as hi/lo pairs.  One
// loop per radix keeps each pass's registers separate.
template <bool INV, class W>
__device__ __forceinline__ void line_fft(float2* p, int es, const LinePlan& pl, const W* tw, int lane) {
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
    constexpr KPair r2 = kpair(0.70710678118654752440);
    // two radix-4 transforms of the even and odd samples
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    // odd twiddles W8^k, k = 1..3 (conjugate for the inverse)
    const float s = INV ? 1.f : -1.f;
    const float2 o1 = make_float2(kmul(o[1].x - s * o[1].y, r2), kmul(o[1].y + s * o[1].x, r2));
    const float2 o2 = make_float2(-s * o[2].y, s * o[2].x);
    const float2 o3 = make_float2(kmul(-o[3].x - s * o[3].y, r2), kmul(-o[3].y + s * o[3].x, r2));
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

// ---- composite radices, evaluated in registers ----------------------------
// W_N^e = exp(-2 pi i e / N) (conjugated for the inverse) for the few
// exponents the Cooley-Tukey splits 3x3 and 4x4 need.
template <int N, int E>
__device__ __forceinline__ Tw wconst() {
    static_assert(N == 9 || N == 16, "no constants for this length");
    double c = 1.0, s = 0.0;  // cos, sin of 2 pi E / N
    if (N == 9) {
        if (E == 1) { c = 0.766044443118978035202; s = 0.642787609686539326323; }
        if (E == 2) { c = 0.173648177666930348852; s = 0.984807753012208059367; }
        if (E == 4) { c = -0.939692620785908384054; s = 0.342020143325668733044; }
    } else {
        if (E == 1) { c = 0.923879532511286756128; s = 0.382683432365089771728; }
        if (E == 2) { c = 0.707106781186547524401; s = 0.707106781186547524401; }
        if (E == 3) { c = 0.382683432365089771728; s = 0.923879532511286756128; }
        if (E == 4) { c = 0.0; s = 1.0; }
        if (E == 6) { c = -0.707106781186547524401; s = 0.707106781186547524401; }
        if (E == 9) { c = -0.923879532511286756128; s = -0.382683432365089771728; }
    }
    const KPair cr = kpair(c), ci = kpair(-s);
    return make_float4(cr.h, ci.h, cr.l, ci.l);
}

// Cooley-Tukey in registers, N = R1 R2, input index R2 n1 + n2, output
// k1 + R1 k2: R2 transforms of length R1, twiddles W_N^(n2 k1), R1
// transforms of length R2.
template <int R1, int R2, bool INV, int N2 = 0, int K1 = 1>
__device__ __forceinline__ void ct_twiddle(float2 (&Y)[R1 * R2]) {
    if constexpr (N2 < R2) {
        if constexpr (K1 < R1) {
            if constexpr (N2 > 0) {
                const Tw w = wconst<R1 * R2, N2 * K1>();
                Y[N2 * R1 + K1] = tw_mul<INV>(Y[N2 * R1 + K1], w);
            }
            ct_twiddle<R1, R2, INV, N2, K1 + 1>(Y);
        } else {
            ct_twiddle<R1, R2, INV, N2 + 1, 1>(Y);
        }
    }
}

template <int R1, int R2, bool INV>
__device__ __forceinline__ void dft_ct(float2* v) {
    float2 Y[R1 * R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
        float2 t[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + n2];
        dft<R1, INV>(t);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) Y[n2 * R1 + k1] = t[k1];
    }
    ct_twiddle<R1, R2, INV>(Y);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        float2 t[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) t[n2] = Y[n2 * R1 + k1];
        dft<R2, INV>(t);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[k2];
    }
}

constexpr int inv_mod(int a, int m) {
    for (int x = 1; x < m; ++x)
        if ((a * x) % m == 1) return x;
    return 1;
}

// Good-Thomas (prime-factor) split for coprime R1, R2: input index
// (R2 n1 + R1 n2) mod N, output index by the Chinese remainder theorem; no
// twiddles between the two sets of short transforms.
template <int R1, int R2, bool INV>
__device__ __forceinline__ void dft_pfa(float2* v) {
    constexpr int N = R1 * R2;
    constexpr int i1 = inv_mod(R2 % R1, R1), i2 = inv_mod(R1 % R2, R2);
    float2 Y[N];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
        float2 t[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[(R2 * n1 + R1 * n2) % N];
        dft<R1, INV>(t);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) Y[n2 * R1 + k1] = t[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        float2 t[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) t[n2] = Y[n2 * R1 + k1];
        dft<R2, INV>(t);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[(k1 * R2 * i1 + k2 * R1 * i2) % N] = t[k2];
    }
}

template <> __device__ __forceinline__ void dft<6, false>(float2* v) { dft_pfa<2, 3, false>(v); }
template <> __device__ __forceinline__ void dft<6, true>(float2* v) { dft_pfa<2, 3, true>(v); }
template <> __device__ __forceinline__ void dft<9, false>(float2* v) { dft_ct<3, 3, false>(v); }
template <> __device__ __forceinline__ void dft<9, true>(float2* v) { dft_ct<3, 3, true>(v); }
template <> __device__ __forceinline__ void dft<10, false>(float2* v) { dft_pfa<2, 5, false>(v); }
template <> __device__ __forceinline__ void dft<10, true>(float2* v) { dft_pfa<2, 5, true>(v); }
template <> __device__ __forceinline__ void dft<12, false>(float2* v) { dft_pfa<4, 3, false>(v); }
template <> __device__ __forceinline__ void dft<12, true>(float2* v) { dft_pfa<4, 3, true>(v); }
template <> __device__ __forceinline__ void dft<15, false>(float2* v) { dft_pfa<5, 3, false>(v); }
template <> __device__ __forceinline__ void dft<15, true>(float2* v) { dft_pfa<5, 3, true>(v); }
template <> __device__ __forceinline__ void dft<16, false>(float2* v) { dft_ct<4, 4, false>(v); }
template <> __device__ __forceinline__ void dft<16, true>(float2* v) { dft_ct<4, 4, true>(v); }

// Radix schedule of a compile-time length: the first radix is the one (among
// the in-register lengths) that leaves the fewest passes, the larger on a tie.
// maxr caps the radix (register pressure in kernels that hold much else).
constexpr int CT_RADICES[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
constexpr int ct_passes_greedy(int n, int maxr);
constexpr int ct_radix(int n, int maxr = 16) {
    int best = 0, bestp = 1 << 20, bestd = 1 << 20;
    for (int r : CT_RADICES) {
        if (r > maxr || n % r != 0) continue;
        const int p = 1 + ct_passes_greedy(n / r, maxr);
        const int d = r > n / r ? r - n / r : n / r - r;  // prefer balanced splits
        if (p < bestp || (p == bestp && d < bestd)) {
            bestp = p;
            bestd = d;
            best = r;
        }
    }
    return best;
}
constexpr int ct_passes_greedy(int n, int maxr) {
    if (n <= 1) return 0;
    for (int r : CT_RADICES)
        if (r <= maxr && n % r == 0) return 1 + ct_passes_greedy(n / r, maxr);
    return 1 << 20;
}
constexpr int ct_npasses(int n, int maxr = 16) { return n <= 1 ? 0 : 1 + ct_npasses(n / ct_radix(n, maxr), maxr); }
// radix of pass s (in order) and the product Ns of the radices before it
constexpr int ct_radix_at(int n, int s, int maxr = 16) {
    return s == 0 ? ct_radix(n, maxr) : ct_radix_at(n / ct_radix(n, maxr), s - 1, maxr);
}
constexpr int ct_ns_at(int n, int s, int maxr = 16) {
    return s == 0 ? 1 : ct_radix(n, maxr) * ct_ns_at(n / ct_radix(n, maxr), s - 1, maxr);
}
// largest butterfly count N / R over the passes, and the lines one warp
// transforms together so that its lanes stay busy
constexpr int ct_max_m(int n, int maxr = 16, int s = 0) {
    return s >= ct_npasses(n, maxr) ? 0
                                    : (n / ct_radix_at(n, s, maxr) > ct_max_m(n, maxr, s + 1) ? n / ct_radix_at(n, s, maxr)
                                                                                                : ct_max_m(n, maxr, s + 1));
}
// (two lines of at most 16 butterflies go one per half-warp, see ct_pass)
constexpr int ct_lines_per_warp(int n, int maxr = 16) {
    const int m = ct_max_m(n, maxr);
    if (m <= 16) return 2;
    const int l = 32 / m;
    return l < 1 ? 1 : (l > 4 ? 4 : l);
}

// Twiddle table of a compile-time length N, laid out by pass: pass s with
// Ns > 1 keeps W_N^(r k TS) (r = 1 .. R-1, k = 0 .. Ns-1, TS = N/(Ns R)) at
// ct_tw_off(N, s) + (r - 1) Ns + k, so that the lanes of a pass, which take
// consecutive k, read consecutive entries (no bank conflicts).  At most N
// entries in all.
constexpr int ct_tw_off(int n, int s, int maxr = 16) {
    return s == 0 ? 0
                  : ct_tw_off(n, s - 1, maxr) +
                        (ct_ns_at(n, s - 1, maxr) > 1 ? (ct_radix_at(n, s - 1, maxr) - 1) * ct_ns_at(n, s - 1, maxr) : 0);
}
// Fills the table from the plain one (src[e] = W_N^e), all threads of the block.
template <int N, int MAXR = 16, int S = 0, class W>
__device__ __forceinline__ void ct_load_twiddles(W* dst, const Tw* src) {
    if constexpr (S < ct_npasses(N, MAXR)) {
        constexpr int R = ct_radix_at(N, S, MAXR), Ns = ct_ns_at(N, S, MAXR);
        if constexpr (Ns > 1) {
            constexpr int TS = N / (Ns * R), off = ct_tw_off(N, S, MAXR);
            for (int i = threadIdx.x; i < (R - 1) * Ns; i += blockDim.x) {
                const int r = 1 + i / Ns, k = i - (r - 1) * Ns;
                tw_put(dst + off + i, src[r * k * TS]);
            }
        }
        ct_load_twiddles<N, MAXR, S + 1>(dst, src);
    }
}

// One pass over L lines (line l at p + l*ls, element stride es) by one warp.
// Two lines of at most 16 butterflies go one per half-warp: a 64-bit shared
// access is served per half-warp, so the two lines never compete for banks
// whatever their distance, and consecutive butterflies of one line hit
// distinct banks.  The first pass (Ns = 1) has no twiddles; the others read
// the pass-ordered table of ct_load_twiddles.
template <int N, int S, int L, bool INV, int MAXR, class W>
__device__ __forceinline__ void ct_pass(float2* p, int es, int ls, const W* tw, int lane) {
    constexpr int R = ct_radix_at(N, S, MAXR);
    constexpr int Ns = ct_ns_at(N, S, MAXR);
    constexpr int M = N / R;
    constexpr int TOT = L * M;
    constexpr bool HALF = (L == 2) && (M <= 16);
    constexpr int B = HALF ? 1 : (TOT + 31) / 32;
    float2 v[B][R];
    int lj[B][2];
    bool act[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if constexpr (HALF) {
            lj[b][0] = lane >> 4;
            lj[b][1] = lane & 15;
            act[b] = (M == 16) || lj[b][1] < M;
        } else {
            const int t0 = lane + 32 * b;
            act[b] = (TOT % 32 == 0) || t0 < TOT;
            const int t = act[b] ? t0 : 0;  // in-range index for tail lanes
            lj[b][0] = t / M;
            lj[b][1] = t - lj[b][0] * M;
        }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if (act[b]) {
            const int l = lj[b][0], j = lj[b][1];
            const int k = j % Ns;
            const float2* q = p + l * ls;
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = q[(j + r * M) * es];
            if constexpr (Ns > 1) {
                constexpr int off = ct_tw_off(N, S, MAXR);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const W w = tw[off + (r - 1) * Ns + k];
                    v[b][r] = tw_mul<INV>(v[b][r], w);
                }
            }
            dft<R, INV>(v[b]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if (act[b]) {
            const int l = lj[b][0], j = lj[b][1];
            const int k = j % Ns;
            float2* q = p + l * ls;
            const int base = (j - k) * R + k;
            if constexpr (HALF && Ns == 1 && R == 16) {
                // the outputs of butterfly j go to 16 j + r: with the same r in
                // every lane the 16 lanes of a half-warp would hit one bank.
                // Rotate each lane's outputs by j (four conditional rotations
                // by 1, 2, 4, 8) so that step r' stores output (r' + j) mod 16.
#pragma unroll
                for (int bit = 0; bit < 4; ++bit) {
                    const bool rot = (j >> bit) & 1;
                    float2 t[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) t[r] = v[b][(r + (1 << bit)) & (R - 1)];
#pragma unroll
                    for (int r = 0; r < R; ++r) v[b][r] = rot ? t[r] : v[b][r];
                }
#pragma unroll
                for (int r = 0; r < R; ++r) q[(base + ((r + j) & (R - 1))) * es] = v[b][r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) q[(base + r * Ns) * es] = v[b][r];
            }
        }
    }
    __syncwarp();
}

template <int N, int L, bool INV, int MAXR = 16, int S = 0, class W>
__device__ __forceinline__ void ct_fft(float2* p, int es, int ls, const W* tw, int lane) {
    if constexpr (S < ct_npasses(N, MAXR)) {
        ct_pass<N, S, L, INV, MAXR>(p, es, ls, tw, lane);
        ct_fft<N, L, INV, MAXR, S + 1>(p, es, ls, tw, lane);
    }
}

}  // namespace vdw
