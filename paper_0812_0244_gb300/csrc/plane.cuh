// Shared pieces of the transform kernels: block reductions, twiddle loads,
// dispatch between the compile-time and runtime line transforms, and the
// forward / inverse transform of one y plane (N3 rows of N1 reals <-> N3 x Nh
// half spectrum) held in shared memory.
#pragma once
#include <type_traits>

#include "fft.cuh"

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
__device__ inline double block_sum(double v, double* red) {
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

template <class W>
__device__ __forceinline__ void load_twiddles(W* dst, const Tw* src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw_put(dst + i, src[i]);
}
// Shared-memory twiddles of a line length: the pass-ordered table of the
// compile-time transforms when CN > 0 (CN == n), the plain table otherwise;
// W = Tw keeps the hi/lo pairs, W = float2 the FP32 values only.
template <int CN, class W>
__device__ __forceinline__ void load_line_twiddles(W* dst, const Tw* src, int n) {
    if constexpr (CN > 0) ct_load_twiddles<CN>(dst, src);
    else load_twiddles(dst, src, n);
}

// i / d for a small divisor (1 <= d < 256) and 0 <= i < 2^24 by one
// multiply-high with m = ceil(2^32 / d): the error term i (m d - 2^32) / 2^32 /
// d stays below 1/d, so the quotient is exact in that range.
struct SmallDiv {
    unsigned m;
    int d;
};
__device__ __forceinline__ SmallDiv small_div(int d) {
    SmallDiv s;
    s.d = d;
    s.m = d == 1 ? 0u : 0xFFFFFFFFu / (unsigned)d + 1u;
    return s;
}
__device__ __forceinline__ int sdiv(int i, SmallDiv s) { return s.d == 1 ? i : (int)__umulhi((unsigned)i, s.m); }

// 8-byte asynchronous copy global -> shared memory (cp.async), zero-filled
// instead when !valid (src is then not read; it must still be a mapped
// address).  A thread issues all its copies without waiting on any;
// cp_async_wait_all then waits for the thread's own copies.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
// 4-byte form of the same
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---------------------------------------------------------------------------
// line-transform dispatch: compile-time length when CN > 0
// ---------------------------------------------------------------------------
// the Nh columns of a plane (element stride Nh), several columns per warp for short lines
template <int CN, bool INV, int MAXR = 16, class W>
__device__ __forceinline__ void columns_fft(float2* plane, int Nh, const LinePlan& pl, const W* tw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if constexpr (CN > 0) {
        constexpr int L = ct_lines_per_warp(CN, MAXR);
        const int full = (Nh / L) * L;
        for (int col = warp * L; col < full; col += nw * L) ct_fft<CN, L, INV, MAXR>(plane + col, Nh, 1, tw, lane);
        for (int col = full + warp; col < Nh; col += nw) ct_fft<CN, 1, INV, MAXR>(plane + col, Nh, 1, tw, lane);
    } else {
        for (int col = warp; col < Nh; col += nw) line_fft<INV>(plane + col, Nh, pl, tw, lane);
    }
}

// lines of length N2 (pencils) at a stride of ls values (ls = N2: contiguous),
// several lines per warp for short lines
template <int CN, bool INV, class W>
__device__ __forceinline__ void pencils_fft(float2* lines, int nlines, int N2, const LinePlan& pl, const W* tw,
                                            int ls = 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (ls == 0) ls = N2;
    if constexpr (CN > 0) {
        constexpr int L = ct_lines_per_warp(CN);
        const int full = (nlines / L) * L;
        for (int l = warp * L; l < full; l += nw * L) ct_fft<CN, L, INV>(lines + l * ls, 1, ls, tw, lane);
        for (int l = full + warp; l < nlines; l += nw) ct_fft<CN, 1, INV>(lines + l * ls, 1, 0, tw, lane);
    } else {
        for (int l = warp; l < nlines; l += nw) line_fft<INV>(lines + l * ls, 1, pl, tw, lane);
    }
}

// Line stride of the pencil kernels' shared-memory lines [field][column][y]:
// the staging loops give the 16 lanes of a half-warp 8 columns x 2 rows, at
// (column S + y) float2 values; with S = 2 (mod 16) those are the 16
// distinct 8-byte banks.
__host__ __device__ __forceinline__ int pencil_stride(int N2) { return N2 + ((2 - N2) % 16 + 16) % 16; }

// ---------------------------------------------------------------------------
// plane helpers (one y plane, N3 rows of N1 reals <-> N3 x Nh half spectrum)
// ---------------------------------------------------------------------------
// Points in packed order: q = ((y (N3/2) + j) N1 + x) 2 + s is the point
// (x, y, z = 2j + s).  A field written in this order fills the packed real
// rows of its y plane (real rows 2j and 2j + 1 interleaved in complex row j)
// with consecutive addresses.  Sets (y, z, x, j); returns the flat index
// (z N2 + y) N1 + x.
__device__ __forceinline__ long long packed_point(long long q, const GridArgs& g, int& y, int& z, int& x, int& j) {
    const int s = (int)(q & 1);
    const int nh3 = g.N3 >> 1;
    if (g.fast) {
        const unsigned t = (unsigned)(q >> 1);
        const unsigned rr = __umulhi(t, g.m1);
        x = (int)(t - rr * (unsigned)g.N1);
        y = (int)__umulhi(rr, g.mh3);
        j = (int)(rr - (unsigned)y * (unsigned)nh3);
    } else {
        const long long t = q >> 1;
        const long long rr = t / g.N1;
        x = (int)(t - rr * g.N1);
        y = (int)(rr / nh3);
        j = (int)(rr - (long long)y * nh3);
    }
    z = 2 * j + s;
    return ((long long)z * g.N2 + y) * g.N1 + x;
}
// (x, y, z) of flat index i = (z N2 + y) N1 + x
__device__ __forceinline__ void flat_point(long long i, const GridArgs& g, int& x, int& y, int& z) {
    if (g.fast) {
        const unsigned r = __umulhi((unsigned)i, g.m1);
        x = (int)((unsigned)i - r * (unsigned)g.N1);
        z = (int)__umulhi(r, g.m2);
        y = (int)(r - (unsigned)z * (unsigned)g.N2);
    } else {
        const long long r = i / g.N1;
        x = (int)(i - r * g.N1);
        z = (int)(r / g.N2);
        y = (int)(r - (long long)z * g.N2);
    }
}
// Packed real rows: real rows 2j and 2j+1 of a plane are the real and
// imaginary parts of complex row j, which starts at complex offset 2 Nh j.
// This is the float offset, within its plane, of real point (x, z = 2j + s).
__device__ __forceinline__ int packed_offset(int x, int j, int s, int Nh) { return 4 * j * Nh + 2 * x + s; }

// Rows of a plane (complex row j holds real rows 2j and 2j+1) through the
// x transform, several rows per warp at compile-time lengths; each row is
// then untangled into the two half spectra (forward), or tangled before the
// transform (inverse).
template <int CN1, bool INV, int MAXR = 16, class W>
__device__ __forceinline__ void plane_rows(float2* plane, const GridArgs& g, const W* tw1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nrows = g.N3 / 2, rs = 2 * g.Nh;
    if constexpr (CN1 > 0) {
        constexpr int L = ct_lines_per_warp(CN1, MAXR);
        const int full = (nrows / L) * L;
        for (int row = warp * L; row < full; row += nw * L) {
            float2* p = plane + row * rs;
            if (INV)
                for (int l = 0; l < L; ++l) c2r_tangle(p + l * rs, g.N1, lane);
            ct_fft<CN1, L, INV, MAXR>(p, 1, rs, tw1, lane);
            if (!INV)
                for (int l = 0; l < L; ++l) r2c_untangle(p + l * rs, g.N1, lane);
        }
        for (int row = full + warp; row < nrows; row += nw) {
            float2* p = plane + row * rs;
            if (INV) c2r_tangle(p, g.N1, lane);
            ct_fft<CN1, 1, INV, MAXR>(p, 1, 0, tw1, lane);
            if (!INV) r2c_untangle(p, g.N1, lane);
        }
    } else {
        for (int row = warp; row < nrows; row += nw) {
            float2* p = plane + row * rs;
            if (INV) c2r_tangle(p, g.N1, lane);
            line_fft<INV>(p, 1, g.p1, tw1, lane);
            if (!INV) r2c_untangle(p, g.N1, lane);
        }
    }
}

// Forward: packed real rows -> half spectrum (x R2C, then z C2C).
template <int CN1, int CN3, int MAXR = 16, class W>
__device__ void plane_forward(float2* plane, const GridArgs& g, const W* tw1, const W* tw3) {
    plane_rows<CN1, false, MAXR>(plane, g, tw1);
    __syncthreads();
    columns_fft<CN3, false, MAXR>(plane, g.Nh, g.p3, tw3);
    __syncthreads();
}

// Inverse: half spectrum -> packed real rows (z C2C inverse, then x C2R), unscaled.
template <int CN1, int CN3, int MAXR = 16, class W>
__device__ void plane_inverse(float2* plane, const GridArgs& g, const W* tw1, const W* tw3) {
    columns_fft<CN3, true, MAXR>(plane, g.Nh, g.p3, tw3);
    __syncthreads();
    plane_rows<CN1, true, MAXR>(plane, g, tw1);
    __syncthreads();
}

constexpr int PLANE_THREADS = 256;  // threads of the plane kernels (P1, P5)

// Twiddles in shared memory after n float2 values, on a 16-byte boundary.
__host__ __device__ __forceinline__ size_t tw_offset(size_t n) { return (n + 1) & ~(size_t)1; }
template <class W = Tw>
__device__ __forceinline__ W* twiddles_after(float2* base, size_t n) {
    return reinterpret_cast<W*>(base + tw_offset(n));
}
// The twiddle kind of a transform: hi/lo pairs (EXACT) or FP32 values.
template <bool EXACT>
using TwOf = typename std::conditional<EXACT, Tw, float2>::type;

}  // namespace vdw
