// The y stage of the 3D transforms and the per-G contraction of Eqs. (Eoffk),
// (epsofk) in |G| order.
//
// The kernel phi_ab(|G|) depends on G only through |G|, by a cubic spline on
// a uniform k mesh (the radial table, text after Eq. Eoffk).  In the natural
// (kx, ky, kz) order neighbouring points fall in unrelated intervals of that
// table, so the 32 lanes of a warp would fetch 32 different table rows at
// every step of the Nq (Nq + 1) / 2 pair loop.  Here the points of the half
// spectrum are sorted once per plan by |G|: consecutive points then share
// their table interval, a warp's table fetch is one broadcast row, and the
// contraction is a plain stream over the sorted points.
//
//   P2a k_pencil_fwd      C2C along y of 4 fields for C columns; each point's
//                         4 values (32 bytes) go to its sorted position
//   P2b k_contract_sorted per sorted point: u_a = sum_b phi_ab(|G|) theta_b,
//                         the energy of Eq. (Eoffk) in FP64, u / N written back
//   P2c k_pencil_inv      gathers the 4 values of each point of C columns from
//                         the sorted records, inverse C2C along y, back into
//                         the plane layout
//
// Record layout ("quads"): field a = 4 q + i of sorted point r is float2 i of
// the 32-byte record r of quad q: Q[q * qstride + 2 r], Q[... + 2 r + 1]
// (float4 units), qstride = 2 Npad.  Npad is the number of half-spectrum
// points N2 N3 (N1/2 + 1) rounded up to a whole number of contraction blocks;
// the padding records stay zero.  (Writing u in pencil order instead, so that
// the inverse y kernel reads contiguous runs, moves the scattered accesses
// into the contraction's stores and measured no faster.)
#include "plane.cuh"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace vdw {

constexpr int SORT_THREADS = SORTED_BLOCK;  // points per contraction block
constexpr int PEN_THREADS = 256;   // threads of the y-pencil kernels
constexpr int PEN_COLS = 8;        // columns per y-pencil block (64-byte runs per plane row)

// The inverse y kernel stages the sorted positions of its C columns,
// pos[c0 N2 .. (c0 + C) N2), in shared memory after the lines and the room for
// their twiddles, by 4-byte asynchronous copies (zero past the last column),
// before its gather: all of them in flight at once rather than a few per
// thread ahead of the copies that need them (0.138 against 0.143 ms at
// 180 x 180 x 72; the forward kernel, whose positions are only needed for
// its stores, gains nothing from it).
__host__ __device__ __forceinline__ size_t pencil_pos_offset(int C, int S, int N2) {
    return sizeof(float2) * tw_offset((size_t)4 * C * S) + sizeof(Tw) * (size_t)N2;
}
__device__ __forceinline__ void stage_pos(unsigned* pos_s, const unsigned* __restrict__ pos, int c0, int C, int N2,
                                          int ncols, SmallDiv sN2) {
    const unsigned* pb = pos + (long long)c0 * N2;
    for (int i = threadIdx.x; i < C * N2; i += blockDim.x) {
        const bool ok = c0 + sdiv(i, sN2) < ncols;
        cp_async4(pos_s + i, ok ? pb + i : pos, ok);
    }
}

// ---------------------------------------------------------------------------
// P2a: forward y transforms of one quad of fields, records in |G| order
// ---------------------------------------------------------------------------
// Block (column tile, quad q): the fields 4q .. 4q+3 of C consecutive
// half-spectrum columns, all N2 rows, staged as lines [4][C][N2].
template <int CN2>
__global__ void __launch_bounds__(PEN_THREADS) k_pencil_fwd(const float2* __restrict__ spec, GridArgs g,
                                                            const Tw* __restrict__ tw,
                                                            const unsigned* __restrict__ pos, float4* __restrict__ Q,
                                                            long long qstride, int C) {
    extern __shared__ float2 sm[];
    const int N2 = CN2 > 0 ? CN2 : g.N2;
    const int S = pencil_stride(N2);
    float2* lines = sm;  // [4][C][S]
    Tw* tw2 = twiddles_after(lines, (size_t)(4 * C * S));
    load_line_twiddles<CN2>(tw2, tw + g.N1, N2);
    const int c0 = blockIdx.x * C, q = blockIdx.y;
    spec += blockIdx.z * g.bs_spec;  // density blockIdx.z of a batch
    Q += blockIdx.z * g.bs_Q;
    const float2* src = spec + (long long)4 * q * N2 * g.ncols;
    const SmallDiv sC = small_div(C), sN2 = small_div(N2);
    const int tot = 4 * N2 * C;
    // consecutive threads read consecutive columns of one plane row; the
    // copies are asynchronous, so each thread has all of its loads in flight
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        const int r = sdiv(i, sC), cc = i - r * C;  // r = a N2 + y
        const int a = sdiv(r, sN2), y = r - a * N2;
        const int col = c0 + cc;
        const bool ok = col < g.ncols;
        cp_async8(lines + (a * C + cc) * S + y, ok ? src + (long long)r * g.ncols + col : src, ok);
    }
    cp_async_wait_all();
    __syncthreads();
    pencils_fft<CN2, false>(lines, 4 * C, N2, g.p2, tw2, S);
    __syncthreads();
    float4* Qq = Q + q * qstride;
    const int LS = C * S;
#pragma unroll 4
    for (int task = threadIdx.x; task < C * N2; task += blockDim.x) {
        const int cc = sdiv(task, sN2), y = task - cc * N2;
        const int col = c0 + cc;
        if (col >= g.ncols) continue;
        const long long p = pos[(long long)col * N2 + y];
        const float2* l = lines + cc * S + y;
        const float2 v0 = l[0], v1 = l[LS], v2 = l[2 * LS], v3 = l[3 * LS];
        Qq[2 * p] = make_float4(v0.x, v0.y, v1.x, v1.y);
        Qq[2 * p + 1] = make_float4(v2.x, v2.y, v3.x, v3.y);
    }
}

// ---------------------------------------------------------------------------
// P2c: records in |G| order -> inverse y transforms -> plane layout
// ---------------------------------------------------------------------------
template <int CN2>
__global__ void __launch_bounds__(PEN_THREADS) k_pencil_inv(float2* __restrict__ spec, GridArgs g,
                                                            const Tw* __restrict__ tw,
                                                            const unsigned* __restrict__ pos,
                                                            const float4* __restrict__ Q, long long qstride, int C) {
    extern __shared__ float2 sm[];
    const int N2 = CN2 > 0 ? CN2 : g.N2;
    const int S = pencil_stride(N2);
    float2* lines = sm;  // [4][C][S]
    float2* tw2 = twiddles_after<float2>(lines, (size_t)(4 * C * S));
    load_line_twiddles<CN2>(tw2, tw + g.N1, N2);
    const int c0 = blockIdx.x * C, q = blockIdx.y;
    spec += blockIdx.z * g.bs_spec;  // density blockIdx.z of a batch
    Q += blockIdx.z * g.bs_Q;
    const SmallDiv sC = small_div(C), sN2 = small_div(N2);
    const float2* Qq = reinterpret_cast<const float2*>(Q + q * qstride);
    const int LS = C * S;
    // the positions first (all in flight at once), then the gather
    unsigned* pos_s = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(sm) + pencil_pos_offset(C, S, N2));
    stage_pos(pos_s, pos, c0, C, N2, g.ncols, sN2);
    cp_async_wait_all();
    __syncthreads();
    // the four values of a point go to four lines: 8-byte asynchronous copies
#pragma unroll 4
    for (int task = threadIdx.x; task < C * N2; task += blockDim.x) {
        const int cc = sdiv(task, sN2), y = task - cc * N2;
        const int col = c0 + cc;
        const bool ok = col < g.ncols;
        const long long p = ok ? (long long)pos_s[task] : 0;
        float2* l = lines + cc * S + y;
#pragma unroll
        for (int a = 0; a < 4; ++a) cp_async8(l + a * LS, Qq + 4 * p + a, ok);
    }
    cp_async_wait_all();
    __syncthreads();
    pencils_fft<CN2, true>(lines, 4 * C, N2, g.p2, tw2, S);
    __syncthreads();
    float2* dst = spec + (long long)4 * q * N2 * g.ncols;
    const int tot = 4 * N2 * C;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        const int r = sdiv(i, sC), cc = i - r * C;
        const int a = sdiv(r, sN2), y = r - a * N2;
        const int col = c0 + cc;
        if (col < g.ncols) dst[(long long)r * g.ncols + col] = lines[(a * C + cc) * S + y];
    }
}

// ---------------------------------------------------------------------------
// P2b: the contraction over the sorted points
// ---------------------------------------------------------------------------
// gs[r] = |G| of sorted point r (bohr^-1), negative (or -0) where the point
// counts once in the energy (kx = 0 or kx = N1/2) and positive where it
// stands for itself and its conjugate -G (weight 2); non-decreasing in |G|
// (the padding repeats the last |G|).  kcoef: the radial table as cubic
// coefficients in the local position t, [Nk-1][NQ(NQ+1)/2] float4, pair order
// a <= b row by row.  E partial: sum over the block of
// w_G sum_a Re(conj theta_a u_a), unscaled.
//
// The block's points lie in a contiguous run of table intervals [jlo, jhi]
// (|G| is sorted), whose rows are one contiguous piece of the table: they are
// staged in shared memory, so that the pair loop reads them by broadcast from
// shared memory instead of waiting on the L2 cache.
constexpr int CONTRACT_ROWS = 4;  // table rows staged per block at most

// u += Phi(t) theta with the row's pair coefficients cf (shared memory)
template <int NQ>
__device__ __forceinline__ void pair_loop(const float4* cf, float t, const float2 (&th)[NQ], float2 (&u)[NQ]) {
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
        }
    }
}

template <int NQ>
__global__ void __launch_bounds__(SORT_THREADS, 4) k_contract_sorted(float4* __restrict__ Q, long long qstride,
                                                                    const float* __restrict__ gs,
                                                                    const float4* __restrict__ kcoef, float inv_dk,
                                                                    int Nk, float invN, double* __restrict__ epart,
                                                                    int write_back, long long bsQ, int bsE) {
    constexpr int NP = NQ * (NQ + 1) / 2;
    __shared__ double red[32];
    __shared__ float4 rows[CONTRACT_ROWS * NP];
    Q += blockIdx.y * bsQ;  // density blockIdx.y of a batch
    epart += blockIdx.y * bsE;
    const long long r0 = (long long)blockIdx.x * SORT_THREADS;
    const long long r = r0 + threadIdx.x;
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
    const float s = fabsf(gm) * inv_dk;
    const int j = min((int)s, Nk - 2);
    const float t = s - (float)j;
    float2 u[NQ];
#pragma unroll
    for (int a = 0; a < NQ; ++a) u[a] = make_float2(0.f, 0.f);
    // windows of CONTRACT_ROWS rows over the block's interval run; nearly every
    // block needs one (only the few blocks at the smallest |G|, where the
    // shells hold few points, need several)
    const int jlo = min((int)(fabsf(gs[r0]) * inv_dk), Nk - 2);
    const int jhi = min((int)(fabsf(gs[r0 + SORT_THREADS - 1]) * inv_dk), Nk - 2);
    for (int w = jlo; w <= jhi; w += CONTRACT_ROWS) {
        const int nr = min(CONTRACT_ROWS, jhi - w + 1);
        if (w != jlo) __syncthreads();  // the previous window's rows are read
        const float4* src = kcoef + (long long)w * NP;
        for (int i = threadIdx.x; i < nr * NP; i += SORT_THREADS) rows[i] = __ldg(src + i);
        __syncthreads();
        if (j >= w && j < w + nr) pair_loop<NQ>(rows + (j - w) * NP, t, th, u);
    }
    float e = 0.f;
#pragma unroll
    for (int a = 0; a < NQ; ++a) e = fmaf(th[a].x, u[a].x, fmaf(th[a].y, u[a].y, e));
    const double es = block_sum((double)(wgt * e), red);
    if (threadIdx.x == 0) epart[blockIdx.x] = es;
    if (!write_back) return;
#pragma unroll
    for (int q = 0; q < NQ / 4; ++q) {
        Q[q * qstride + 2 * r] =
            make_float4(u[4 * q].x * invN, u[4 * q].y * invN, u[4 * q + 1].x * invN, u[4 * q + 1].y * invN);
        Q[q * qstride + 2 * r + 1] =
            make_float4(u[4 * q + 2].x * invN, u[4 * q + 2].y * invN, u[4 * q + 3].x * invN, u[4 * q + 3].y * invN);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// forward kernel: lines and twiddles; inverse kernel: also the staged positions
size_t sorted_pencil_smem_fwd(const GridArgs& g) { return pencil_pos_offset(PEN_COLS, pencil_stride(g.N2), g.N2); }
size_t sorted_pencil_smem(const GridArgs& g) {
    return sorted_pencil_smem_fwd(g) + sizeof(unsigned) * PEN_COLS * g.N2;
}

// |G| order of the half spectrum: pos[col N2 + y] = sorted position of the
// point (kx, y, kz), col = kz Nh + kx; gs[sorted position] = |G| with the
// energy weight in its sign.  Ties (equal |G|) keep the (col, y) order, so
// the permutation is deterministic.
int sorted_plan(vdw_ctx* c) {
    const GridArgs& g = c->g;
    const long long nG = (long long)g.ncols * g.N2;
    const long long Npad = (nG + SORT_THREADS - 1) / SORT_THREADS * SORT_THREADS;
    const double PI_D = 3.14159265358979323846;
    const double b1 = 2.0 * PI_D / c->L[0], b2 = 2.0 * PI_D / c->L[1], b3 = 2.0 * PI_D / c->L[2];
    std::vector<double> key((size_t)nG);
    for (int col = 0; col < g.ncols; ++col) {
        const int kx = col % g.Nh, kz = col / g.Nh;
        const int mz = (2 * kz <= g.N3) ? kz : kz - g.N3;
        const double ax = b1 * kx, az = b3 * mz;
        for (int y = 0; y < g.N2; ++y) {
            const int my = (2 * y <= g.N2) ? y : y - g.N2;
            const double ay = b2 * my;
            key[(size_t)col * g.N2 + y] = ax * ax + ay * ay + az * az;
        }
    }
    std::vector<unsigned> idx((size_t)nG);
    std::iota(idx.begin(), idx.end(), 0u);
    std::stable_sort(idx.begin(), idx.end(), [&](unsigned a, unsigned b) { return key[a] < key[b]; });
    std::vector<unsigned> pos((size_t)nG);
    std::vector<float> gs((size_t)Npad, 0.f);
    for (long long s = 0; s < nG; ++s) {
        const unsigned i = idx[(size_t)s];
        pos[i] = (unsigned)s;
        const int col = (int)(i / g.N2), kx = col % g.Nh;
        const bool single = (kx == 0) || (2 * kx == g.N1);
        const float m = (float)std::sqrt(key[i]);
        gs[(size_t)s] = single ? -m : m;
    }
    // padding records (theta = 0): the last |G| again, so that |gs| stays sorted
    for (long long s = nG; s < Npad; ++s) gs[(size_t)s] = std::fabs(gs[(size_t)(nG - 1)]);
    c->nG = nG;
    c->Npad = Npad;
    c->nb_sorted = (int)(Npad / SORT_THREADS);
    VDW_CUDA(cudaMalloc(&c->d_pos, sizeof(unsigned) * (size_t)nG));
    VDW_CUDA(cudaMalloc(&c->d_gs, sizeof(float) * (size_t)Npad));
    VDW_CUDA(cudaMemcpy(c->d_pos, pos.data(), sizeof(unsigned) * (size_t)nG, cudaMemcpyHostToDevice));
    VDW_CUDA(cudaMemcpy(c->d_gs, gs.data(), sizeof(float) * (size_t)Npad, cudaMemcpyHostToDevice));
    c->bytes += sizeof(unsigned) * (size_t)nG + sizeof(float) * (size_t)Npad;
    return VDW_OK;
}

void sorted_free(vdw_ctx* c) {
    cudaFree(c->d_pos);
    cudaFree(c->d_gs);
    c->d_pos = nullptr;
    c->d_gs = nullptr;
}

template <int CN2>
static int configure_sorted_sized(vdw_ctx* c) {
    int rc = raise_smem_limit(k_pencil_fwd<CN2>, (int)sorted_pencil_smem_fwd(c->g));
    if (!rc) rc = raise_smem_limit(k_pencil_inv<CN2>, (int)sorted_pencil_smem(c->g));
    if (rc) return rc;
    int dev = 0;
    VDW_CUDA(cudaGetDevice(&dev));
    VDW_CUDA(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev));
    return VDW_OK;
}

int sorted_configure(vdw_ctx* c) {
    const int N2 = c->g.N2;
    if (N2 == 180) return configure_sorted_sized<180>(c);
    if (N2 == 256) return configure_sorted_sized<256>(c);
    return configure_sorted_sized<0>(c);
}

// the compile-time y lengths are those of the sized grids (180 x 180 x 72,
// 256 x 256 x 96); any other grid uses the runtime-length engine
static int sized_n2(const GridArgs& g) {
    if (g.N1 == 180 && g.N2 == 180 && g.N3 == 72) return 180;
    if (g.N1 == 256 && g.N2 == 256 && g.N3 == 96) return 256;
    return 0;
}

#define VDW_SORTED_LAUNCH(KERNEL, ...)                                                  \
    switch (sized_n2(g)) {                                                            \
        case 180: KERNEL<180><<<grid, PEN_THREADS, sm, s>>>(__VA_ARGS__); break;      \
        case 256: KERNEL<256><<<grid, PEN_THREADS, sm, s>>>(__VA_ARGS__); break;      \
        default: KERNEL<0><<<grid, PEN_THREADS, sm, s>>>(__VA_ARGS__);                \
    }

int sorted_forward(vdw_ctx* c, int nfields, cudaStream_t s, int B) {
    const GridArgs& g = c->g;
    const dim3 grid((g.ncols + PEN_COLS - 1) / PEN_COLS, nfields / 4, B);
    const size_t sm = sorted_pencil_smem_fwd(g);
    VDW_SORTED_LAUNCH(k_pencil_fwd, c->d_spec, g, c->d_tw, c->d_pos, c->d_Q, 2 * c->Npad, PEN_COLS)
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

int sorted_inverse(vdw_ctx* c, int nfields, cudaStream_t s, int B) {
    const GridArgs& g = c->g;
    const dim3 grid((g.ncols + PEN_COLS - 1) / PEN_COLS, nfields / 4, B);
    const size_t sm = sorted_pencil_smem(g);
    VDW_SORTED_LAUNCH(k_pencil_inv, c->d_spec, g, c->d_tw, c->d_pos, c->d_Q, 2 * c->Npad, PEN_COLS)
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}
#undef VDW_SORTED_LAUNCH

int sorted_contract(vdw_ctx* c, double* epart, int write_back, cudaStream_t s, int B) {
    return sorted_contract_table(c, c->p.Nq, c->d_kcoef, c->g.inv_dk, c->g.Nk, epart, write_back, s, B);
}

int sorted_contract_table(vdw_ctx* c, int nq, const float4* table, float inv_dk, int nk, double* epart,
                          int write_back, cudaStream_t s, int B) {
    const GridArgs& g = c->g;
    const long long qs = 2 * c->Npad;
#define VDW_CONTRACT(NQ)                                                                                  \
    k_contract_sorted<NQ><<<dim3(c->nb_sorted, B), SORT_THREADS, 0, s>>>(c->d_Q, qs, c->d_gs, table, inv_dk, nk, \
                                                                         g.invN, epart, write_back, g.bs_Q,      \
                                                                         g.bs_epart)
    switch (nq) {
        case 20: VDW_CONTRACT(20); break;
        case 8: VDW_CONTRACT(8); break;
        case 12: VDW_CONTRACT(12); break;
        case 16: VDW_CONTRACT(16); break;
        default: set_error("Nq not compiled in"); return VDW_ERR_UNSUPPORTED;
    }
#undef VDW_CONTRACT
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}

}  // namespace vdw
