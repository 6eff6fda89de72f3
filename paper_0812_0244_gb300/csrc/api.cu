// C ABI of the vdwnl library (declared in include/vdwnl.h).
#include "common.cuh"

#include <algorithm>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

namespace vdw {

static thread_local std::string g_last_error;
static std::mutex g_smem_mu;

void smem_limit_lock(bool lock) {
    if (lock) g_smem_mu.lock();
    else g_smem_mu.unlock();
}

void set_error(const std::string& s) { g_last_error = s; }

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return (e == cudaErrorMemoryAllocation) ? VDW_ERR_OOM : VDW_ERR_CUDA;
}

int check_wait(vdw_ctx* c) {
    volatile int* f = c->h_flags;
    if (!f || (f[0] == 0 && f[1] == 0)) return VDW_OK;
    c->wait_seen = 1;
    f[0] = 0;
    f[1] = 0;
    g_last_error = "a bounded wait inside a kernel of an earlier call gave up; that call's results may be wrong";
    return VDW_ERR_TIMEOUT;
}

static bool smooth235(int n) {
    if (n < 1) return false;
    for (int r : {2, 3, 5})
        while (n % r == 0) n /= r;
    return n == 1;
}

static void free_plan(vdw_ctx* c) {
    cudaFree(c->d_tw);
    cudaFree(c->d_Q);
    c->d_Q = nullptr;
    c->batch_max = 0;
    cudaFree(c->d_spec);
    cudaFree(c->d_wspec);
    cudaFree(c->d_t);
    cudaFree(c->d_k);
    cudaFree(c->d_aux);
    cudaFree(c->d_epart);
    cudaFree(c->d_invalid);
    cudaFree(c->d_in);
    cudaFree(c->d_v);
    cudaFree(c->d_E);
    c->d_tw = nullptr;
    c->d_spec = c->d_wspec = nullptr;
    c->d_t = nullptr;
    c->d_k = nullptr;
    c->d_aux = nullptr;
    c->d_epart = nullptr;
    c->d_invalid = nullptr;
    c->d_in = c->d_v = nullptr;
    c->d_E = nullptr;
    cudaFree(c->d_gtmp);
    c->d_gtmp = nullptr;
    cudaFree(c->d_gg);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    c->h_flags = nullptr;
    cudaFree(c->d_xc);
    c->d_gg = nullptr;
    c->d_flags = nullptr;
    c->d_xc = nullptr;
    learned_free(c);
    sorted_free(c);
    if (c->s_copy) cudaStreamDestroy(c->s_copy);
    if (c->s_side) cudaStreamDestroy(c->s_side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    c->s_side = nullptr;
    c->ev_fork = c->ev_join = nullptr;
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    for (int i = 0; i < 4; ++i)
        if (c->ev_slab[i]) cudaEventDestroy(c->ev_slab[i]);
    c->s_copy = nullptr;
    c->ev_in = nullptr;
    for (int i = 0; i < 4; ++i) c->ev_slab[i] = nullptr;
    c->planned = 0;
}

// The per-density workspaces for Bmax densities at once (spectra, records,
// w spectra, the pointwise results and the energy partial sums), with the
// batch strides the kernels use.  Frees the previous ones.
int alloc_density_work(vdw_ctx* c, int Bmax) {
    GridArgs& g = c->g;
    const size_t Nq = (size_t)c->p.Nq, N = (size_t)g.N;
    const size_t spec_n = Nq * g.N2 * g.ncols, wspec_n = 3 * (size_t)g.N2 * g.ncols;
    const size_t q_n = Nq * (size_t)c->Npad / 2;  // float4 values (Nq/4 quads of Npad 32-byte records)
    const size_t ep_n = (size_t)c->nb_point + c->nb_sorted + 2 * EPART_SPLIT;
    const size_t old = c->batch_max > 0
                           ? (size_t)c->batch_max * (8 * (spec_n + wspec_n) + 16 * q_n + 25 * N + 8 * ep_n)
                           : 0;
    cudaFree(c->d_spec);
    cudaFree(c->d_wspec);
    cudaFree(c->d_Q);
    cudaFree(c->d_t);
    cudaFree(c->d_k);
    cudaFree(c->d_aux);
    cudaFree(c->d_gg);
    cudaFree(c->d_epart);
    c->d_spec = c->d_wspec = nullptr;
    c->d_Q = nullptr;
    c->d_t = c->d_gg = nullptr;
    c->d_k = nullptr;
    c->d_aux = nullptr;
    c->d_epart = nullptr;
    c->bytes -= old;
    c->batch_max = 0;
    const size_t B = (size_t)Bmax;
    VDW_CUDA(cudaMalloc(&c->d_spec, sizeof(float2) * spec_n * B));
    VDW_CUDA(cudaMalloc(&c->d_wspec, sizeof(float2) * wspec_n * B));
    VDW_CUDA(cudaMalloc(&c->d_Q, sizeof(float4) * q_n * B));
    VDW_CUDA(cudaMemset(c->d_Q, 0, sizeof(float4) * q_n * B));  // padding records stay zero
    VDW_CUDA(cudaMalloc(&c->d_t, sizeof(float) * N * B));
    VDW_CUDA(cudaMalloc(&c->d_k, N * B));
    VDW_CUDA(cudaMalloc(&c->d_aux, sizeof(float4) * N * B));
    VDW_CUDA(cudaMalloc(&c->d_gg, sizeof(float) * N * B));
    VDW_CUDA(cudaMalloc(&c->d_epart, sizeof(double) * ep_n * B));
    g.bs_spec = (long long)spec_n;
    g.bs_wspec = (long long)wspec_n;
    g.bs_Q = (long long)q_n;
    g.bs_epart = (int)ep_n;
    c->batch_max = Bmax;
    c->bytes += B * (8 * (spec_n + wspec_n) + 16 * q_n + 25 * N + 8 * ep_n);
    return VDW_OK;
}

}  // namespace vdw

using namespace vdw;

extern "C" {

int vdw_params_default(vdw_params* p) {
    if (!p) return VDW_ERR_ARG;
    p->Nq = 20;
    p->q_1 = 1e-5;
    p->q_c = 5.0;
    p->lambda = 1.2;
    p->m_c = 12;
    p->d_s = 1.0;
    p->na = 256;
    p->a_max = 64.0;
    p->d_asym = 8.0;
    p->r_c = 100.0;
    p->Nr = 4096;
    p->k_max = 40.0;
    p->Nk = 1024;
    p->n_cs = 64;
    p->n_min = 1e-12;
    return VDW_OK;
}

int vdw_kernel_table(const vdw_params* p, double* q_mesh, double* phi_k, double* phi0, double* C_s) {
    return table_build(p, q_mesh, phi_k, phi0, C_s);
}

int vdw_create(vdw_handle* h, const vdw_params* p, const double* phi_k, double C_s) {
    if (!h || !p) return VDW_ERR_ARG;
    *h = nullptr;
    if (p->Nq != 8 && p->Nq != 12 && p->Nq != 16 && p->Nq != 20) {
        set_error("Nq must be one of 8, 12, 16, 20");
        return VDW_ERR_UNSUPPORTED;
    }
    vdw_ctx* c = new (std::nothrow) vdw_ctx();
    if (!c) return VDW_ERR_OOM;
    std::memset((void*)c, 0, sizeof(vdw_ctx));
    c->p = *p;
    cudaGetDevice(&c->device);
    int rc = VDW_OK;
    const int Nq = p->Nq, Nk = p->Nk;
    double* table = nullptr;
    if (!phi_k) {
        table = new (std::nothrow) double[(size_t)Nq * Nq * Nk];
        if (!table) { delete c; return VDW_ERR_OOM; }
        rc = table_build(p, nullptr, table, &c->phi0, &C_s);
        phi_k = table;
    }
    if (rc == VDW_OK) rc = table_upload(c, phi_k, C_s);
    delete[] table;
    if (rc != VDW_OK) {
        cudaFree(c->d_kcoef);
        delete c;
        return rc;
    }
    c->bytes = sizeof(float4) * (size_t)(Nk - 1) * (Nq * (Nq + 1) / 2);
    *h = c;
    return VDW_OK;
}

int vdw_plan(vdw_handle c, int n1, int n2, int n3, const double L[3]) {
    if (!c || !L) return VDW_ERR_ARG;
    if (!(L[0] > 0 && L[1] > 0 && L[2] > 0)) return VDW_ERR_ARG;
    const int dims[3] = {n1, n2, n3};
    for (int d : dims)
        if (d < 4 || d > MAX_DIM || !smooth235(d)) {
            set_error("grid dimensions must be {2,3,5}-smooth and in [4, 256]");
            return VDW_ERR_SIZE;
        }
    if ((n1 & 1) || (n3 & 1)) {
        set_error("N1 and N3 must be even");
        return VDW_ERR_SIZE;
    }
    const double PI_D = 3.14159265358979323846;
    const double gmax = 2.0 * PI_D * std::sqrt(std::pow((n1 / 2) / L[0], 2) + std::pow((n2 / 2) / L[1], 2) +
                                               std::pow((n3 / 2) / L[2], 2));
    if (gmax > c->p.k_max) {
        set_error("largest |G| of the grid exceeds k_max of the kernel table");
        return VDW_ERR_SIZE;
    }
    cudaSetDevice(c->device);
    free_plan(c);
    c->bytes = 0;  // recounted below (tables included)
    GridArgs& g = c->g;
    g.N1 = n1;
    g.N2 = n2;
    g.N3 = n3;
    g.Nh = n1 / 2 + 1;
    g.N = (long long)n1 * n2 * n3;
    {
        const unsigned long long dmax = (unsigned long long)std::max(n1, std::max(n2, n3));
        g.fast = (n1 > 1 && n2 > 1 && n3 / 2 > 1 && (unsigned long long)g.N * dmax < (1ull << 32)) ? 1 : 0;
        g.m1 = g.fast ? 0xFFFFFFFFu / (unsigned)n1 + 1u : 0u;
        g.m2 = g.fast ? 0xFFFFFFFFu / (unsigned)n2 + 1u : 0u;
        g.mh3 = g.fast ? 0xFFFFFFFFu / (unsigned)(n3 / 2) + 1u : 0u;
    }
    g.ncols = n3 * g.Nh;
    for (int d = 0; d < 3; ++d) c->L[d] = L[d];
    g.gx = (float)(2.0 * PI_D / L[0]);
    g.gy = (float)(2.0 * PI_D / L[1]);
    g.gz = (float)(2.0 * PI_D / L[2]);
    g.gx2 = g.gx * g.gx;
    g.gy2 = g.gy * g.gy;
    g.gz2 = g.gz * g.gz;
    g.Nk = c->p.Nk;
    g.inv_dk = (float)((c->p.Nk - 1) / c->p.k_max);
    g.invN = (float)(1.0 / (double)g.N);
    int rc = make_line_plan(n1, &g.p1);
    if (!rc) rc = make_line_plan(n2, &g.p2);
    if (!rc) rc = make_line_plan(n3, &g.p3);
    if (rc) return rc;
    size_t sp, spen, sa, sd;
    rc = pipeline_plan_check(c, &sp, &spen, &sa, &sd);
    if (rc) {
        set_error("grid too large for on-chip staging");
        return rc;
    }
    const int Nq = c->p.Nq;
    const size_t spec_n = (size_t)Nq * n2 * g.ncols;
    {
        // pointwise slabs: 4, 3, 2 or 1 equal slabs of the N3/2 complex rows
        const int nh3 = n3 / 2;
        c->p0_chunks = (nh3 % 4 == 0) ? 4 : (nh3 % 3 == 0) ? 3 : (nh3 % 2 == 0) ? 2 : 1;
        c->p0_nj = nh3 / c->p0_chunks;
        c->p0_mnj = c->p0_nj > 1 ? 0xFFFFFFFFu / (unsigned)c->p0_nj + 1u : 0u;
        const long long nb = std::min<long long>((g.N + 255) / 256, 4096);
        c->nb_p0 = (int)((nb + c->p0_chunks - 1) / c->p0_chunks);
        c->nb_point = c->nb_p0 * c->p0_chunks;
    }
    VDW_CUDA(cudaMalloc(&c->d_tw, sizeof(float4) * (n1 + n2 + n3)));
    rc = sorted_plan(c);
    if (rc) return rc;
    rc = alloc_density_work(c, 1);
    if (rc) return rc;
    VDW_CUDA(cudaMalloc(&c->d_invalid, sizeof(unsigned long long)));
    VDW_CUDA(cudaHostAlloc(&c->h_flags, 2 * sizeof(int), cudaHostAllocMapped));
    c->h_flags[0] = c->h_flags[1] = 0;
    VDW_CUDA(cudaHostGetDevicePointer((void**)&c->d_flags, c->h_flags, 0));
    c->wait_seen = 0;
    VDW_CUDA(cudaMalloc(&c->d_xc, sizeof(double) * (4 + 2 * 1024)));
    VDW_CUDA(cudaStreamCreateWithFlags(&c->s_copy, cudaStreamNonBlocking));
    VDW_CUDA(cudaStreamCreateWithFlags(&c->s_side, cudaStreamNonBlocking));
    VDW_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    VDW_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    VDW_CUDA(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    for (int i = 0; i < 4; ++i) VDW_CUDA(cudaEventCreateWithFlags(&c->ev_slab[i], cudaEventDisableTiming));
    VDW_CUDA(cudaMemset(c->d_invalid, 0, sizeof(unsigned long long)));
    rc = pipeline_make_twiddles(c);
    if (rc) return rc;
    rc = pipeline_configure(c);
    if (rc) return rc;
    const int npairs = Nq * (Nq + 1) / 2;
    (void)spec_n;
    c->bytes += sizeof(float4) * (size_t)(c->p.Nk - 1) * npairs + sizeof(float4) * (n1 + n2 + n3);
    c->planned = 1;
    return VDW_OK;
}

int vdw_energy_potential(vdw_handle c, const float* n, const float* grad, double* E, float* v, float* w,
                         void* stream) {
    if (!c || !n) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    if (const int rw = check_wait(c)) return rw;
    if (!grad) {
        // grad n = D n with the library's spectral derivative
        if (!c->d_gtmp) VDW_CUDA(cudaMalloc(&c->d_gtmp, sizeof(float) * 3 * (size_t)c->g.N));
        const int rc = vdw_spectral_gradient(c, n, c->d_gtmp, stream);
        if (rc) return rc;
        grad = c->d_gtmp;
    }
    return pipeline_run(c, n, grad, E, v, w, (cudaStream_t)stream);
}

int vdw_plan_cell(vdw_handle c, int n1, int n2, int n3, const double cell[9]) {
    if (!c || !cell) return VDW_ERR_ARG;
    double dmax = 0.0;
    for (int i = 0; i < 3; ++i) dmax = std::max(dmax, std::fabs(cell[4 * i]));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (i != j && !(std::fabs(cell[3 * i + j]) <= 1e-12 * dmax)) {
                set_error("vdw_plan_cell: only orthorhombic cells (diagonal lattice vectors) are supported");
                return VDW_ERR_UNSUPPORTED;
            }
    const double L[3] = {cell[0], cell[4], cell[8]};
    return vdw_plan(c, n1, n2, n3, L);
}

int vdw_plan_batch(vdw_handle c, int Bmax) {
    if (!c || Bmax < 1) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    cudaSetDevice(c->device);
    VDW_CUDA(cudaDeviceSynchronize());  // no call of the context may still use the old workspaces
    const int rc = alloc_density_work(c, Bmax);
    if (rc) {
        c->planned = 0;  // the workspaces are gone; the caller has to plan again
        return rc;
    }
    return VDW_OK;
}

int vdw_energy_potential_batched(vdw_handle c, int B, const float* n, const float* grad, double* E, float* v,
                                 void* stream) {
    if (!c || !n || !grad || !E || B < 1) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    if (B > c->batch_max) {
        set_error("batch larger than the workspaces of vdw_plan_batch");
        return VDW_ERR_SIZE;
    }
    if (const int rw = check_wait(c)) return rw;
    return pipeline_run(c, n, grad, E, v, nullptr, (cudaStream_t)stream, 0, 0, nullptr, B);
}

int vdw_energy_potential_fd(vdw_handle c, const float* n, const float* grad, double* E, float* v, void* stream) {
    if (!c || !n) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    if (const int rw = check_wait(c)) return rw;
    if (!grad) {
        if (!c->d_gtmp) VDW_CUDA(cudaMalloc(&c->d_gtmp, sizeof(float) * 3 * (size_t)c->g.N));
        const int rc = pipeline_stencil_gradient(c, n, c->d_gtmp, (cudaStream_t)stream);
        if (rc) return rc;
        grad = c->d_gtmp;
    }
    return pipeline_run(c, n, grad, E, v, nullptr, (cudaStream_t)stream, 1);
}

int vdw_xc_energy_potential(vdw_handle c, const float* n, const float* grad, double* E, float* v, int fd,
                            void* stream) {
    if (!c || !n || !E) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (const int rw = check_wait(c)) return rw;
    if (!grad) {
        if (!c->d_gtmp) VDW_CUDA(cudaMalloc(&c->d_gtmp, sizeof(float) * 3 * (size_t)c->g.N));
        const int rc = fd ? pipeline_stencil_gradient(c, n, c->d_gtmp, s) : vdw_spectral_gradient(c, n, c->d_gtmp, stream);
        if (rc) return rc;
        grad = c->d_gtmp;
    }
    int rc = pipeline_run(c, n, grad, c->d_xc, v, nullptr, s, fd ? 1 : 0, 1);
    if (rc) return rc;
    return pipeline_xc_final(c, E, s);
}

int vdw_energy_potential_host(vdw_handle c, const float* n, const float* grad, double* E, float* v, void* stream) {
    if (!c || !n || !grad) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    if (const int rw = check_wait(c)) return rw;
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = c->g.N;
    if (!c->d_in) {
        VDW_CUDA(cudaMalloc(&c->d_in, sizeof(float) * 4 * N));
        VDW_CUDA(cudaMalloc(&c->d_v, sizeof(float) * N));
        VDW_CUDA(cudaMalloc(&c->d_E, sizeof(double) * 3));
        c->bytes += sizeof(float) * 5 * N + sizeof(double) * 3;
    }
    // the inputs go up slab by slab on the copy stream; the pointwise pass
    // takes each slab as soon as it has arrived
    VDW_CUDA(cudaEventRecord(c->ev_in, s));
    VDW_CUDA(cudaStreamWaitEvent(c->s_copy, c->ev_in, 0));
    const long long slab = 2LL * c->p0_nj * c->g.N2 * c->g.N1;  // points of a slab (contiguous in z)
    for (int sl = 0; sl < c->p0_chunks; ++sl) {
        const long long off = sl * slab;
        VDW_CUDA(cudaMemcpyAsync(c->d_in + off, n + off, sizeof(float) * slab, cudaMemcpyHostToDevice, c->s_copy));
        for (int d = 0; d < 3; ++d)
            VDW_CUDA(cudaMemcpyAsync(c->d_in + N + d * N + off, grad + d * N + off, sizeof(float) * slab,
                                     cudaMemcpyHostToDevice, c->s_copy));
        VDW_CUDA(cudaEventRecord(c->ev_slab[sl], c->s_copy));
    }
    int rc = pipeline_run(c, c->d_in, c->d_in + N, c->d_E, v ? c->d_v : nullptr, nullptr, s, 0, 0, c->ev_slab);
    if (rc) return rc;
    if (E) VDW_CUDA(cudaMemcpyAsync(E, c->d_E, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    if (v) VDW_CUDA(cudaMemcpyAsync(v, c->d_v, sizeof(float) * N, cudaMemcpyDeviceToHost, s));
    VDW_CUDA(cudaStreamSynchronize(s));
    return VDW_OK;
}

int vdw_last_invalid_points(vdw_handle c, long long* count) {
    if (!c || !count) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    unsigned long long v = 0;
    VDW_CUDA(cudaDeviceSynchronize());
    VDW_CUDA(cudaMemcpy(&v, c->d_invalid, sizeof(v), cudaMemcpyDeviceToHost));
    *count = (long long)v;
    return VDW_OK;
}

int vdw_profile_enable(vdw_handle c, int enable) {
    if (!c) return VDW_ERR_ARG;
    if (enable && !c->ev[0]) {
        for (int i = 0; i <= VDW_NSTAGES; ++i) VDW_CUDA(cudaEventCreate(&c->ev[i]));
    }
    c->prof = enable ? 1 : 0;
    return VDW_OK;
}

int vdw_profile_read(vdw_handle c, float* ms) {
    if (!c || !ms) return VDW_ERR_ARG;
    if (!c->ev[0]) return VDW_ERR_STATE;
    int last = -1;
    for (int i = 0; i < VDW_NSTAGES; ++i)
        if (c->ev_done[i]) last = i;
    if (last < 0) return VDW_ERR_STATE;
    VDW_CUDA(cudaEventSynchronize(c->ev[last + 1]));
    int prev = 0;  // event that opened the next recorded stage
    for (int i = 0; i < VDW_NSTAGES; ++i) {
        ms[i] = -1.f;
        if (!c->ev_done[i]) continue;
        VDW_CUDA(cudaEventElapsedTime(&ms[i], c->ev[prev], c->ev[i + 1]));
        prev = i + 1;
    }
    return VDW_OK;
}

int vdw_wait_status(vdw_handle c, int* gave_up) {
    if (!c || !gave_up) return VDW_ERR_ARG;
    if (!c->planned) return VDW_ERR_STATE;
    VDW_CUDA(cudaDeviceSynchronize());
    volatile int* f = c->h_flags;
    *gave_up = (f[0] || f[1] || c->wait_seen) ? 1 : 0;
    return VDW_OK;
}

int vdw_workspace_bytes(vdw_handle c, size_t* bytes) {
    if (!c || !bytes) return VDW_ERR_ARG;
    *bytes = c->bytes;
    return VDW_OK;
}

int vdw_destroy(vdw_handle c) {
    if (!c) return VDW_ERR_ARG;
    cudaSetDevice(c->device);
    free_plan(c);
    cudaFree(c->d_kcoef);
    for (int i = 0; i <= VDW_NSTAGES; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    delete c;
    return VDW_OK;
}

const char* vdw_error_string(int code) {
    switch (code) {
        case VDW_OK: return "ok";
        case VDW_ERR_ARG: return "invalid argument";
        case VDW_ERR_SIZE: return "unsupported grid size";
        case VDW_ERR_CUDA: return "CUDA runtime error";
        case VDW_ERR_OOM: return "device out of memory";
        case VDW_ERR_STATE: return "context not planned";
        case VDW_ERR_UNSUPPORTED: return "unsupported parameter";
        case VDW_ERR_TIMEOUT: return "a bounded wait in a kernel gave up";
        default: return "unknown error";
    }
}

const char* vdw_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
