// vdw_delta_energy_noalloc: the local softening correction Delta E computed
// without any device allocation.
//
// Who needs it: code that may not call cudaMalloc at the point where it
// evaluates the energy, e.g. a host program that hands every device byte to
// its own pool allocator, a plugin whose host forbids allocations inside its
// step, or a caller that wants the call to stay free of allocator
// synchronisation.  Such callers create the context (which does allocate its
// tables) once at start-up, and then call this entry point as often as they
// like.
//
// The kernel is the pointwise q0 / saturation / Delta E stage of
// vdw_energy_potential, but it writes its per-block FP64 partial sums into a
// fixed file-scope device array instead of the context's workspace, and a
// second kernel sums them in a fixed order.  That array is reserved in every
// GPU that loads the library, for the life of the process.
#include "common.cuh"
#include "pointwise.cuh"

#include <mutex>

namespace vdw {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PTS_PER_THREAD = 16;
constexpr long long NA_PTS_PER_BLOCK = (long long)NA_THREADS * NA_PTS_PER_THREAD;  // 4096
constexpr int NA_MAX_BLOCKS = 4096;  // scratch slots: one FP64 partial per block
static_assert((long long)NA_MAX_BLOCKS * NA_PTS_PER_BLOCK == VDW_NOALLOC_MAX_POINTS, "scratch limit");

// The scratch: 4096 doubles (32 KiB).  Every call writes each slot it later
// reads, so nothing in it has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
double* g_dev_ptr[NA_MAX_DEVICES] = {nullptr};

// Block b handles points [b*4096, (b+1)*4096): the partition, and hence the
// summation order, depends only on the number of points.
__global__ void __launch_bounds__(NA_THREADS) k_delta_energy_blocks(const float* __restrict__ n,
                                                                    const float* __restrict__ grad, long long N,
                                                                    PointParams P, double* __restrict__ partials) {
    __shared__ double red[NA_THREADS / 32];
    const long long base = (long long)blockIdx.x * NA_PTS_PER_BLOCK;
    double acc = 0.0;
    for (int r = 0; r < NA_PTS_PER_THREAD; ++r) {
        const long long i = base + (long long)r * NA_THREADS + threadIdx.x;
        if (i >= N) break;
        const float ni = n[i];
        const QPoint qp = q_point(ni, grad[i], grad[N + i], grad[2 * N + i], P, P.qm);
        if (qp.k != K_INVALID) acc += (double)(0.5f * P.C_s * ni * ni / (qp.q * qp.q * qp.q));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void k_delta_energy_sum(const double* __restrict__ partials, int nb, double dOmega,
                                   double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partials[b];
    *out = dOmega * s;
}

// Device address of the scratch on the current device (looked up once per device).
int scratch_pointer(double** p) {
    int dev = 0;
    VDW_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("device index beyond the no-alloc scratch table");
        return VDW_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partials)");
        g_dev_ptr[dev] = static_cast<double*>(ptr);
    }
    *p = g_dev_ptr[dev];
    return VDW_OK;
}

}  // namespace
}  // namespace vdw

using namespace vdw;

extern "C" int vdw_delta_energy_noalloc(vdw_handle h, const float* n, const float* grad, long long npoints,
                                        double dOmega, double* dE, void* stream) {
    if (!h || !n || !grad || !dE || npoints <= 0 || !(dOmega > 0.0)) return VDW_ERR_ARG;
    if (npoints > VDW_NOALLOC_MAX_POINTS) {
        set_error("vdw_delta_energy_noalloc: more points than its fixed scratch covers (max 16777216)");
        return VDW_ERR_SIZE;
    }
    double* partials = nullptr;
    const int rc = scratch_pointer(&partials);
    if (rc) return rc;
    const int nb = (int)((npoints + NA_PTS_PER_BLOCK - 1) / NA_PTS_PER_BLOCK);
    cudaStream_t s = (cudaStream_t)stream;
    k_delta_energy_blocks<<<nb, NA_THREADS, 0, s>>>(n, grad, npoints, h->pp, partials);
    k_delta_energy_sum<<<1, 32, 0, s>>>(partials, nb, dOmega, dE);
    VDW_CUDA(cudaGetLastError());
    return VDW_OK;
}
