// Shared definitions of the vdwnl CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>

#include "../../include/vdwnl.h"

namespace vdw {

// Stages of one call, for vdw_profile_read (include/vdwnl.h lists them).
enum Stage {
    ST_POINTWISE = 0,
    ST_PLANES_FWD,
    ST_PENCILS_FWD,
    ST_CONTRACT,
    ST_ENERGY,
    ST_PENCILS_INV,
    ST_PLANES_INV,
    ST_USUM,
    ST_W_PLANES,
    ST_PENCIL_DIV,
    ST_DIV_FINAL,
    ST_COUNT
};
static_assert(ST_COUNT == VDW_NSTAGES, "stage list");

constexpr int MAX_NQ = 32;     // largest interpolation mesh the kernels take
constexpr int MAX_MC = 32;     // largest order m_c of the saturation sum of Eq. (Sat)
constexpr int MAX_DIM = 256;   // largest grid dimension (FFT line length)
constexpr uint8_t K_INVALID = 255;  // interval code of a point with theta = 0

// Radix schedule of one line length: Stockham passes of radix 4 (c4 times),
// then 2, 3 and 5, with n = 4^c4 2^c2 3^c3 5^c5.
struct LinePlan {
    int n;
    int c4, c2, c3, c5;
};

// Pointwise constants, passed by value (kernel parameter space).
struct PointParams {
    int Nq;
    int m_c;
    float q_c;
    float n_min;
    float C_s;
    float inv_m[MAX_MC + 1];     // 1/m, m = 1 .. m_c (terms of the saturation sum)
    float qm[MAX_NQ];            // q mesh
    float Mq[MAX_NQ][MAX_NQ];    // Mq[a][k]: second derivative of p_a at knot k
};

// Grid geometry shared by the plane and pencil kernels.
struct GridArgs {
    int N1, N2, N3, Nh;    // Nh = N1/2 + 1
    long long N;           // N1 N2 N3
    int ncols;             // N3 * Nh: columns of the half spectrum per y
    float gx2, gy2, gz2;   // (2 pi / L_d)^2
    float gx, gy, gz;      // 2 pi / L_d
    float inv_dk;          // 1 / Delta k of the radial table
    int Nk;                // points of the radial table
    float invN;            // 1 / N
    LinePlan p1, p2, p3;   // line transforms along x, y, z
    // Flat-index divisions by N1, N2 and N3/2 as multiply-high by
    // m = ceil(2^32 / d), exact for i d < 2^32; fast = 0 (plain division)
    // when N max(N1, N2, N3) reaches 2^32 or a divisor is 1.
    unsigned m1, m2, mh3;
    int fast;
    // batches (vdw_energy_potential_batched): density b of a batch uses the
    // workspaces at these element offsets times b; the kernels take b from
    // their last grid dimension (0 for a single density)
    long long bs_spec;   // float2 values between two densities' spectrum buffers
    long long bs_wspec;  // float2 values between two w-spectrum buffers
    long long bs_Q;      // float4 values between two record buffers (contract.cu)
    int bs_epart;        // energy partial sums per density
};

// Learned reduced basis: sizes fixed at compile time.
constexpr int LRN_H = 64;                          // hidden units of the channel network
constexpr int LRN_M = 8;                           // channels
constexpr int LRN_P = LRN_M * (LRN_M + 1) / 2;     // learned pair kernels m <= n
constexpr int LRN_N3 = 16;                         // last layer padded to a legal MMA width
// offsets in the flat parameter vector: W1 [H][2], b1, W2 [H][H], b2, W3 [M][H], b3, K [P][J]
constexpr int LRN_OFF_W1 = 0;
constexpr int LRN_OFF_B1 = LRN_OFF_W1 + LRN_H * 2;
constexpr int LRN_OFF_W2 = LRN_OFF_B1 + LRN_H;
constexpr int LRN_OFF_B2 = LRN_OFF_W2 + LRN_H * LRN_H;
constexpr int LRN_OFF_W3 = LRN_OFF_B2 + LRN_H;
constexpr int LRN_OFF_B3 = LRN_OFF_W3 + LRN_M * LRN_H;
constexpr int LRN_OFF_K = LRN_OFF_B3 + LRN_M;

// Device view of a loaded learned model (kernel parameter).  The bf16
// operands are stored in the tensor-core layout (tc.cuh) as raw 16-bit words.
struct LearnedArgs {
    int J;                  // knots
    float dk, inv_dk;       // knot spacing and its inverse
    float mu1, inv_sig1, mu2, inv_sig2, eps2;  // feature standardisation, eps^2
    const float* w1;        // [H][2] bf16-rounded values
    const float* b1;        // [H]
    const float* b2;        // [H]
    const float* b3;        // [M]
    const uint16_t* w2f;    // forward operand W2 [H out][H in]
    const uint16_t* w3f;    // forward operand W3 [16 (M padded)][H]
    const float* w2r;       // W2 bf16-rounded values, row-major [H][H] (CUDA-core kernels)
    const float* w3r;       // W3 bf16-rounded values, row-major [M][H]
    const float4* knots;    // [J-1][P]: cubic coefficients in t of the Catmull-Rom piece on interval j
    int* err;               // set when a tensor-core wait gives up
    int base;               // channel weights = spline base + network (1) or network alone (0)
    // the network tabulated on the feature nodes (vdw_learned_tabulate): node
    // (i1, i2), i = 0 .. T + 1, at x = -D + (i - 1) h, its 8 outputs at
    // node (i1, i2): channels 0-3 at tab[i1 (T + 2) + i2], 4-7 at the same
    // index + (T + 2)^2; tabT = 0: no table
    const float4* tab;
    int tabT;
    float tabD, tab_h, tab_inv_h;
    float bqm[LRN_M];       // base mesh
    float bMq[LRN_M * LRN_M];  // bMq[m * M + k]: second derivative of base spline m at knot k
};

}  // namespace vdw

// The context behind the opaque vdw_handle.
struct vdw_ctx {
    vdw_params p;
    int device;
    // tables
    vdw::PointParams pp;        // host copy of the pointwise constants
    double phi0, C_s;
    float4* d_kcoef;            // [Nk-1][npairs] cubic coefficients in local t
    // plan
    int planned;
    vdw::GridArgs g;
    double L[3];
    float4* d_tw;               // twiddles (hi/lo pairs): N1, N2, N3 entries
    float2* d_spec;             // [Nq][N2][N3][Nh] theta(G), then u(G), then real u (N3 x N1 per plane), in place
    float2* d_wspec;            // [3][N2][N3][Nh] w(G); component 0 then D.w
    float* d_t;                 // [N] position of q inside its mesh interval
    uint8_t* d_k;               // [N] mesh interval of q (K_INVALID: theta = 0)
    float4* d_aux;              // [N] n dq/dn, n dq/d|grad n| / |grad n|, and the Delta E derivatives
    double* d_epart;            // per-block energy partial sums
    int nb_point;               // their count for the pointwise kernel
    // points of the half spectrum in |G| order (contract.cu)
    long long nG, Npad;         // N2 N3 (N1/2 + 1), rounded up to whole contraction blocks
    int nb_sorted;              // contraction blocks (and energy partials)
    unsigned* d_pos;            // [N3 Nh][N2] sorted position of point (col, y)
    float* d_gs;                // [Npad] |G| of each sorted point, sign = energy weight
    float4* d_Q;                // [Nq/4][Npad][2] field quads of the sorted points
    int batch_max;              // densities the per-density workspaces hold (vdw_plan_batch)
    int nsm;                    // SMs of the device (persistent grids)
    int usum_per_sm;            // resident blocks per SM of the field-sum kernel
    // the pointwise pass runs in p0_chunks slabs of p0_nj complex rows (2 p0_nj
    // z values) with nb_p0 blocks each, so that the host entry point can copy
    // slab c + 1 while slab c is processed (nb_point = p0_chunks * nb_p0)
    int p0_chunks, p0_nj, nb_p0;
    unsigned p0_mnj;            // ceil(2^32 / p0_nj) (multiply-high division)
    cudaStream_t s_copy;        // copy stream of the host entry point
    cudaEvent_t ev_in;          // orders the copy stream after the caller's stream
    cudaEvent_t ev_slab[4];     // slab c of the inputs is on the device
    cudaStream_t s_side;        // the energy reduction beside the inverse transforms
    cudaEvent_t ev_fork, ev_join;
    unsigned long long* d_invalid;  // count of negative / non-finite densities
    int bulk_planes;            // inverse plane transforms load their planes by bulk copies
    float* d_gg;                // [N] g of w = g grad n (assembly -> w plane transforms)
    // give-up flags of the bounded waits, in mapped page-locked host memory so
    // that an entry point can read them without synchronising: [0] the bulk
    // copies of the plane kernels, [1] the tensor-core waits of the learned path
    int* h_flags;               // host view
    int* d_flags;               // device view of the same two words
    int wait_seen;              // a give-up was reported since vdw_plan
    double* d_xc;               // [4 + 2 XC_BLOCKS] nonlocal E and semilocal partial sums
    // buffers of the host-pointer entry point (allocated on first use)
    float* d_in;                // [4N]
    float* d_v;                 // [N]
    double* d_E;                // [3]
    float* d_gtmp;              // [3N] spectral gradient when the caller passes none
    size_t bytes;
    // learned reduced basis (vdw_learned_load)
    int lrn_loaded;
    int lrn_J;
    double lrn_kmax;
    void* d_lrn;                // one allocation behind the LearnedArgs pointers
    vdw::LearnedArgs la;
    float* d_U;                 // [M][N] real-space u_m for the parameter gradient (on first use)
    float* d_lw;                // [2M + 2][N] per-point coefficients of the learned assembly (on first use)
    double* d_gK;               // [P][J] knot-gradient accumulator (on first use)
    float4* d_lrn_tab;          // the tabulated network (vdw_learned_tabulate)
    size_t lrn_tab_bytes;
    // per-stage timing (vdw_profile_enable)
    int prof;
    cudaEvent_t ev[VDW_NSTAGES + 1];
    int ev_done[VDW_NSTAGES];
};

namespace vdw {

void set_error(const std::string& s);
int cuda_fail(cudaError_t e, const char* what);
// VDW_ERR_TIMEOUT (and clears the flags) if a kernel of an earlier call gave up
// a bounded wait since the last check, else VDW_OK
int check_wait(vdw_ctx* c);
// per-density workspaces for Bmax densities (api.cu)
int alloc_density_work(vdw_ctx* c, int Bmax);

#define VDW_CUDA(call)                                         \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return ::vdw::cuda_fail(_e, #call); \
    } while (0)

// Serialises raise_smem_limit across threads (api.cu).
void smem_limit_lock(bool lock);

// Raises (never lowers) a kernel's dynamic shared-memory limit to bytes.
// The limit belongs to the kernel, for the whole process, not to a context:
// contexts of different grids (or learned models of different knot counts)
// that share a kernel would otherwise lower each other's limit, and their
// launches would then fail.
template <class K>
int raise_smem_limit(K kernel, size_t bytes) {
    smem_limit_lock(true);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < bytes)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    smem_limit_lock(false);
    if (e != cudaSuccess) return cuda_fail(e, "raise_smem_limit");
    return VDW_OK;
}

// pipeline launchers (pipeline.cu)
// slab_ready (optional): per slab of the pointwise pass, an event to wait on
// before processing it (the host entry point's copies)
// B > 1: a batch of B densities (n [B][N], grad [B][3][N], E [B][3], v [B][N],
// w [B][3][N]), one launch per stage; needs the batch workspaces of vdw_plan_batch
int pipeline_run(vdw_ctx* c, const float* n, const float* grad, double* E, float* v, float* w,
                 cudaStream_t s, int fd = 0, int xc = 0, const cudaEvent_t* slab_ready = nullptr, int B = 1);
// E[4] of the functional from the nonlocal energy (d_xc[0]) and the semilocal sums
int pipeline_xc_final(vdw_ctx* c, double* E, cudaStream_t s);
// central-difference gradient of a field (into grad [3][N])
int pipeline_stencil_gradient(vdw_ctx* c, const float* f, float* grad, cudaStream_t s);
int pipeline_plan_check(vdw_ctx* c, size_t* smem_plane, size_t* smem_pencil, size_t* smem_assemble,
                        size_t* smem_div);
int pipeline_make_twiddles(vdw_ctx* c);
int pipeline_configure(vdw_ctx* c);
// the divergence term of a potential (w(G) in d_wspec) and the energy reduction
int pipeline_divergence(vdw_ctx* c, float* v, cudaStream_t s);
// in-place plane transforms of the first nfields fields of d_spec: inverse
// (half spectrum -> N3 x N1 real rows at the start of each plane) or forward
// (packed real rows -> half spectrum)
int pipeline_planes_inplace(vdw_ctx* c, int nfields, bool inverse, cudaStream_t s);
// forward plane transforms of w = g grad n with g in d_gg (into d_wspec)
int pipeline_w_planes(vdw_ctx* c, const float* grad, cudaStream_t s);
int pipeline_energy_final(vdw_ctx* c, const double* epart, int nb0, int nb2, double* E, cudaStream_t s);

// y transforms and contraction in |G| order (contract.cu)
size_t sorted_pencil_smem(const GridArgs& g);
int sorted_plan(vdw_ctx* c);
void sorted_free(vdw_ctx* c);
int sorted_configure(vdw_ctx* c);
int sorted_forward(vdw_ctx* c, int nfields, cudaStream_t s, int B = 1);
int sorted_inverse(vdw_ctx* c, int nfields, cudaStream_t s, int B = 1);
int sorted_contract(vdw_ctx* c, double* epart, int write_back, cudaStream_t s, int B = 1);
// the same contraction of the first nq fields with another table of the same
// layout ([nk-1][nq(nq+1)/2] float4 cubic coefficients on a uniform mesh)
int sorted_contract_table(vdw_ctx* c, int nq, const float4* table, float inv_dk, int nk, double* epart,
                          int write_back, cudaStream_t s, int B = 1);
constexpr int SORTED_BLOCK = 128;  // sorted points per contraction block
// The energy's partial sums (one per block of the pointwise pass and of the
// contraction) are reduced in two passes: EPART_SPLIT blocks each sum a fixed
// contiguous share of both arrays, one block sums their EPART_SPLIT results in
// index order.  The per-density partial-sum array ends with those 2
// EPART_SPLIT values.
constexpr int EPART_SPLIT = 64;

// learned reduced basis (learned.cu)
int learned_run(vdw_ctx* c, const float* n, const float* grad, double* E, float* v, float* w, cudaStream_t s);
void learned_free(vdw_ctx* c);

// table launchers (table.cu)
int table_build(const vdw_params* p, double* h_qmesh, double* h_phik, double* phi0, double* C_s);
int table_upload(vdw_ctx* c, const double* h_phik, double C_s);

int make_line_plan(int n, LinePlan* lp);

}  // namespace vdw
