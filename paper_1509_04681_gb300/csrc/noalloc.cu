// cggm_lambda_sweep_noalloc: the Lambda coordinate pass for callers that must not
// allocate device memory.  Its working memory is one file-scope device array.
#include <mutex>

#include "common.cuh"
#include "dense.cuh"
#include "iter.cuh"
#include "sweeps.cuh"

using namespace cggm;

namespace {

constexpr int64_t kMaxQ = CGGM_NOALLOC_MAX_Q;
constexpr int kBatch = 64;
// Byte offsets of the regions inside the array (each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_G = 0;                                                   // q x q double
constexpr size_t OFF_U = align256(OFF_G + 8 * kMaxQ * kMaxQ);                 // q x q double
constexpr size_t OFF_SD = align256(OFF_U + 8 * kMaxQ * kMaxQ);                // q double
constexpr size_t OFF_PD = align256(OFF_SD + 8 * kMaxQ);                       // q double
constexpr size_t OFF_MU = align256(OFF_PD + 8 * kMaxQ);                       // 2 B double
constexpr size_t OFF_SUB1 = align256(OFF_MU + 8 * 2 * kBatch);                // step constants
constexpr size_t kSub1 = scratch_sub1_bytes(kBatch, sizeof(double));
constexpr size_t OFF_SUB2 = align256(OFF_SUB1 + kSub1);                       // coefficients
constexpr size_t kSub2 = scratch_sub2_bytes(kBatch, sizeof(double));
constexpr size_t OFF_BAR = align256(OFF_SUB2 + kSub2);                        // barrier
constexpr size_t OFF_ERR = align256(OFF_BAR + sizeof(GridBarrier));
constexpr size_t kBytes = align256(OFF_ERR + sizeof(int));
static_assert(kBytes <= (size_t)CGGM_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds its size");

// The scratch array.  Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_scratch[CGGM_NOALLOC_SCRATCH_BYTES];

// Device address of g_scratch per device, taken once with that device current (the host
// name of the array is only a stand-in for it).
constexpr int kMaxDevices = 64;
unsigned char *g_base[kMaxDevices] = {};
std::mutex g_mutex;

cggm_status scratch_base(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return CGGM_EINVAL;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_base[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return CGGM_ECUDA;
        }
        g_base[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_base[dev];
    return CGGM_OK;
}

// Every active coordinate must satisfy 0 <= ai <= aj < q: the pass indexes its q x q
// matrices with them unchecked.  A bad pair sets the status word.
__global__ void check_pairs_kernel(int64_t m, const int32_t *__restrict__ ai,
                                   const int32_t *__restrict__ aj, int64_t q, int *err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = ai[k], b = aj[k];
        if (a < 0 || a > b || b >= q) {
            atomicCAS(err, 0, (int)DEV_BADINDEX);
            return;
        }
    }
}

bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) &&
           a.device == dev;
}

}  // namespace

extern "C" cggm_status cggm_lambda_sweep_noalloc(int64_t q, const double *Sigma,
                                                 const double *Psi, const double *Syy,
                                                 const double *Lambda, int64_t m,
                                                 const int32_t *ai, const int32_t *aj,
                                                 double lam_L, int penalize_diag,
                                                 double *D_out, void *cuda_stream) {
    if (q < 1 || q > kMaxQ || m < 0 || m > q * (q + 1) / 2) return CGGM_EINVAL;
    if (!Sigma || !Psi || !Syy || !Lambda || !D_out || (m > 0 && (!ai || !aj)))
        return CGGM_EINVAL;
    if (!(lam_L >= 0.0)) return CGGM_EINVAL;
    int dev = 0;
    CGGM_CUDA_TRY(cudaGetDevice(&dev));
    const void *ptrs[] = {Sigma, Psi, Syy, Lambda, D_out};
    for (const void *p : ptrs)
        if (!on_device(p, dev)) return CGGM_EINVAL;
    if (m > 0 && (!on_device(ai, dev) || !on_device(aj, dev))) return CGGM_EINVAL;
    unsigned char *base = nullptr;
    CGGM_TRY(scratch_base(dev, &base));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    double *G = reinterpret_cast<double *>(base + OFF_G);
    double *U = reinterpret_cast<double *>(base + OFF_U);
    double *Sd = reinterpret_cast<double *>(base + OFF_SD);
    double *Pd = reinterpret_cast<double *>(base + OFF_PD);
    SweepScratch scr;
    scr.mu = reinterpret_cast<double *>(base + OFF_MU);
    scr.sub1 = base + OFF_SUB1;
    scr.sub2 = base + OFF_SUB2;
    scr.bar = reinterpret_cast<GridBarrier *>(base + OFF_BAR);
    scr.err = reinterpret_cast<int *>(base + OFF_ERR);

    // What must start at zero: the direction and the cache U = D Sigma.  The gradient,
    // and the diagonals are rewritten in full below.
    const size_t qq = (size_t)q * q;
    CGGM_CUDA_TRY(cudaMemsetAsync(D_out, 0, 8 * qq, st));
    if (m == 0) {  // the direction is zero; return once it has been written
        CGGM_CUDA_TRY(cudaStreamSynchronize(st));
        return CGGM_OK;
    }
    // the coordinate list is checked on the device before the pass reads it
    int bad = 0;
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    note_launch();
    check_pairs_kernel<<<(unsigned)((m + 255) / 256 < 64 ? (m + 255) / 256 : 64), 256, 0, st>>>(
        m, ai, aj, q, scr.err);
    CGGM_CUDA_TRY(cudaGetLastError());
    CGGM_CUDA_TRY(cudaMemcpyAsync(&bad, scr.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CGGM_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad != 0) return CGGM_EINVAL;
    CGGM_CUDA_TRY(cudaMemsetAsync(U, 0, 8 * qq, st));
    grad_lambda<double>(q, Syy, Sigma, Psi, G, st);
    diag_to_double<double>(q, Sigma, Sd, st);
    diag_to_double<double>(q, Psi, Pd, st);
    CGGM_CUDA_TRY(cudaGetLastError());
    const double lamd = penalize_diag ? lam_L : 0.0;
    return lambda_sweep_preplanned_f64(q, Sigma, Psi, Sd, Pd, G, Lambda, m, ai, aj, lam_L,
                                       lamd, D_out, U, kBatch, scr, st);
}
