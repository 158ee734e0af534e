// Inputs of the solve (Section 2.1).  The paper's genomic inputs (Section 5.2) are genotypes, counts in
// {0, 1, 2} per individual and marker; stored as int8 they take an eighth of the bytes of
// the double matrix the solver works on, and the standardisation (per-column mean and
// population standard deviation, which makes diag(S_xx) = 1) runs on the device.
#include <cuda_bf16.h>

#include "load.cuh"

namespace cggm {

namespace {

// sum and sum of squares of each column of an int8 rows x cols matrix (exact in int64),
// then mean and 1 / population sd (0 for a constant column)
__global__ void colstats_i8_kernel(int64_t rows, int64_t cols, const int8_t *__restrict__ X,
                                   double *mean, double *inv_sd) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cols) return;
    long long s = 0, s2 = 0;
    for (int64_t i = 0; i < rows; i++) {
        const int v = X[i * cols + k];
        s += v;
        s2 += (long long)v * v;
    }
    const double n = (double)rows;
    const double mu = (double)s / n;
    // population variance from the exact integer sums: (n s2 - s^2) / n^2
    const double var = ((double)s2 * n - (double)s * (double)s) / (n * n);
    mean[k] = mu;
    inv_sd[k] = var > 0.0 ? 1.0 / sqrt(var) : 0.0;
}

// 32 x 32 tiles through shared memory: coalesced reads of src rows, coalesced writes of
// dst rows.  Element conversion by Conv.
template <typename Tin, typename Conv>
__global__ void transpose_to_double_kernel(int64_t rows, int64_t cols, const Tin *__restrict__ in,
                                           double *__restrict__ out, Conv conv) {
    __shared__ double tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = conv(in[r * cols + c], c);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][k];
    }
}

struct StdI8 {
    const double *mean, *inv_sd;
    __device__ double operator()(int8_t v, int64_t c) const {
        return ((double)v - mean[c]) * inv_sd[c];
    }
};

struct FromBF16 {
    __device__ double operator()(__nv_bfloat16 v, int64_t) const {
        return (double)__bfloat162float(v);
    }
};

template <typename Tin, typename Conv>
void launch_transpose(int64_t rows, int64_t cols, const Tin *in, double *out, Conv conv,
                      cudaStream_t st) {
    dim3 grid(ceil_div(cols, 32), ceil_div(rows, 32)), block(32, 8);
    note_launch();
    transpose_to_double_kernel<Tin, Conv><<<grid, block, 0, st>>>(rows, cols, in, out, conv);
}

}  // namespace

size_t dtype_size(int dt) {
    switch (dt) {
        case CGGM_F32: return 4;
        case CGGM_F64: return 8;
        case CGGM_BF16: return 2;
        case CGGM_I8_GENO: return 1;
        default: return 0;
    }
}

cggm_status load_input_transposed(const void *src, int dt, int64_t rows, int64_t cols,
                                  double *dst, double *stats, cudaStream_t st) {
    if (dt == CGGM_BF16) {
        launch_transpose(rows, cols, static_cast<const __nv_bfloat16 *>(src), dst, FromBF16{}, st);
    } else if (dt == CGGM_I8_GENO) {
        if (!stats) return CGGM_EINVAL;
        note_launch();
        colstats_i8_kernel<<<ceil_div(cols, 128), 128, 0, st>>>(
            rows, cols, static_cast<const int8_t *>(src), stats, stats + cols);
        launch_transpose(rows, cols, static_cast<const int8_t *>(src), dst,
                         StdI8{stats, stats + cols}, st);
    } else {
        return CGGM_EINVAL;
    }
    CGGM_CUDA_TRY(cudaGetLastError());
    return CGGM_OK;
}

}  // namespace cggm
