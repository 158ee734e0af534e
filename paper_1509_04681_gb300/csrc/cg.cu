// Conjugate gradient on a sparse symmetric positive definite matrix with many right-hand
// sides at once (Section 4 computes blocks of Sigma = Lambda^-1 by CG on the sparse Lambda).
// Right-hand sides are the columns of a row-major q x k block, so that the sparse product
// A P reads and writes whole rows of k contiguous values; per-column scalars (p^T A p,
// r^T z, r^T r) are reduced over fixed row chunks and then over the chunks in order, so
// the result does not depend on scheduling.
#include "cg.cuh"

#include <cmath>

namespace cggm {

namespace {

enum { COL_RZ, COL_ALPHA, COL_BETA, COL_BNORM, COL_RES, COL_SPARE, COL_N };

__global__ void csr_check_kernel(int64_t q, int64_t nnz, const int64_t *row_ptr,
                                 const int32_t *col, int *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= q; i += stride) {
        const int64_t a = row_ptr[i];
        if (a < 0 || a > nnz || (i == 0 && a != 0) || (i == q && a != nnz) ||
            (i > 0 && row_ptr[i - 1] > a))
            atomicCAS(err, 0, (int)DEV_BADINDEX);
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
        if (col[e] < 0 || col[e] >= q) atomicCAS(err, 0, (int)DEV_BADINDEX);
}

// dinv[i] = 1 / A_ii; a missing or non-positive diagonal is not positive definite
__global__ void jacobi_kernel(int64_t q, const int64_t *row_ptr, const int32_t *col,
                              const double *val, double *dinv, int *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < q;
         i += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++)
            if (col[e] == i) d += val[e];
        if (!(d > 0.0)) {
            atomicCAS(err, 0, (int)DEV_NOTPD);
            d = 1.0;
        }
        dinv[i] = 1.0 / d;
    }
}

// X = 0, R = B, Z = D^-1 R, P = Z
__global__ void init_kernel(int64_t q, int64_t k, const double *B, int64_t c0, const double *dinv,
                            double *X, double *R, double *Z, double *P) {
    const int64_t total = q * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k, c = e - i * k;
        const double b = B ? B[e] : (i == c0 + c ? 1.0 : 0.0);
        X[e] = 0.0;
        R[e] = b;
        const double z = dinv[i] * b;
        Z[e] = z;
        P[e] = z;
    }
}

// AP = A P: block row i (grid-stride over rows), threads over the k columns
__global__ void spmm_kernel(int64_t q, int64_t k, const int64_t *row_ptr, const int32_t *col,
                            const double *val, const double *__restrict__ P,
                            double *__restrict__ AP) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    for (int64_t i = blockIdx.y; i < q; i += gridDim.y) {
        double s = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) s = fma(val[e], P[col[e] * k + c], s);
        AP[i * k + c] = s;
    }
}

// part[(chunk * 2 + t) * k + c] = sum over the chunk's rows of A_t[r][c] B_t[r][c] (t = 0, 1)
__global__ void coldot2_kernel(int64_t q, int64_t k, const double *A0, const double *B0,
                               const double *A1, const double *B1, double *part) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    const int64_t rows = (q + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = (int64_t)blockIdx.y * rows, r1 = (r0 + rows) < q ? (r0 + rows) : q;
    double s0 = 0.0, s1 = 0.0;
    for (int64_t r = r0; r < r1; r++) {
        s0 = fma(A0[r * k + c], B0[r * k + c], s0);
        if (A1) s1 = fma(A1[r * k + c], B1[r * k + c], s1);
    }
    part[(blockIdx.y * 2 + 0) * k + c] = s0;
    part[(blockIdx.y * 2 + 1) * k + c] = s1;
}

__device__ __forceinline__ double chunk_sum(const double *part, int64_t k, int64_t c, int t) {
    double s = 0.0;
    for (int ch = 0; ch < kCgChunks; ch++) s += part[(ch * 2 + t) * k + c];
    return s;
}

// after the initial dots (r.z, r.r): r.z and |b|
__global__ void start_kernel(int64_t k, const double *part, double *colv) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < k;
         c += (int64_t)gridDim.x * blockDim.x) {
        colv[COL_RZ * k + c] = chunk_sum(part, k, c, 0);
        const double bn = sqrt(chunk_sum(part, k, c, 1));
        colv[COL_BNORM * k + c] = bn;
    }
}

// alpha = r.z / p.Ap (0 for a column already at zero residual)
__global__ void alpha_kernel(int64_t k, const double *part, double *colv, int *err) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < k;
         c += (int64_t)gridDim.x * blockDim.x) {
        const double pap = chunk_sum(part, k, c, 0);
        const double rz = colv[COL_RZ * k + c];
        double a = 0.0;
        if (rz > 0.0) {
            if (!(pap > 0.0)) atomicCAS(err, 0, (int)DEV_NOTPD);
            else a = rz / pap;
        }
        colv[COL_ALPHA * k + c] = a;
    }
}

// X += alpha P, R -= alpha AP, Z = D^-1 R
__global__ void update1_kernel(int64_t q, int64_t k, const double *colv, const double *dinv,
                               const double *P, const double *AP, double *X, double *R, double *Z) {
    const int64_t total = q * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k, c = e - i * k;
        const double a = colv[COL_ALPHA * k + c];
        X[e] = fma(a, P[e], X[e]);
        const double r = fma(-a, AP[e], R[e]);
        R[e] = r;
        Z[e] = dinv[i] * r;
    }
}

// beta = r'.z' / r.z, the residual ratios; one block writes their maximum to *res_max
__global__ void beta_kernel(int64_t k, const double *part, double *colv, double *res_max) {
    __shared__ double red[1024];
    double m = 0.0;
    for (int64_t c = threadIdx.x; c < k; c += blockDim.x) {
        const double rz_new = chunk_sum(part, k, c, 0);
        const double rr = chunk_sum(part, k, c, 1);
        const double rz = colv[COL_RZ * k + c];
        colv[COL_BETA * k + c] = rz > 0.0 ? rz_new / rz : 0.0;
        colv[COL_RZ * k + c] = rz_new;
        const double bn = colv[COL_BNORM * k + c];
        const double res = bn > 0.0 ? sqrt(rr) / bn : 0.0;
        colv[COL_RES * k + c] = res;
        m = fmax(m, res);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h /= 2) {
        if ((int)threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *res_max = red[0];
}

// P = Z + beta P
__global__ void update2_kernel(int64_t q, int64_t k, const double *colv, const double *Z, double *P) {
    const int64_t total = q * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e % k;
        P[e] = fma(colv[COL_BETA * k + c], P[e], Z[e]);
    }
}

unsigned grid_elems(int64_t n) {
    const int64_t g = (n + 255) / 256, cap = (int64_t)sm_count() * 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

cggm_status read_status(int *err, cudaStream_t st) {
    int h = 0;
    CGGM_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CGGM_CUDA_TRY(cudaStreamSynchronize(st));
    if (h == DEV_NOTPD) return CGGM_ENOTPD;
    if (h != 0) return CGGM_EINVAL;
    return CGGM_OK;
}

}  // namespace

size_t cg_work_doubles(int64_t q, int64_t k) {
    return 4 * (size_t)q * k + (size_t)q + COL_N * (size_t)k + 2 * (size_t)kCgChunks * k + 8;
}

CgWork cg_work_at(double *base, int *err, int64_t q, int64_t k) {
    CgWork w;
    const size_t qk = (size_t)q * k;
    w.R = base;
    w.Z = w.R + qk;
    w.P = w.Z + qk;
    w.AP = w.P + qk;
    w.dinv = w.AP + qk;
    w.col = w.dinv + q;
    w.part = w.col + COL_N * (size_t)k;
    w.err = err;
    return w;
}

cggm_status csr_check(int64_t q, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                      int *err, cudaStream_t st) {
    CGGM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    note_launch();
    csr_check_kernel<<<grid_elems(q + 1 > nnz ? q + 1 : nnz), 256, 0, st>>>(q, nnz, row_ptr, col, err);
    CGGM_CUDA_TRY(cudaGetLastError());
    return read_status(err, st);
}

cggm_status pcg_solve(int64_t q, const int64_t *row_ptr, const int32_t *col, const double *val,
                      int64_t k, const double *B, int64_t c0, double tol, int max_iter,
                      double *X, CgWork w, int *iters, double *resid, cudaStream_t st) {
    const unsigned ge = grid_elems(q * k);
    const dim3 gcol(ceil_div(k, 128), kCgChunks), gsp(ceil_div(k, 128), (unsigned)(q < 65535 ? q : 65535));
    double *res_max = w.col + COL_SPARE * k;
    CGGM_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    note_launch();
    jacobi_kernel<<<grid_elems(q), 256, 0, st>>>(q, row_ptr, col, val, w.dinv, w.err);
    note_launch();
    init_kernel<<<ge, 256, 0, st>>>(q, k, B, c0, w.dinv, X, w.R, w.Z, w.P);
    note_launch();
    coldot2_kernel<<<gcol, 128, 0, st>>>(q, k, w.R, w.Z, w.R, w.R, w.part);
    note_launch();
    start_kernel<<<grid_elems(k), 256, 0, st>>>(k, w.part, w.col);
    CGGM_CUDA_TRY(cudaGetLastError());
    CGGM_TRY(read_status(w.err, st));
    // the starting ratios (1, or 0 for a zero right-hand side) and their maximum; run on the
    // initial dots, the kernel leaves r.z as it is
    double h_res = 0.0;
    note_launch();
    beta_kernel<<<1, 1024, 0, st>>>(k, w.part, w.col, res_max);
    CGGM_CUDA_TRY(cudaMemcpyAsync(&h_res, res_max, sizeof(double), cudaMemcpyDeviceToHost, st));
    CGGM_CUDA_TRY(cudaStreamSynchronize(st));
    int it = 0;
    while (!(h_res <= tol) && it < max_iter) {
        note_launch();
        spmm_kernel<<<gsp, 128, 0, st>>>(q, k, row_ptr, col, val, w.P, w.AP);
        note_launch();
        coldot2_kernel<<<gcol, 128, 0, st>>>(q, k, w.P, w.AP, nullptr, nullptr, w.part);
        note_launch();
        alpha_kernel<<<grid_elems(k), 256, 0, st>>>(k, w.part, w.col, w.err);
        note_launch();
        update1_kernel<<<ge, 256, 0, st>>>(q, k, w.col, w.dinv, w.P, w.AP, X, w.R, w.Z);
        note_launch();
        coldot2_kernel<<<gcol, 128, 0, st>>>(q, k, w.R, w.Z, w.R, w.R, w.part);
        note_launch();
        beta_kernel<<<1, 1024, 0, st>>>(k, w.part, w.col, res_max);
        note_launch();
        update2_kernel<<<ge, 256, 0, st>>>(q, k, w.col, w.Z, w.P);
        CGGM_CUDA_TRY(cudaGetLastError());
        CGGM_CUDA_TRY(cudaMemcpyAsync(&h_res, res_max, sizeof(double), cudaMemcpyDeviceToHost, st));
        CGGM_TRY(read_status(w.err, st));
        it++;
        if (!std::isfinite(h_res)) return CGGM_ENONFINITE;
    }
    if (iters) *iters = it;
    if (resid) *resid = h_res;
    return h_res <= tol ? CGGM_OK : CGGM_EMAXITER;
}

}  // namespace cggm
